// Split-precision DFT-as-GEMM linear sub-step on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), inside a persistent overlap-save DBP
// kernel.  Precision variant of the linear sub-step of Section II (Eq. 1) with
// N = NB * NA, NA = 64, n = na + NA nb, k = kb + NB ka:
//   SIMT    NB-point DFTs over nb of every (block, polarization, na) column, twiddle
//           W_N^{na kb}                                                       (FP32)
//   GEMM 1  X[kb + NB ka] = sum_na u(kb, na) W_NA^{na ka}: rows (block, pol, kb), the
//           complex product as a real one [Re u | Im u] x [[C, S], [-S, C]]
//           (C = cos, S = -sin of 2 pi na ka / NA), M = 128, N = 128, K = 128
//   SIMT    Y = X H_s (1/N folded in, natural frequency order), in the GEMM-1 output
//           layout (each tensor-memory lane holds one row)                   (FP32)
//   GEMM 2  y'(kb, na) = sum_ka Y(kb + NB ka) W_NA^{-na ka}: the same real matrix
//           transposed ([[C, -S], [S, C]], C and S are symmetric), read from the same
//           shared-memory bytes as an MN-major operand
//   SIMT    conjugate twiddle W_N^{-na kb}, NB-point inverse DFTs over kb     (FP32)
// then the nonlinear sub-step (Eqs. 2-3) in FP32.  Every GEMM operand is split into two
// parts of the 16-bit type, x = hi + lo (hi the rounding of x, lo that of the
// remainder), and three products are accumulated in FP32 in two TMEM accumulators,
// D_hh = A_hi B_hi and D_x = A_hi B_lo + A_lo B_hi (so that the small cross terms round
// at their own magnitude), added once on readback.  Before each GEMM the tile is scaled
// by a power of two (exact) so that its largest possible value is about 2^12: no value
// can overflow FP16, the remainders of all but negligibly small values stay normal, and
// a hi + lo pair keeps ~22 significant bits (BF16: ~16).
//
// One CTA (256 threads) owns one 128-row tile at a time: G = 64 / NB overlap-save
// blocks, both polarizations.  Shared memory: the time-domain tile (float2
// [G][2][N]); the GEMM A operand (hi and lo, 32 KB each), which also holds the spectrum
// rows between GEMM 2 and the inverse DFTs and the intensity P of the nonlinear step;
// the DFT matrix hi / lo (64 KB, copied once per CTA); H_s; the taps.  Tensor memory:
// 512 columns: D_hh in 0-127, D_x in 128-255, each thread's twiddles W_N^{na kb}
// (written once per kernel) in 256-383.  One thread issues the MMAs and waits for their
// completion (tcgen05.commit on an mbarrier) with a bounded wait; on timeout the kernel
// records DBP_ERR_TIMEOUT in *err, frees its TMEM and returns.
#pragma once
#include "gemm_kernel.cuh"
#include "umma.cuh"

namespace dbp {

template <int N, int TY>
struct UGeo {
    static constexpr int NA = 64, NB = N / NA;
    static constexpr int G = 64 / NB;                     // overlap-save blocks per 128-row tile
    static constexpr int T = 256;
    static constexpr int FB_RS = NA * 8 + 16;             // spectrum row stride (bytes), padded
    static constexpr size_t TB = (size_t)G * 2 * N * 8;
    static constexpr size_t OFF_A = TB;                   // A hi | A lo (and aliases)
    static constexpr size_t A_BYTES = 65536;
    static constexpr size_t R_BYTES = (128 * FB_RS > (int)A_BYTES) ? 128 * FB_RS : A_BYTES;
    static constexpr size_t OFF_B = OFF_A + ((R_BYTES + 1023) / 1024) * 1024;
    static constexpr size_t OFF_H = OFF_B + 65536;
    static constexpr size_t OFF_TAPS = OFF_H + (size_t)N * 8;
    static constexpr int TAPS_MAX = 1 + DBP_MAX_TAPS + 15;
    static constexpr size_t SMEM = OFF_TAPS + TAPS_MAX * 4;
    static constexpr int PPAD = N + N / 4;                // P of one block, +4 floats per 16
    static constexpr int PER = G * 2 * N / T;             // tile elements per thread (load / store)
    static constexpr uint32_t TW_COL = 256;               // TMEM: D_hh 0-127, D_x 128-255, twiddles after
    static_assert(NB == 16 || NB == 32, "NB-point register DFTs of 16 or 32");
    static_assert(G * N / 16 == T, "one thread per 16 consecutive positions in the nonlinear step");
    static_assert(N % T == 0 && (G * 2 * NA) % T == 0, "whole units per thread");
    static_assert((size_t)G * PPAD * 4 <= R_BYTES, "P fits the operand region");
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

// Byte offsets in the no-swizzle canonical layouts of a 128 x 128 16-bit operand.
// K-major (16-byte rows along K): core (r / 8, k / 8) at 2048 (r / 8) + 128 (k / 8).
// MN-major (16-byte rows along the row index r): core at 2048 (k / 8) + 128 (r / 8).
__host__ __device__ __forceinline__ uint32_t off_kmaj(int r, int k) {
    return (uint32_t)((r >> 3) * 2048 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
__host__ __device__ __forceinline__ uint32_t off_mnmaj(int r, int k) {
    return (uint32_t)((k >> 3) * 2048 + (r >> 3) * 128 + (k & 7) * 16 + (r & 7) * 2);
}

// x = hi + lo, both of the 16-bit type: hi the rounding of x, lo the rounding of the
// remainder.  The tiles are scaled so that their largest possible value is about 2^12,
// so the remainders of all but negligibly small values are normal numbers and need no
// extra scaling (for FP16; BF16 has the FP32 exponent range).
template <int TY>
struct Pack16;
template <>
struct Pack16<DBP_SPLIT_FP16> {
    __device__ __forceinline__ static void split(float a, float b, uint32_t &hi, uint32_t &lo) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
};
template <>
struct Pack16<DBP_SPLIT_BF16> {
    __device__ __forceinline__ static void split(float a, float b, uint32_t &hi, uint32_t &lo) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
};

// 2^(12 - ceil(log2(bound))) for bound > 0 (1 otherwise): the scale that puts the tile's
// largest possible value near 2^12.
__device__ __forceinline__ float pow2_scale(float bound) {
    if (!(bound > 0.f)) return 1.f;
    return ldexpf(1.f, 12 - (ilogbf(bound) + 1));
}

__device__ __forceinline__ void smem_max(unsigned *slot, float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(slot, __float_as_uint(v));
}

// Symmetric filter of 16 consecutive positions k0..k0+15 of one block (circular, length
// N), P in the padded layout (+4 floats per 16): th_r = a_0 P_k + sum_i a_i (P_{k-i} +
// P_{k+i}) for 8 n_tapblk taps a side (Eq. 3 up to the factor gamma_eff in a).
template <int N>
__device__ __forceinline__ void fir16_block(const float *P, const float *a, int n_tapblk, int k0, float (&th)[16]) {
    auto pp = [](int e) { return e + 4 * (e >> 4); };
    {
        const float4 *pc = reinterpret_cast<const float4 *>(P + pp(k0));
        const float a0 = a[0];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 f = pc[q];
            th[4 * q + 0] = a0 * f.x;
            th[4 * q + 1] = a0 * f.y;
            th[4 * q + 2] = a0 * f.z;
            th[4 * q + 3] = a0 * f.w;
        }
    }
    for (int blk = 0; blk < n_tapblk; ++blk) {
        const int i0 = 8 * blk;
        float lw[24], rw[24];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const int el = (k0 - i0 - 8 + 4 * q) & (N - 1);
            const int er = (k0 + i0 + 4 * q) & (N - 1);
            const float4 fl = *reinterpret_cast<const float4 *>(P + pp(el));
            const float4 fr = *reinterpret_cast<const float4 *>(P + pp(er));
            lw[4 * q + 0] = fl.x; lw[4 * q + 1] = fl.y; lw[4 * q + 2] = fl.z; lw[4 * q + 3] = fl.w;
            rw[4 * q + 0] = fr.x; rw[4 * q + 1] = fr.y; rw[4 * q + 2] = fr.z; rw[4 * q + 3] = fr.w;
        }
#pragma unroll
        for (int ii = 1; ii <= 8; ++ii) {
            const float ai = a[i0 + ii];
#pragma unroll
            for (int r = 0; r < 16; ++r) th[r] = fmaf(ai, lw[r - ii + 8] + rw[r + ii], th[r]);
        }
    }
}

struct UmmaParams {
    GemmParams g;
    const uint4 *Fu;        // DFT matrix hi | lo in the K-major canonical layout (64 KB)
    int *err;               // DBP_ERR_TIMEOUT on a bounded-wait timeout
    int total_blocks;       // n_wave * n_blocks
    int essfm;
};

template <int N, int TY>
__global__ void __launch_bounds__(256, 1) dbp_umma_kernel(const UmmaParams u) {
    using U = UGeo<N, TY>;
    constexpr int NA = U::NA, NB = U::NB, G = U::G, T = U::T;
    constexpr bool BF = TY == DBP_SPLIT_BF16;
    constexpr uint32_t ID1 = umma::idesc_f16(BF, 128, 128, true, false);    // A MN-major, B K-major
    constexpr uint32_t ID2 = umma::idesc_f16(BF, 128, 128, false, true);    // A K-major, B MN-major
    constexpr uint64_t LIMIT_NS = 1000000000ull;
    constexpr int TWQ = (2 * (NB - 1) + 31) / 32;                           // 32-column twiddle loads
    const FwdParams &p = u.g.f;
    extern __shared__ __align__(1024) unsigned char sm[];
    float2 *Tb = reinterpret_cast<float2 *>(sm);
    unsigned char *Ahi = sm + U::OFF_A, *Alo = Ahi + 32768;
    unsigned char *Fb = Ahi;                                       // spectrum rows (after GEMM 2)
    float *Pb = reinterpret_cast<float *>(Ahi);                    // intensity (nonlinear step)
    unsigned char *Bm = sm + U::OFF_B;                             // DFT matrix hi | lo
    float2 *sH = reinterpret_cast<float2 *>(sm + U::OFF_H);
    float *sa = reinterpret_cast<float *>(sm + U::OFF_TAPS);
    __shared__ uint32_t s_tmem;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ unsigned s_max[2];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int na_t = t & (NA - 1);          // the column na of every (block, pol, na) unit of this thread
    const long long n = p.n;
    const int n_tiles = (u.total_blocks + G - 1) / G;

    for (int i = t; i < 4096; i += T) reinterpret_cast<uint4 *>(Bm)[i] = __ldg(u.Fu + i);
    if (warp == 0) {
        tmem_alloc(&s_tmem, 512);
        tmem_relinquish();
    }
    if (t == 0) umma::mbar_init(&s_mbar, 1);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tm = s_tmem;
    const uint32_t tq = tm + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lane quarter
    // this thread's twiddles W_N^{na kb}, kb = 1 .. NB-1 (re, im), kept in TMEM columns
    // TW_COL + 64 (warp / 4) .. of its lane for the whole kernel
    const uint32_t twt = tq + U::TW_COL + 64u * (uint32_t)(warp >> 2);
    {
        uint32_t r[32];
#pragma unroll
        for (int q = 0; q < TWQ; ++q) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int kb = 1 + (32 * q + j) / 2;
                float2 w = make_float2(0.f, 0.f);
                if (kb < NB) w = __ldg(u.g.Wn + ((na_t * kb) & (N - 1)));
                r[j] = __float_as_uint((j & 1) ? w.y : w.x);
            }
            tmem_st32(twt + 32 * q, r);
        }
    }
    auto load_tw = [&](float2 (&w)[NB]) {
        uint32_t r[32 * TWQ];
#pragma unroll
        for (int q = 0; q < TWQ; ++q) {
            uint32_t (&rq)[32] = *reinterpret_cast<uint32_t(*)[32]>(r + 32 * q);
            umma::ld4x8(twt + 32 * q, twt + 32 * q + 8, twt + 32 * q + 16, twt + 32 * q + 24, rq);
        }
        w[0] = make_float2(1.f, 0.f);
#pragma unroll
        for (int kb = 1; kb < NB; ++kb) w[kb] = make_float2(__uint_as_float(r[2 * kb - 2]), __uint_as_float(r[2 * kb - 1]));
    };
    uint32_t phase = 0;
    bool ok = true;

    // issues one split GEMM (24 MMAs into D_hh = A_hi B_hi and D_x = A_hi B_lo + A_lo B_hi)
    // and waits for it (one polling thread); false on timeout (the whole CTA agrees)
    auto gemm = [&](bool second) -> bool {
        fence_proxy_async_smem();   // operand writes -> tensor-core (async proxy) reads
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        int done = 1;
        if (t == 0) {
            const uint32_t a0 = umma::saddr(Ahi), a1 = umma::saddr(Alo), b0 = umma::saddr(Bm), b1 = b0 + 32768;
#pragma unroll 1
            for (int ks = 0; ks < 8; ++ks) {
                uint64_t ah, al, bh, bl;
                if (!second) {   // A MN-major (K groups 2048 B apart), B K-major (K groups 128 B apart)
                    ah = umma::desc(a0 + ks * 4096, 2048, 128);
                    al = umma::desc(a1 + ks * 4096, 2048, 128);
                    bh = umma::desc(b0 + ks * 256, 128, 2048);
                    bl = umma::desc(b1 + ks * 256, 128, 2048);
                } else {         // A K-major, B read transposed (MN-major)
                    ah = umma::desc(a0 + ks * 256, 128, 2048);
                    al = umma::desc(a1 + ks * 256, 128, 2048);
                    bh = umma::desc(b0 + ks * 4096, 2048, 128);
                    bl = umma::desc(b1 + ks * 4096, 2048, 128);
                }
                const uint32_t id = second ? ID2 : ID1;
                umma::mma(tm, ah, bh, id, ks > 0);
                umma::mma(tm + 128, ah, bl, id, ks > 0);
                umma::mma(tm + 128, al, bh, id, 1);
            }
            umma::commit(&s_mbar);
            done = umma::mbar_wait(&s_mbar, phase, LIMIT_NS) ? 1 : 0;
        }
        phase ^= 1u;
        const int all = __syncthreads_and(done);
        tmem_fence_after_sync();
        if (!all && t == 0) atomicCAS(u.err, 0, DBP_ERR_TIMEOUT);
        return all != 0;
    };

    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        // window start and waveform of each block of the tile (-1: past the end)
        long long wstart[G], woff[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int gid = tile * G + g;
            wstart[g] = -1;
            woff[g] = 0;
            if (gid < u.total_blocks) {
                const int w = gid / p.n_blocks, b = gid - w * p.n_blocks;
                wstart[g] = (long long)b * p.valid;
                woff[g] = (long long)w * 2 * n;
            }
        }
        // ---- load the tile's G windows (both polarizations) into Tb: every load of the
        // thread in flight at once, then the stores
        if (t == 0) s_max[0] = 0u;
        __syncthreads();
        float mloc = 0.f;
        {
            float2 v[U::PER];
#pragma unroll
            for (int j = 0; j < U::PER; ++j) {
                constexpr int PG = 2 * N / T, PP = N / T;
                const int g = j / PG, pol = (j / PP) & 1, pos = t + T * (j % PP);
                v[j] = make_float2(0.f, 0.f);
                if (wstart[g] >= 0) {
                    const float2 *in = p.in + woff[g] + (size_t)pol * n;
                    long long idx = wstart[g] - p.half_overlap + pos;
                    if (idx >= 0 && idx < n) {
                        v[j] = __ldg(in + idx);
                    } else if (p.boundary == DBP_PERIODIC) {
                        idx %= n;
                        if (idx < 0) idx += n;
                        v[j] = __ldg(in + idx);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < U::PER; ++j) {
                Tb[t + T * j] = v[j];
                mloc = fmaxf(mloc, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
            }
        }
        // the windows of the tile this CTA runs next, into L2 (a hint): 16 KB pieces
        if (t < 2 * G * ((N * 8 + 16383) / 16384)) {
            constexpr int CH = (N * 8 + 16383) / 16384;
            const int g = t / (2 * CH), pol = (t / CH) & 1, c = t % CH;
            const int gid = (tile + (int)gridDim.x) * G + g;
            if (gid < u.total_blocks) {
                const int w = gid / p.n_blocks, b = gid - w * p.n_blocks;
                const long long lo = (long long)b * p.valid - p.half_overlap;
                long long a0 = lo < 0 ? 0 : lo, a1 = lo + N > n ? n : lo + N;
                const char *row = reinterpret_cast<const char *>(p.in + (size_t)w * 2 * n + (size_t)pol * n);
                unsigned long long x0 = reinterpret_cast<unsigned long long>(row + a0 * 8) + (unsigned long long)c * 16384;
                unsigned long long x1 = reinterpret_cast<unsigned long long>(row + a1 * 8);
                if (x0 + 16384 < x1) x1 = x0 + 16384;
                x0 = (x0 + 15) & ~15ull;
                x1 &= ~15ull;
                if (a1 > a0 && x1 > x0) bulk_prefetch_l2(reinterpret_cast<const void *>(x0), (unsigned)(x1 - x0));
            }
        }
        smem_max(&s_max[0], mloc);
        int cur = 0;
        for (int s = 0; s < p.n_steps && ok; ++s) {
            // stage this step's H and taps (their last readers finished before the last barrier)
            if ((s == 0 && tile == (int)blockIdx.x) || p.h_stride != 0) {
                const uint4 *hs = reinterpret_cast<const uint4 *>(u.g.Hn + p.h_stride * s);
                for (int i = t; i < N / 2; i += T) reinterpret_cast<uint4 *>(sH)[i] = __ldg(hs + i);
            }
            if (u.essfm) for (int i = t; i < p.taps_stride; i += T) sa[i] = __ldg(p.taps + p.taps_stride * s + i);
            __syncthreads();   // Tb, its maximum, H and taps visible
            const float m = __uint_as_float(s_max[cur]);
            const float sc1 = pow2_scale(1.5f * NB * m), sc2 = pow2_scale(1.5f * m);
            // ---- NB-point DFTs, twiddle, scale, split into the MN-major A operand
            {
                float2 w[NB];
                load_tw(w);
#pragma unroll 1
                for (int unit = t; unit < G * 2 * NA; unit += T) {
                    const int gp = unit / NA;          // 2 g + pol: rows gp * NB + kb
                    const float2 *col = Tb + (size_t)gp * N + na_t;
                    float2 v[NB];
#pragma unroll
                    for (int nb = 0; nb < NB; ++nb) v[nb] = col[NA * nb];
                    Dft<NB, false>::run(v);
#pragma unroll
                    for (int kb = 0; kb < NB; ++kb) {
                        const float2 z = kb ? cmul(v[kb], w[kb]) : v[kb];
                        v[kb] = make_float2(z.x * sc1, z.y * sc1);
                    }
#pragma unroll
                    for (int c = 0; c < NB / 8; ++c) {
                        uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float2 e0 = v[8 * c + 2 * j], e1 = v[8 * c + 2 * j + 1];
                            Pack16<TY>::split(e0.x, e1.x, rh[j], rl[j]);
                            Pack16<TY>::split(e0.y, e1.y, ih[j], il[j]);
                        }
                        const int r0 = gp * NB + 8 * c;
                        *reinterpret_cast<uint4 *>(Ahi + off_mnmaj(r0, na_t)) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                        *reinterpret_cast<uint4 *>(Alo + off_mnmaj(r0, na_t)) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                        *reinterpret_cast<uint4 *>(Ahi + off_mnmaj(r0, NA + na_t)) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                        *reinterpret_cast<uint4 *>(Alo + off_mnmaj(r0, NA + na_t)) = make_uint4(il[0], il[1], il[2], il[3]);
                    }
                }
            }
            if (t == 0) s_max[cur ^ 1] = 0u;
            if (!(ok = gemm(false))) break;
            // ---- X -> Y = X H (x sc2 / sc1), split into the K-major A operand (each lane one row)
            const int row = 32 * (warp & 3) + lane;
            const int kb = row % NB;
            const float r12 = sc2 / sc1;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int kc = 32 * (warp >> 2) + 8 * c;
                uint32_t r[32];
                umma::ld4x8(tq + kc, tq + NA + kc, tq + 128 + kc, tq + 128 + NA + kc, r);
                {
                    uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        float2 y[2];
#pragma unroll
                        for (int d = 0; d < 2; ++d) {
                            const int e = 2 * j + d;
                            const float2 x = make_float2(__uint_as_float(r[e]) + __uint_as_float(r[16 + e]),
                                                         __uint_as_float(r[8 + e]) + __uint_as_float(r[24 + e]));
                            const float2 h = sH[kb + NB * (kc + e)];
                            y[d] = cmul(x, make_float2(h.x * r12, h.y * r12));
                        }
                        Pack16<TY>::split(y[0].x, y[1].x, rh[j], rl[j]);
                        Pack16<TY>::split(y[0].y, y[1].y, ih[j], il[j]);
                    }
                    *reinterpret_cast<uint4 *>(Ahi + off_kmaj(row, kc)) = make_uint4(rh[0], rh[1], rh[2], rh[3]);
                    *reinterpret_cast<uint4 *>(Alo + off_kmaj(row, kc)) = make_uint4(rl[0], rl[1], rl[2], rl[3]);
                    *reinterpret_cast<uint4 *>(Ahi + off_kmaj(row, NA + kc)) = make_uint4(ih[0], ih[1], ih[2], ih[3]);
                    *reinterpret_cast<uint4 *>(Alo + off_kmaj(row, NA + kc)) = make_uint4(il[0], il[1], il[2], il[3]);
                }
            }
            if (!(ok = gemm(true))) break;
            // ---- y' (unscaled) -> spectrum rows (float2, padded stride)
            const float us2 = 1.f / sc2;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int na0 = 32 * (warp >> 2) + 8 * c;
                uint32_t r[32];
                umma::ld4x8(tq + na0, tq + NA + na0, tq + 128 + na0, tq + 128 + NA + na0, r);
                float2 *dst = reinterpret_cast<float2 *>(Fb + (size_t)row * U::FB_RS) + na0;
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    dst[e] = make_float2((__uint_as_float(r[e]) + __uint_as_float(r[16 + e])) * us2,
                                         (__uint_as_float(r[8 + e]) + __uint_as_float(r[24 + e])) * us2);
            }
            tmem_fence_before_sync();
            __syncthreads();
            // ---- conjugate twiddle W_N^{-na kb}, NB-point inverse DFTs over kb -> time domain
            {
                float2 w[NB];
                load_tw(w);
#pragma unroll 1
                for (int unit = t; unit < G * 2 * NA; unit += T) {
                    const int gp = unit / NA;
                    float2 v[NB];
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        const float2 y = *(reinterpret_cast<const float2 *>(Fb + (size_t)(gp * NB + k) * U::FB_RS) + na_t);
                        v[k] = k ? cmulc(y, w[k]) : y;
                    }
                    Dft<NB, true>::run(v);
                    float2 *col = Tb + (size_t)gp * N + na_t;
#pragma unroll
                    for (int nb = 0; nb < NB; ++nb) col[NA * nb] = v[nb];
                }
            }
            __syncthreads();
            // ---- nonlinear sub-step on 16 consecutive positions per thread
            const int g = t / (N / 16), k0 = 16 * (t % (N / 16));
            float2 *x0 = Tb + (size_t)(2 * g) * N + k0, *x1 = x0 + N;
            float th[16];
            float mloc2 = 0.f;
            if (!p.linear_only) {
                if (u.essfm) {
                    float *P = Pb + (size_t)g * U::PPAD;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float pk[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) pk[e] = joint_intensity(x0[4 * q + e], x1[4 * q + e]);
                        *reinterpret_cast<float4 *>(P + (k0 + 4 * q) + 4 * ((k0 + 4 * q) >> 4)) =
                            make_float4(pk[0], pk[1], pk[2], pk[3]);
                    }
                    __syncthreads();
                    fir16_block<N>(P, sa, p.n_tapblk, k0, th);
                } else {
                    const float a0 = __ldg(p.taps + p.taps_stride * s);
#pragma unroll
                    for (int r = 0; r < 16; ++r) th[r] = a0 * joint_intensity(x0[r], x1[r]);
                }
                if (p.fast_exp) {
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        const float2 e = expj<true>(th[r]);
                        x0[r] = cmul(x0[r], e);
                        x1[r] = cmul(x1[r], e);
                    }
                } else {
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        const float2 e = expj<false>(th[r]);
                        x0[r] = cmul(x0[r], e);
                        x1[r] = cmul(x1[r], e);
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 16; ++r)
                mloc2 = fmaxf(mloc2, fmaxf(fmaxf(fabsf(x0[r].x), fabsf(x0[r].y)), fmaxf(fabsf(x1[r].x), fabsf(x1[r].y))));
            smem_max(&s_max[cur ^ 1], mloc2);
            cur ^= 1;
            __syncthreads();   // Tb complete; P and the operand region free
        }
        if (!ok) break;
        // ---- overlap-and-save: the central V samples of every block
        const int h = p.half_overlap;
#pragma unroll
        for (int j = 0; j < U::PER; ++j) {
            constexpr int PG = 2 * N / T, PP = N / T;
            const int g = j / PG, pol = (j / PP) & 1, pos = t + T * (j % PP);
            if (wstart[g] < 0 || pos < h || pos >= h + p.valid) continue;
            const long long gi = wstart[g] - h + pos;
            if (gi < n) __stcs(p.out + woff[g] + (size_t)pol * n + gi, Tb[t + T * j]);
        }
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 0) tmem_dealloc(tm, 512);
}

}  // namespace dbp
