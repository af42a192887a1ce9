// Split-precision DFT-as-GEMM linear sub-step inside a fused overlap-save DBP kernel.
//
// Precision variant of the linear sub-step of Section II (Eq. 1): with N = NB * NA,
//   GEMM 1  NA-point DFTs of the NB interleaved sub-sequences, as a dense matrix
//           product on the tensor cores (mma.sync m16n8k16, BF16 or FP16 inputs, FP32
//           accumulate).  Complex data enter as a real GEMM [Re | Im] x
//           [[F_r, F_i], [-F_i, F_r]]; every operand is split into hi + lo parts of the
//           16-bit type (lo stored scaled by 2^8 / 2^11) and three products
//           hi*hi + (hi*lo + lo*hi) / scale are accumulated in FP32.
//   FP32    twiddles W_N^{nb ka}, NB-point DFTs, x H(f_k) (1/N folded in), inverse
//           NB-point DFTs and conjugate twiddles, in registers.
//   GEMM 2  inverse NA-point DFTs (conjugate DFT matrix), same splitting.
// The nonlinear sub-step (Eqs. 2-3) is FP32 as in the FFT path.  For FP16 each GEMM's
// input is scaled by a power of two (exact) so that the low parts stay normal numbers.
// Shared memory: two buffers [pol][re/im][NB rows][NA + 8 cols] (the +8 columns make
// the 8-byte fragment loads conflict-free); time-domain sample p sits at row p mod NB,
// column p div NB.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "block_fft.cuh"

namespace dbp {

struct GemmParams {
    FwdParams f;                 // geometry, taps, input/output
    const float2 *Hn;            // [steps][N] H_s / N in natural frequency order
    const float2 *Wn;            // [N] W_N^m
    const uint32_t *F;           // [4][NA][NA/2] packed pairs: Fr hi, Fr lo, Fi hi, Fi lo (transposed)
};

template <int TY>
struct Split16;

// The low part is stored scaled by LO = 2^(significand bits) so that it stays in the
// normal range of the 16-bit type (FP16 subnormals would lose the low part of small
// elements); products with one low factor are accumulated separately and rescaled once.
template <>
struct Split16<DBP_SPLIT_BF16> {
    static constexpr float LO = 256.0f, INV_LO = 1.0f / 256.0f;
    __device__ __forceinline__ static void split(float a, float b, uint32_t &hi, uint32_t &lo) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn((a - hf.x) * LO, (b - hf.y) * LO);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
    __device__ __forceinline__ static void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

template <>
struct Split16<DBP_SPLIT_FP16> {
    static constexpr float LO = 2048.0f, INV_LO = 1.0f / 2048.0f;
    __device__ __forceinline__ static void split(float a, float b, uint32_t &hi, uint32_t &lo) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn((a - hf.x) * LO, (b - hf.y) * LO);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
    __device__ __forceinline__ static void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
};

template <int N, int NA>
struct GemmGeo {
    static constexpr int NB = N / NA;
    static constexpr int RS = NA + 8;                 // row stride (floats)
    static constexpr int PLANE = NB * RS;             // one (pol, re/im) plane
    static constexpr int BUF = 4 * PLANE;             // floats per buffer
    static constexpr int T = 256;
    static constexpr int R = 2 * NB;                  // GEMM rows (pol, nb)
    static constexpr int RT = (R + 15) / 16;          // row tiles
    static constexpr int CT = (2 * NA) / 8;           // column tiles
    static constexpr int KS = (2 * NA) / 16;          // k steps
    static constexpr size_t SMEM = (size_t)2 * BUF * sizeof(float) + 64 * sizeof(float);
    static_assert(NB >= 4 && NB <= 32, "NB in 4..32");
    static_assert(2 * N <= BUF, "P and theta fit in one buffer");
};

__device__ __forceinline__ float block_absmax(float v, float *red) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    __syncthreads();
    return m;
}

// out[(pol, nb)][n] = sum_k in[(pol, nb)][k] F^{(+/-)}[k][n] over the NA-point complex
// DFT (INV: conjugate matrix); buffers laid out [pol][re/im][nb][RS].
template <int N, int NA, int TY, bool INV>
__device__ __forceinline__ void dft_gemm(const float *in, float *out, const uint32_t *__restrict__ F, float scale,
                                         float unscale) {
    using GG = GemmGeo<N, NA>;
    using S = Split16<TY>;
    constexpr int NB = GG::NB, RS = GG::RS, PLANE = GG::PLANE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const uint32_t *FrH = F, *FrL = F + NA * NA / 2, *FiH = F + NA * NA, *FiL = F + 3 * NA * NA / 2;
    constexpr uint32_t NEG = 0x80008000u;
    for (int tile = warp; tile < GG::RT * GG::CT; tile += GG::T / 32) {
        const int rt = tile % GG::RT, ct = tile / GG::RT;
        float c[4] = {0.f, 0.f, 0.f, 0.f}, cx[4] = {0.f, 0.f, 0.f, 0.f};
        const int r0 = rt * 16 + g, r1 = r0 + 8;
        const bool v0 = r0 < GG::R, v1 = r1 < GG::R;
        const int pol0 = v0 ? r0 / NB : 0, nb0 = v0 ? r0 % NB : 0;
        const int pol1 = v1 ? r1 / NB : 0, nb1 = v1 ? r1 % NB : 0;
        const int np = ct * 8 + g;                       // output column of this lane's B fragment
        const bool out_im = np >= NA;
        const int n = out_im ? np - NA : np;
#pragma unroll 4
        for (int ks = 0; ks < GG::KS; ++ks) {
            const bool in_im = ks * 16 >= NA;
            const int k0 = ks * 16 - (in_im ? NA : 0);
            const float *p0 = in + (pol0 * 2 + (in_im ? 1 : 0)) * PLANE + nb0 * RS + k0 + 2 * tq;
            const float *p1 = in + (pol1 * 2 + (in_im ? 1 : 0)) * PLANE + nb1 * RS + k0 + 2 * tq;
            float2 a00 = v0 ? *reinterpret_cast<const float2 *>(p0) : make_float2(0.f, 0.f);
            float2 a10 = v1 ? *reinterpret_cast<const float2 *>(p1) : make_float2(0.f, 0.f);
            float2 a01 = v0 ? *reinterpret_cast<const float2 *>(p0 + 8) : make_float2(0.f, 0.f);
            float2 a11 = v1 ? *reinterpret_cast<const float2 *>(p1 + 8) : make_float2(0.f, 0.f);
            uint32_t ah[4], al[4];
            S::split(a00.x * scale, a00.y * scale, ah[0], al[0]);
            S::split(a10.x * scale, a10.y * scale, ah[1], al[1]);
            S::split(a01.x * scale, a01.y * scale, ah[2], al[2]);
            S::split(a11.x * scale, a11.y * scale, ah[3], al[3]);
            // B block: re->re Fr, im->im Fr, re->im +Fi (forward) / -Fi (inverse),
            //          im->re -Fi (forward) / +Fi (inverse)
            const bool use_i = in_im != out_im;
            const bool neg = use_i && (in_im ? !INV : INV);
            const uint32_t *TH = use_i ? FiH : FrH, *TL = use_i ? FiL : FrL;
            const int bidx = n * (NA / 2) + k0 / 2 + tq;
            uint32_t bh0 = __ldg(TH + bidx), bh1 = __ldg(TH + bidx + 4);
            uint32_t bl0 = __ldg(TL + bidx), bl1 = __ldg(TL + bidx + 4);
            if (neg) {
                bh0 ^= NEG; bh1 ^= NEG; bl0 ^= NEG; bl1 ^= NEG;
            }
            S::mma(c, ah, bh0, bh1);
            S::mma(cx, ah, bl0, bl1);
            S::mma(cx, al, bh0, bh1);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) c[i] = fmaf(cx[i], S::INV_LO, c[i]);
        // c0, c1: row g, columns ct*8 + 2tq, +1;  c2, c3: row g + 8
        const int nc = ct * 8 + 2 * tq;
        const bool oim = nc >= NA;
        const int nn = oim ? nc - NA : nc;
        if (v0)
            *reinterpret_cast<float2 *>(out + (pol0 * 2 + (oim ? 1 : 0)) * PLANE + nb0 * RS + nn) =
                make_float2(c[0] * unscale, c[1] * unscale);
        if (v1)
            *reinterpret_cast<float2 *>(out + (pol1 * 2 + (oim ? 1 : 0)) * PLANE + nb1 * RS + nn) =
                make_float2(c[2] * unscale, c[3] * unscale);
    }
}

template <int N, int NA, int TY>
__global__ void __launch_bounds__(256, 1) dbp_gemm_kernel(const GemmParams q, int essfm) {
    using GG = GemmGeo<N, NA>;
    constexpr int NB = GG::NB, RS = GG::RS, PLANE = GG::PLANE;
    const FwdParams &p = q.f;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *Tb = reinterpret_cast<float *>(smem_raw);          // time domain
    float *Fb = Tb + GG::BUF;                                  // spectrum / scratch
    float *red = Fb + GG::BUF;
    const int t = threadIdx.x;
    const int w = blockIdx.x / p.n_blocks;
    const int b = blockIdx.x - w * p.n_blocks;
    const long long n = p.n;
    const float2 *__restrict__ in = p.in + (size_t)w * 2 * n;
    float2 *__restrict__ out = p.out + (size_t)w * 2 * n;
    const long long win0 = (long long)b * p.valid - p.half_overlap;
    auto tidx = [](int pos) { return (pos % NB) * RS + pos / NB; };

    for (int pos = t; pos < N; pos += GG::T)
        for (int pol = 0; pol < 2; ++pol) {
            long long idx = win0 + pos;
            float2 v = make_float2(0.f, 0.f);
            if (idx >= 0 && idx < n) {
                v = __ldg(in + pol * n + idx);
            } else if (p.boundary == DBP_PERIODIC) {
                idx %= n;
                if (idx < 0) idx += n;
                v = __ldg(in + pol * n + idx);
            }
            Tb[(pol * 2) * PLANE + tidx(pos)] = v.x;
            Tb[(pol * 2 + 1) * PLANE + tidx(pos)] = v.y;
        }
    __syncthreads();

    for (int s = 0; s < p.n_steps; ++s) {
        // ---- GEMM 1: NA-point DFTs, time -> (nb, ka)
        float sc = 1.f, usc = 1.f;
        if (TY == DBP_SPLIT_FP16) {
            float m = 0.f;
            for (int i = t; i < GG::BUF; i += GG::T) m = fmaxf(m, fabsf(Tb[i]));
            m = block_absmax(m, red);
            const int e = m > 0.f ? ilogbf(m) + 1 : 0;
            sc = ldexpf(1.f, -e);
            usc = ldexpf(1.f, e);
        }
        dft_gemm<N, NA, TY, false>(Tb, Fb, q.F, sc, usc);
        __syncthreads();
        // ---- FP32: twiddle, NB-point DFT, x H, inverse, conjugate twiddle
        const float2 *__restrict__ H = q.Hn + p.h_stride * s;
        for (int col = t; col < 2 * NA; col += GG::T) {
            const int pol = col / NA, ka = col - pol * NA;
            float *re = Fb + (pol * 2) * PLANE + ka, *im = Fb + (pol * 2 + 1) * PLANE + ka;
            float2 u[NB];
#pragma unroll
            for (int nb = 0; nb < NB; ++nb) u[nb] = cmul(make_float2(re[nb * RS], im[nb * RS]), __ldg(q.Wn + (nb * ka) % N));
            Dft<NB, false>::run(u);
#pragma unroll
            for (int kb = 0; kb < NB; ++kb) u[kb] = cmul(u[kb], __ldg(H + ka + NA * kb));
            Dft<NB, true>::run(u);
#pragma unroll
            for (int nb = 0; nb < NB; ++nb) {
                const float2 v = cmulc(u[nb], __ldg(q.Wn + (nb * ka) % N));
                re[nb * RS] = v.x;
                im[nb * RS] = v.y;
            }
        }
        __syncthreads();
        // ---- GEMM 2: inverse NA-point DFTs, (nb, ka) -> time
        if (TY == DBP_SPLIT_FP16) {
            float m = 0.f;
            for (int i = t; i < GG::BUF; i += GG::T) m = fmaxf(m, fabsf(Fb[i]));
            m = block_absmax(m, red);
            const int e = m > 0.f ? ilogbf(m) + 1 : 0;
            sc = ldexpf(1.f, -e);
            usc = ldexpf(1.f, e);
        }
        dft_gemm<N, NA, TY, true>(Fb, Tb, q.F, sc, usc);
        __syncthreads();
        // ---- nonlinear sub-step (FP32), P and theta in the spectrum buffer
        const float *__restrict__ a = p.taps + p.taps_stride * s;
        float *sP = Fb, *sT = Fb + N;
        for (int pos = t; pos < N; pos += GG::T) {
            const int i = tidx(pos);
            sP[pos] = joint_intensity(make_float2(Tb[i], Tb[PLANE + i]), make_float2(Tb[2 * PLANE + i], Tb[3 * PLANE + i]));
        }
        __syncthreads();
        const int ntaps = essfm ? 8 * p.n_tapblk : 0;
        for (int pos = t; pos < N; pos += GG::T) {
            float th = __ldg(a) * sP[pos];
            for (int k = 1; k <= ntaps; ++k)
                th = fmaf(__ldg(a + k), sP[(pos - k) & (N - 1)] + sP[(pos + k) & (N - 1)], th);
            sT[pos] = th;
        }
        __syncthreads();
        for (int pos = t; pos < N; pos += GG::T) {
            const int i = tidx(pos);
            const float2 e = expj(sT[pos]);
            for (int pol = 0; pol < 2; ++pol) {
                const float2 z = cmul(make_float2(Tb[(2 * pol) * PLANE + i], Tb[(2 * pol + 1) * PLANE + i]), e);
                Tb[(2 * pol) * PLANE + i] = z.x;
                Tb[(2 * pol + 1) * PLANE + i] = z.y;
            }
        }
        __syncthreads();
    }
    const int h = p.half_overlap;
    for (int pos = t; pos < N; pos += GG::T) {
        const long long g = (long long)b * p.valid - h + pos;
        if (pos >= h && pos < h + p.valid && g < n) {
            const int i = tidx(pos);
            __stcs(out + g, make_float2(Tb[i], Tb[PLANE + i]));
            __stcs(out + n + g, make_float2(Tb[2 * PLANE + i], Tb[3 * PLANE + i]));
        }
    }
}

template <int N, int NA, int TY>
int launch_gemm_n(const GemmParams &q, int n_wave, bool essfm, cudaStream_t st) {
    using GG = GemmGeo<N, NA>;
    static unsigned long long done = 0;
    const long long grid = (long long)q.f.n_blocks * n_wave;
    if (grid <= 0 || grid > 0x7fffffffLL) return DBP_ERR_ARG;
    if (!set_smem_once(dbp_gemm_kernel<N, NA, TY>, GG::SMEM, done)) return DBP_ERR_CUDA;
    dbp_gemm_kernel<N, NA, TY><<<(unsigned)grid, GG::T, GG::SMEM, st>>>(q, essfm ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

}  // namespace dbp
