// Adjoint (reverse mode) of the fused overlap-save DBP: gradients of a real loss with
// respect to the input waveform, the ESSFM coefficients c_{s,i}, the per-step
// nonlinear strengths gamma_eff_s and the step lengths dz_s (through H_s only).
//
// Gradient convention: g = dL/dRe + j dL/dIm.  Derived from the forward operators of
// Section II (Eqs. 1-3) and Section III's overlap-and-save:
//   nonlinear z = y exp(j theta), theta = gamma_eff sum_i c_i S_i (S_0 = P_k,
//     S_i = P_{k-i} + P_{k+i}):  s_k = dL/dtheta_k = -sum_pol Im(conj(g_z) z);
//     R_i = sum_k s_k S_{k,i} (dL/dc_i = gamma_eff R_i, dL/dgamma_eff = sum_i c_i R_i);
//     dL/dP = the same symmetric filter applied to s;  g_y = g_z exp(-j theta) + 2 (dL/dP) y
//   linear y = IDFT(H' DFT(x)), H' = H / N:  g_x = IDFT(conj(H') DFT(g_y));
//     dL/ddz = sum_k phi'_k Re(j conj(G_k) U_k), G = DFT(g_y), U = H' DFT(x),
//     phi'_k = 2 pi^2 beta2 f_k^2
//   overlap-and-save transposes to overlap-add of the block input gradients.
// One CTA per block: a forward sweep stores each step's input (checkpoints); the reverse
// sweep recomputes each step's linear sub-step from its checkpoint.  Per-warp partial
// sums of R_i and dL/ddz go to scratch (no CTA barrier) and are reduced in a fixed
// order, so the result is bitwise reproducible.  ESSFM plans of at most two steps use the
// forward kernel's hardware exponential, so the gradient is that of what dbp_run
// computes.  At N = 4096 (two CTAs per SM, 128 registers a thread) and N = 8192 (one)
// each thread's spectrum U and gradient g live in tensor memory (tcgen05.st /
// tcgen05.ld of its own TMEM lane, 128 columns a thread) instead of global scratch;
// y stays in global scratch.
#pragma once
#include "block_fft.cuh"
#include "umma.cuh"

namespace dbp {

struct AdjParams {
    FwdParams f;             // in = waveform x, plan tables
    const float2 *gout;      // [n_wave][2][n] dL/d(out)
    float4 *gblk;            // [blocks][N] block gradient (both polarizations per position)
    float4 *uscr;            // [blocks][N] U = H' DFT(x) of the step being reversed
    float4 *yscr;            // [blocks][N] y of the step being reversed
    float4 *ckpt;            // [blocks][n_steps - 1][N] inputs of steps 1..n_steps-1
    float *part;             // [blocks][n_steps * nr + n_steps]: R_{s,i} then dL/ddz_s
    int nr;                  // correlations per step: 1 + 8 n_tapblk
    float cphi;              // 2 pi^2 beta2 (f_s / N)^2
};

// Sum of val[k] over the warp; lane 0 writes the K sums to dst (the warp's own row of
// partial sums: no barrier, the fixed-order FP64 reduction over all rows follows later).
template <int K>
__device__ __forceinline__ void warp_sum(float (&val)[K], float *dst) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float x = val[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        val[k] = x;
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) dst[k] = val[k];
    }
}

// pass-3 operation of the recomputed linear sub-step: x H_s, and keep U = H' X
template <int N>
struct MidRecompute {
    const float2 *sH;
    float4 *U;
    __device__ __forceinline__ void two(float2 (&u0)[16], float2 (&u1)[16], int base) {
        MidMulH<N>{sH}.two(u0, u1, base);
#pragma unroll
        for (int j = 0; j < 16; ++j) U[base + j] = make_float4(u0[j].x, u0[j].y, u1[j].x, u1[j].y);
    }
    template <int R>
    __device__ __forceinline__ void one(float2 (&u)[R], int pol, int base) {
        MidMulH<N>{sH}.one(u, pol, base);
        float2 *uh = reinterpret_cast<float2 *>(U);
#pragma unroll
        for (int j = 0; j < R; ++j) uh[2 * (base + j) + pol] = u[j];
    }
};

// pass-3 operation of the linear adjoint: accumulate dL/ddz, then x conj(H_s)
template <int N>
struct MidAdjoint {
    const float2 *sH;
    const float4 *U;
    float cphi;
    float acc;
    __device__ __forceinline__ float phi_prime(int p) const {
        using G = Geo<N>;
        const int k2 = p % G::N0, k1 = (p / G::N0) % G::N1, k0 = p / (G::N0 * G::N1);
        int k = k0 + G::N2 * k1 + G::N2 * G::N1 * k2;
        if (k >= N / 2) k -= N;
        const float kk = (float)k;
        return cphi * kk * kk;
    }
    __device__ __forceinline__ static float mimag(float2 g, float2 u) { return g.y * u.x - g.x * u.y; }  // -Im(conj(g) u)
    __device__ __forceinline__ void two(float2 (&u0)[16], float2 (&u1)[16], int base) {
        const float4 *hrow = reinterpret_cast<const float4 *>(sH + hphys<16>(base));
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const float4 uu = U[base + j];
            acc = fmaf(phi_prime(base + j),
                       mimag(u0[j], make_float2(uu.x, uu.y)) + mimag(u1[j], make_float2(uu.z, uu.w)), acc);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 h = hrow[j];
            u0[2 * j] = cmulc(u0[2 * j], make_float2(h.x, h.y));
            u1[2 * j] = cmulc(u1[2 * j], make_float2(h.x, h.y));
            u0[2 * j + 1] = cmulc(u0[2 * j + 1], make_float2(h.z, h.w));
            u1[2 * j + 1] = cmulc(u1[2 * j + 1], make_float2(h.z, h.w));
        }
    }
    template <int R>
    __device__ __forceinline__ void one(float2 (&u)[R], int pol, int base) {
        const float2 *uh = reinterpret_cast<const float2 *>(U);
        const float4 *hrow = reinterpret_cast<const float4 *>(sH + hphys<R>(base));
#pragma unroll
        for (int j = 0; j < R; ++j) acc = fmaf(phi_prime(base + j), mimag(u[j], uh[2 * (base + j) + pol]), acc);
#pragma unroll
        for (int j = 0; j < R / 2; ++j) {
            const float4 h = hrow[j];
            u[2 * j] = cmulc(u[2 * j], make_float2(h.x, h.y));
            u[2 * j + 1] = cmulc(u[2 * j + 1], make_float2(h.z, h.w));
        }
    }
};

// Tensor memory as per-thread scratch of the reverse sweep (N = 4096: 256 threads, two
// per TMEM lane; N = 8192: 512 threads, four per lane; 128 columns a thread): the
// thread's U (its pass-3 positions) and the gradient g (its 16 pass-1 positions, one
// float4 of both polarizations per position), 64 32-bit columns each.  Every access is
// to the thread's own positions, so TMEM replaces the round trip through global memory.
__device__ __forceinline__ void tm_st16(uint32_t a, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};\n" ::"r"(a),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
// 16 consecutive columns (4 float4: 4 positions, both polarizations) of the thread's lane
__device__ __forceinline__ void tm_store4(uint32_t a, float4 v0, float4 v1, float4 v2, float4 v3) {
    const uint32_t r[16] = {__float_as_uint(v0.x), __float_as_uint(v0.y), __float_as_uint(v0.z), __float_as_uint(v0.w),
                            __float_as_uint(v1.x), __float_as_uint(v1.y), __float_as_uint(v1.z), __float_as_uint(v1.w),
                            __float_as_uint(v2.x), __float_as_uint(v2.y), __float_as_uint(v2.z), __float_as_uint(v2.w),
                            __float_as_uint(v3.x), __float_as_uint(v3.y), __float_as_uint(v3.z), __float_as_uint(v3.w)};
    tm_st16(a, r);
}
__device__ __forceinline__ void tm_load4(uint32_t a, float4 (&v)[4]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(a)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int j = 0; j < 4; ++j)
        v[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]), __uint_as_float(r[4 * j + 2]),
                           __uint_as_float(r[4 * j + 3]));
}

// MidRecompute with U kept in TMEM.  two: pass 3 with N0 = 16 (positions base .. base + 15,
// both polarizations, one float4 per position); one: N0 = 32 (one polarization of
// positions base .. base + 31, two complex values per float4).  64 columns either way.
template <int N>
struct MidRecomputeTM {
    const float2 *sH;
    uint32_t ucol;
    __device__ __forceinline__ void two(float2 (&u0)[16], float2 (&u1)[16], int base) {
        MidMulH<N>{sH}.two(u0, u1, base);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            tm_store4(ucol + 16 * q, make_float4(u0[4 * q].x, u0[4 * q].y, u1[4 * q].x, u1[4 * q].y),
                      make_float4(u0[4 * q + 1].x, u0[4 * q + 1].y, u1[4 * q + 1].x, u1[4 * q + 1].y),
                      make_float4(u0[4 * q + 2].x, u0[4 * q + 2].y, u1[4 * q + 2].x, u1[4 * q + 2].y),
                      make_float4(u0[4 * q + 3].x, u0[4 * q + 3].y, u1[4 * q + 3].x, u1[4 * q + 3].y));
        tm_wait_st();
    }
    template <int R>
    __device__ __forceinline__ void one(float2 (&u)[R], int pol, int base) {
        static_assert(R == 32, "64 columns: 32 complex values of one polarization");
        MidMulH<N>{sH}.one(u, pol, base);
#pragma unroll
        for (int q = 0; q < R / 8; ++q)
            tm_store4(ucol + 16 * q, make_float4(u[8 * q].x, u[8 * q].y, u[8 * q + 1].x, u[8 * q + 1].y),
                      make_float4(u[8 * q + 2].x, u[8 * q + 2].y, u[8 * q + 3].x, u[8 * q + 3].y),
                      make_float4(u[8 * q + 4].x, u[8 * q + 4].y, u[8 * q + 5].x, u[8 * q + 5].y),
                      make_float4(u[8 * q + 6].x, u[8 * q + 6].y, u[8 * q + 7].x, u[8 * q + 7].y));
        tm_wait_st();
    }
};

// MidAdjoint with U read from TMEM, four positions at a time
template <int N>
struct MidAdjointTM {
    const float2 *sH;
    uint32_t ucol;
    float cphi;
    float acc;
    __device__ __forceinline__ void two(float2 (&u0)[16], float2 (&u1)[16], int base) {
        MidAdjoint<N> m{sH, nullptr, cphi, 0.f};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 uu[4];
            tm_load4(ucol + 16 * q, uu);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int j = 4 * q + jj;
                acc = fmaf(m.phi_prime(base + j),
                           MidAdjoint<N>::mimag(u0[j], make_float2(uu[jj].x, uu[jj].y)) +
                               MidAdjoint<N>::mimag(u1[j], make_float2(uu[jj].z, uu[jj].w)),
                           acc);
            }
        }
        const float4 *hrow = reinterpret_cast<const float4 *>(sH + hphys<16>(base));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float4 h = hrow[j];
            u0[2 * j] = cmulc(u0[2 * j], make_float2(h.x, h.y));
            u1[2 * j] = cmulc(u1[2 * j], make_float2(h.x, h.y));
            u0[2 * j + 1] = cmulc(u0[2 * j + 1], make_float2(h.z, h.w));
            u1[2 * j + 1] = cmulc(u1[2 * j + 1], make_float2(h.z, h.w));
        }
    }
    template <int R>
    __device__ __forceinline__ void one(float2 (&u)[R], int pol, int base) {
        static_assert(R == 32, "64 columns: 32 complex values of one polarization");
        MidAdjoint<N> m{sH, nullptr, cphi, 0.f};
#pragma unroll
        for (int q = 0; q < R / 8; ++q) {
            float4 uu[4];
            tm_load4(ucol + 16 * q, uu);
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int j = 8 * q + 2 * jj;
                acc = fmaf(m.phi_prime(base + j), MidAdjoint<N>::mimag(u[j], make_float2(uu[jj].x, uu[jj].y)), acc);
                acc = fmaf(m.phi_prime(base + j + 1), MidAdjoint<N>::mimag(u[j + 1], make_float2(uu[jj].z, uu[jj].w)),
                           acc);
            }
        }
        const float4 *hrow = reinterpret_cast<const float4 *>(sH + hphys<R>(base));
#pragma unroll
        for (int j = 0; j < R / 2; ++j) {
            const float4 h = hrow[j];
            u[2 * j] = cmulc(u[2 * j], make_float2(h.x, h.y));
            u[2 * j + 1] = cmulc(u[2 * j + 1], make_float2(h.z, h.w));
        }
    }
};

// The adjoint's three pass-3 operations behind one run-time selector (uniform across the
// CTA), so that one non-inlined copy of the pass-3 DFTs serves the forward sweep (x H),
// the recomputed linear sub-step (x H, keep U) and the linear adjoint (dL/ddz, x conj(H)).
enum { MID_MULH = 0, MID_RECOMPUTE = 1, MID_ADJOINT = 2 };
template <int N, bool TM>
struct MidSelect {
    int mode;
    const float2 *sH;
    uint32_t ucol;   // TM: the thread's U columns
    float4 *U;       // otherwise: the block's U scratch
    float cphi;
    float acc;
    __device__ __forceinline__ void two(float2 (&u0)[16], float2 (&u1)[16], int base) {
        if (mode == MID_MULH) {
            MidMulH<N>{sH}.two(u0, u1, base);
        } else if (mode == MID_RECOMPUTE) {
            if constexpr (TM) {
                MidRecomputeTM<N>{sH, ucol}.two(u0, u1, base);
            } else {
                MidRecompute<N>{sH, U}.two(u0, u1, base);
            }
        } else {
            if constexpr (TM) {
                MidAdjointTM<N> m{sH, ucol, cphi, acc};
                m.two(u0, u1, base);
                acc = m.acc;
            } else {
                MidAdjoint<N> m{sH, U, cphi, acc};
                m.two(u0, u1, base);
                acc = m.acc;
            }
        }
    }
    template <int R>
    __device__ __forceinline__ void one(float2 (&u)[R], int pol, int base) {
        if (mode == MID_MULH) {
            MidMulH<N>{sH}.one(u, pol, base);
        } else if (mode == MID_RECOMPUTE) {
            if constexpr (TM) {
                MidRecomputeTM<N>{sH, ucol}.one(u, pol, base);
            } else {
                MidRecompute<N>{sH, U}.one(u, pol, base);
            }
        } else {
            if constexpr (TM) {
                MidAdjointTM<N> m{sH, ucol, cphi, acc};
                m.one(u, pol, base);
                acc = m.acc;
            } else {
                MidAdjoint<N> m{sH, U, cphi, acc};
                m.one(u, pol, base);
                acc = m.acc;
            }
        }
    }
};

// Pass 3 of the adjoint as one called copy (pointers and scalars only cross the call);
// returns the dL/ddz accumulator of MID_ADJOINT (0 otherwise).
template <int N, bool TM>
__device__ __noinline__ float pass3_one_copy(int t, float4 *xs, int mode, const float2 *sH, uint32_t ucol,
                                             float4 *U, float cphi) {
    MidSelect<N, TM> mid{mode, sH, ucol, U, cphi, 0.f};
    Blk<N>::pass3_at(t, xs, mid);
    return mid.acc;
}

template <int N, bool ESSFM, bool FAST = false>
__global__ void __launch_bounds__(Geo<N>::T, (N == 4096) ? 2 : 1) dbp_adj_kernel(const AdjParams q) {
    using B = Blk<N>;
    using G = Geo<N>;
    const FwdParams &p = q.f;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    B blk(smem_raw, threadIdx.x);
    const int t = threadIdx.x;
    // the gather and reduction kernels that follow (launched as programmatic dependents)
    // may be scheduled once every CTA of this grid has started; they wait for its end
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    // N = 4096 (two CTAs per SM) and N = 8192 (one): U and g in tensor memory (128 columns
    // a thread: 256 columns per CTA at N = 4096, all 512 at N = 8192), y in global scratch
    constexpr bool TM = (N == 4096 || N == 8192);
    constexpr uint32_t TM_COLS = (uint32_t)G::T;   // 128 columns for each group of four warps
    __shared__ uint32_t s_tmem;
    uint32_t tcol = 0;
    if constexpr (TM) {
        static_assert((G::T == 256 || G::T == 512) && B::C1 == 1 && B::N2 == 16, "thread-own scratch layout");
        if (t < 32) {
            tmem_alloc(&s_tmem, TM_COLS);
            tmem_relinquish();
        }
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        const int warp = t >> 5;
        tcol = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 128u * (uint32_t)(warp >> 2);
    }
    const uint32_t tm_u = tcol, tm_g = tcol + 64;
    const int blkid = blockIdx.x;
    const int w = blkid / p.n_blocks;
    const int b = blkid - w * p.n_blocks;
    const long long n = p.n;
    const int ns = p.n_steps;
    const float2 *__restrict__ in = p.in + (size_t)w * 2 * n;
    const float2 *__restrict__ gout = q.gout + (size_t)w * 2 * n;
    const long long win0 = (long long)b * p.valid - p.half_overlap;
    float4 *__restrict__ gb = q.gblk + (size_t)blkid * N;
    float4 *__restrict__ ub = q.uscr + (size_t)blkid * N;
    float4 *__restrict__ yb = q.yscr + (size_t)blkid * N;
    // this warp's row of partial sums: R_{s,i} then dL/ddz_s
    float *__restrict__ part = q.part + ((size_t)blkid * (G::T / 32) + (threadIdx.x >> 5)) * (ns * q.nr + ns);

    blk.prefetch_h(p.H);
    blk.load_tables(p.twA, p.twB, p.tw2);
    typename B::Regs v;
    blk.load_window(v, in, n, win0, p.boundary);

    // output gradient in the block's valid region, zero in the discarded overlap
    {
        const int h = p.half_overlap;
        const long long obase = (long long)b * p.valid - h;
        auto gval = [&](int i, int j) {
            const int e = blk.pos1(i, j);
            const long long g = obase + e;
            float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
            if (e >= h && e < h + p.valid && g < n) {
                const float2 g0 = __ldg(gout + g), g1 = __ldg(gout + n + g);
                val = make_float4(g0.x, g0.y, g1.x, g1.y);
            }
            return val;
        };
        if constexpr (TM) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                tm_store4(tm_g + 16 * q, gval(0, 4 * q), gval(0, 4 * q + 1), gval(0, 4 * q + 2), gval(0, 4 * q + 3));
            tm_wait_st();
        } else {
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int j = 0; j < B::N2; ++j) gb[blk.pos1(i, j)] = gval(i, j);
        }
    }
    __syncthreads();

    // ---- forward sweep: steps 0..ns-2, storing each next step's input
    for (int s = 0; s + 1 < ns; ++s) {
        if (s > 0) {
            __syncthreads();
            if (p.h_stride != 0) blk.prefetch_h(p.H + p.h_stride * s);
        }
        blk.pass1_fwd(v);
        __syncthreads();
        pass2_one_copy<N, false>(t, blk.xs, blk.s2);
        cp_async_wait_all();
        __syncwarp();   // passes 2 -> 3 -> 2' stay inside a warp (as in the forward kernel)
        pass3_one_copy<N, TM>(t, blk.xs, MID_MULH, blk.sH, tm_u, ub, q.cphi);
        __syncwarp();
        pass2_one_copy<N, true>(t, blk.xs, blk.s2);
        __syncthreads();
        blk.pass1_inv(v);
        const float *__restrict__ a = p.taps + p.taps_stride * s;
        if constexpr (ESSFM) {
            __syncthreads();
            blk.stage_taps(a, p.taps_stride);
            blk.template essfm_theta<-1, true>(v, blk.sa, p.n_tapblk);
        }
        const float a0 = __ldg(a);
        float4 *ck = q.ckpt + ((size_t)blkid * (ns - 1) + s) * N;
#pragma unroll
        for (int i = 0; i < B::C1; ++i)
#pragma unroll
            for (int j = 0; j < B::N2; ++j) {
                const int e = blk.pos1(i, j);
                const float th = ESSFM ? blk.farr(1)[pphys(e)] : a0 * joint_intensity(v[0][i][j], v[1][i][j]);
                const float2 ex = expj<FAST>(th);
                v[0][i][j] = cmul(v[0][i][j], ex);
                v[1][i][j] = cmul(v[1][i][j], ex);
                ck[e] = make_float4(v[0][i][j].x, v[0][i][j].y, v[1][i][j].x, v[1][i][j].y);
            }
    }

    // ---- reverse sweep
    for (int s = ns - 1; s >= 0; --s) {
        __syncthreads();
        if (s < ns - 1) {
            if (p.h_stride != 0) blk.prefetch_h(p.H + p.h_stride * s);
            if (s == 0) {
                blk.load_window(v, in, n, win0, p.boundary);
            } else {
                const float4 *ck = q.ckpt + ((size_t)blkid * (ns - 1) + (s - 1)) * N;
#pragma unroll
                for (int i = 0; i < B::C1; ++i)
#pragma unroll
                    for (int j = 0; j < B::N2; ++j) {
                        const float4 f = ck[blk.pos1(i, j)];
                        v[0][i][j] = make_float2(f.x, f.y);
                        v[1][i][j] = make_float2(f.z, f.w);
                    }
            }
        } else if (ns > 1 && p.h_stride != 0) {
            blk.prefetch_h(p.H + p.h_stride * s);
        }
        // recompute the linear sub-step, keeping U = H' X
        blk.pass1_fwd(v);
        __syncthreads();
        pass2_one_copy<N, false>(t, blk.xs, blk.s2);
        cp_async_wait_all();
        __syncwarp();
        pass3_one_copy<N, TM>(t, blk.xs, MID_RECOMPUTE, blk.sH, tm_u, ub, q.cphi);   // keeps U
        __syncwarp();
        pass2_one_copy<N, true>(t, blk.xs, blk.s2);
        __syncthreads();
        blk.pass1_inv(v);   // v = y
        const float *__restrict__ a = p.taps + p.taps_stride * s;
        float *rp = part + s * q.nr;
        if constexpr (ESSFM) {
            __syncthreads();
            blk.stage_taps(a, p.taps_stride);
            blk.template essfm_theta<-1, true>(v, blk.sa, p.n_tapblk);
            float *sS = blk.farr(2);
            const float *sT = blk.farr(1);
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int q = 0; q < B::N2 / 4; ++q) {
                    float4 gq[4];
                    if constexpr (TM) tm_load4(tm_g + 16 * q, gq);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = 4 * q + jj;
                        const int e = blk.pos1(i, j);
                        const float2 ex = expj<FAST>(sT[pphys(e)]);
                        const float2 y0 = v[0][i][j], y1 = v[1][i][j];
                        const float2 z0 = cmul(y0, ex), z1 = cmul(y1, ex);
                        const float4 g = TM ? gq[jj] : gb[e];
                        const float2 g0 = make_float2(g.x, g.y), g1 = make_float2(g.z, g.w);
                        sS[pphys(e)] = MidAdjoint<N>::mimag(g0, z0) + MidAdjoint<N>::mimag(g1, z1);
                        const float2 d0 = cmulc(g0, ex), d1 = cmulc(g1, ex);
                        gq[jj] = make_float4(d0.x, d0.y, d1.x, d1.y);
                        if constexpr (!TM) gb[e] = gq[jj];
                        yb[e] = make_float4(y0.x, y0.y, y1.x, y1.y);
                    }
                    if constexpr (TM) tm_store4(tm_g + 16 * q, gq[0], gq[1], gq[2], gq[3]);
                }
            if constexpr (TM) tm_wait_st();
            __syncthreads();
            // correlations R_i = sum_k s_k S_{k,i}, then dL/dP = filter(s) into farr(1)
            {
                const float *sP = blk.farr(0);
                const int k0 = 16 * t;
                float sk[16];
                {
                    const float4 *ps = reinterpret_cast<const float4 *>(sS + pphys(k0));
                    const float4 *pp = reinterpret_cast<const float4 *>(sP + pphys(k0));
                    float r0[1] = {0.f};
#pragma unroll
                    for (int qd = 0; qd < 4; ++qd) {
                        const float4 fs = ps[qd], fp = pp[qd];
                        sk[4 * qd + 0] = fs.x; sk[4 * qd + 1] = fs.y; sk[4 * qd + 2] = fs.z; sk[4 * qd + 3] = fs.w;
                        r0[0] = fmaf(fs.x, fp.x, fmaf(fs.y, fp.y, fmaf(fs.z, fp.z, fmaf(fs.w, fp.w, r0[0]))));
                    }
                    warp_sum<1>(r0, rp);
                }
                for (int tb = 0; tb < p.n_tapblk; ++tb) {
                    const int i0 = 8 * tb;
                    float lw[24], rw[24];
#pragma unroll
                    for (int qd = 0; qd < 6; ++qd) {
                        const int el = (k0 - i0 - 8 + 4 * qd) & (N - 1);
                        const int er = (k0 + i0 + 4 * qd) & (N - 1);
                        const float4 fl = *reinterpret_cast<const float4 *>(sP + pphys(el));
                        const float4 fr = *reinterpret_cast<const float4 *>(sP + pphys(er));
                        lw[4 * qd + 0] = fl.x; lw[4 * qd + 1] = fl.y; lw[4 * qd + 2] = fl.z; lw[4 * qd + 3] = fl.w;
                        rw[4 * qd + 0] = fr.x; rw[4 * qd + 1] = fr.y; rw[4 * qd + 2] = fr.z; rw[4 * qd + 3] = fr.w;
                    }
                    float acc[8];
#pragma unroll
                    for (int ii = 1; ii <= 8; ++ii) {
                        float x = 0.f;
#pragma unroll
                        for (int r = 0; r < 16; ++r) x = fmaf(sk[r], lw[r - ii + 8] + rw[r + ii], x);
                        acc[ii - 1] = x;
                    }
                    warp_sum<8>(acc, rp + 1 + i0);
                }
                fir16_one_copy<N>(t, sS, blk.farr(1), blk.sa, p.n_tapblk);
            }
            __syncthreads();
            const float *sD = blk.farr(1);
            if constexpr (TM) {
#pragma unroll
                for (int q = 0; q < B::N2 / 4; ++q) {
                    float4 gq[4];
                    tm_load4(tm_g + 16 * q, gq);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = 4 * q + jj;
                        const int e = blk.pos1(0, j);
                        const float dp2 = 2.f * sD[pphys(e)];
                        const float4 g = gq[jj], y = yb[e];
                        v[0][0][j] = make_float2(fmaf(dp2, y.x, g.x), fmaf(dp2, y.y, g.y));
                        v[1][0][j] = make_float2(fmaf(dp2, y.z, g.z), fmaf(dp2, y.w, g.w));
                    }
                }
            } else {
#pragma unroll
                for (int i = 0; i < B::C1; ++i)
#pragma unroll
                    for (int j = 0; j < B::N2; ++j) {
                        const int e = blk.pos1(i, j);
                        const float dp2 = 2.f * sD[pphys(e)];
                        const float4 g = gb[e], y = yb[e];
                        v[0][i][j] = make_float2(fmaf(dp2, y.x, g.x), fmaf(dp2, y.y, g.y));
                        v[1][i][j] = make_float2(fmaf(dp2, y.z, g.z), fmaf(dp2, y.w, g.w));
                    }
            }
        } else {
            const float a0 = __ldg(a);
            float r0[1] = {0.f};
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int j = 0; j < B::N2; ++j) {
                    const int e = blk.pos1(i, j);
                    float4 gq[4];
                    if (TM && (j & 3) == 0) tm_load4(tm_g + 4 * j, gq);
                    const float2 y0 = v[0][i][j], y1 = v[1][i][j];
                    const float pk = joint_intensity(y0, y1);
                    const float2 ex = expj<FAST>(a0 * pk);
                    const float2 z0 = cmul(y0, ex), z1 = cmul(y1, ex);
                    const float4 g = TM ? gq[j & 3] : gb[e];
                    const float2 g0 = make_float2(g.x, g.y), g1 = make_float2(g.z, g.w);
                    const float sk = MidAdjoint<N>::mimag(g0, z0) + MidAdjoint<N>::mimag(g1, z1);
                    r0[0] = fmaf(sk, pk, r0[0]);
                    const float dp2 = 2.f * a0 * sk;
                    const float2 d0 = cmulc(g0, ex), d1 = cmulc(g1, ex);
                    v[0][i][j] = make_float2(fmaf(dp2, y0.x, d0.x), fmaf(dp2, y0.y, d0.y));
                    v[1][i][j] = make_float2(fmaf(dp2, y1.x, d1.x), fmaf(dp2, y1.y, d1.y));
                }
            warp_sum<1>(r0, rp);
        }
        // linear adjoint: x conj(H'), with the step-length gradient
        __syncthreads();
        blk.pass1_fwd(v);
        __syncthreads();
        pass2_one_copy<N, false>(t, blk.xs, blk.s2);
        __syncwarp();
        const float dzacc = pass3_one_copy<N, TM>(t, blk.xs, MID_ADJOINT, blk.sH, tm_u, ub, q.cphi);
        __syncwarp();
        pass2_one_copy<N, true>(t, blk.xs, blk.s2);
        __syncthreads();
        blk.pass1_inv(v);   // v = g_x
        {
            float dz[1] = {dzacc};
            warp_sum<1>(dz, part + ns * q.nr + s);
        }
        if (TM && s > 0) {   // the next (earlier) step's output gradient stays in TMEM
            auto gx = [&](int j) { return make_float4(v[0][0][j].x, v[0][0][j].y, v[1][0][j].x, v[1][0][j].y); };
#pragma unroll
            for (int q = 0; q < 4; ++q) tm_store4(tm_g + 16 * q, gx(4 * q), gx(4 * q + 1), gx(4 * q + 2), gx(4 * q + 3));
            tm_wait_st();
        } else {
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int j = 0; j < B::N2; ++j)
                    gb[blk.pos1(i, j)] = make_float4(v[0][i][j].x, v[0][i][j].y, v[1][i][j].x, v[1][i][j].y);
        }
    }
    if constexpr (TM) {   // every tcgen05 access has been waited for; free the columns
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        if (t < 32) tmem_dealloc(s_tmem, TM_COLS);
    }
}

template <int N>
int launch_adj_n(const AdjParams &q, int n_wave, bool essfm, cudaStream_t st) {
    using G = Geo<N>;
    static unsigned long long done_e = 0, done_s = 0, done_f = 0;
    const size_t smem = G::SMEM;
    const long long grid = (long long)q.f.n_blocks * n_wave;
    if (grid <= 0 || grid > 0x7fffffffLL) return DBP_ERR_ARG;
    if (essfm && q.f.fast_exp) {   // the forward kernel's exponential for plans of at most two steps
        if (!set_smem_once(dbp_adj_kernel<N, true, true>, smem, done_f)) return DBP_ERR_CUDA;
        dbp_adj_kernel<N, true, true><<<(unsigned)grid, G::T, smem, st>>>(q);
    } else if (essfm) {
        if (!set_smem_once(dbp_adj_kernel<N, true>, smem, done_e)) return DBP_ERR_CUDA;
        dbp_adj_kernel<N, true><<<(unsigned)grid, G::T, smem, st>>>(q);
    } else {
        if (!set_smem_once(dbp_adj_kernel<N, false>, smem, done_s)) return DBP_ERR_CUDA;
        dbp_adj_kernel<N, false><<<(unsigned)grid, G::T, smem, st>>>(q);
    }
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

}  // namespace dbp
