// Fused overlap-save DBP kernel: one CTA per block of N vector samples, all N_s steps
// in shared memory / registers, FP32.
//
// Per step s (Section II, operations (i)-(iv), inverted for backpropagation):
//   pass 1  radix-N2 DFT over the top digit (stride N0 N1), twiddle W_N^{c k0}
//   pass 2  radix-N1 DFT (stride N0), twiddle W_{N0 N1}^{n0 k1}
//   pass 3  radix-N0 DFT (contiguous) -> x H_s (Eq. 1 inverse, digit-reversed table,
//           1/N folded in) -> radix-N0 inverse DFT        (all in registers)
//   pass 2' and pass 1' undo passes 2 and 1 (conjugate twiddles, inverse DFTs)
//   nonlinear sub-step: theta_k = gamma_eff_s (c_0 P_k + sum_i c_i (P_{k-i} + P_{k+i}))
//           with P_k = |y_k,1|^2 + |y_k,2|^2 (Eq. 3; Eq. 2 when N_c = 0); both
//           polarizations are rotated by exp(+j theta_k).
// Between steps the block stays in registers in the pass-1 layout, so a step costs
// four shared-memory exchanges (plus two for the ESSFM filter).  Both polarizations
// travel together as one float4 per position.  The next step's H table is prefetched
// into shared memory with cp.async while passes 1-2 run.  Overlap-and-save (Section
// III): the block reads input window [b V - O/2, b V - O/2 + N) and writes its central
// V = N - O samples.
#pragma once
#include "dbp_internal.cuh"
#include "dft_regs.cuh"

namespace dbp {

template <int N0>
__device__ __forceinline__ int xphys(int e) { return e + e / N0; }           // float4 slots
template <int N0>
__device__ __forceinline__ int hphys(int e) { return e + 2 * (e / N0); }     // float2 slots
__device__ __forceinline__ int pphys(int e) { return e + 4 * (e >> 4); }     // float slots

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// exp(+j theta) for the nonlinear rotation.
// Default: theta = q pi/2 + r with a three-constant Cody-Waite reduction (pi/2 =
// 1.5703125 + 4.837512969970703e-4 + 7.549790126404332e-8; the first two constants have
// 12 significant bits, so q times each is exact for |q| < 2^12, i.e. |theta| < 6400 rad),
// then Taylor polynomials of sin and cos on |r| <= pi/4 (truncation below 2e-9, under
// half an FP32 ulp), and the quadrant q mod 4 selects/negates.  With DBP_EXPJ_MUFU the
// reduction is by 2 pi and the hardware sine/cosine approximations are used instead
// (absolute error below 4e-7 on [-pi, pi]).
__device__ __forceinline__ float2 expj(float th) {
#ifdef DBP_EXPJ_MUFU
    const float k = rintf(th * 0.15915494309189535f);
    float r = fmaf(-k, 6.28125f, th);
    r = fmaf(-k, 1.9353071795864769e-3f, r);
    float s, c;
    __sincosf(r, &s, &c);
    return make_float2(c, s);
#else
    const float q = rintf(th * 0.63661977236758134f);
    float r = fmaf(-q, 1.5703125f, th);
    r = fmaf(-q, 4.837512969970703e-4f, r);
    r = fmaf(-q, 7.549790126404332e-8f, r);
    const float r2 = r * r;
    // sin r = r - r^3/3! + r^5/5! - r^7/7! + r^9/9!
    float ps = fmaf(r2, 2.7557319223985893e-6f, -1.9841269841269841e-4f);
    ps = fmaf(r2, ps, 8.3333333333333333e-3f);
    ps = fmaf(r2, ps, -1.6666666666666667e-1f);
    const float sn = fmaf(r * r2, ps, r);
    // cos r = 1 - r^2/2! + r^4/4! - r^6/6! + r^8/8! - r^10/10!
    float pc = fmaf(r2, -2.7557319223985891e-7f, 2.4801587301587302e-5f);
    pc = fmaf(r2, pc, -1.3888888888888889e-3f);
    pc = fmaf(r2, pc, 4.1666666666666667e-2f);
    pc = fmaf(r2, pc, -0.5f);
    const float cs = fmaf(r2, pc, 1.0f);
    const int quad = ((int)q) & 3;
    const float c1 = (quad & 1) ? sn : cs;
    const float s1 = (quad & 1) ? cs : sn;
    return make_float2((quad == 1 || quad == 2) ? -c1 : c1, (quad >= 2) ? -s1 : s1);
#endif
}

// Copies this step's H table (N float2, 16-byte chunks) into padded shared memory.
template <int N>
__device__ __forceinline__ void prefetch_h(float2 *sH, const float2 *__restrict__ H, int t) {
    using G = Geo<N>;
    constexpr int CHUNKS = N / 2;                      // 16-byte chunks
#pragma unroll
    for (int q = 0; q < CHUNKS / G::T; ++q) {
        const int ch = t + G::T * q;
        const int e = 2 * ch;                          // first float2 of the chunk
        cp_async16(sH + hphys<G::N0>(e), H + e);
    }
    cp_async_commit();
}

template <int N, bool ESSFM>
__global__ void __launch_bounds__(Geo<N>::T, Geo<N>::MINB) dbp_fwd_kernel(const FwdParams p) {
    using G = Geo<N>;
    constexpr int N0 = G::N0, N1 = G::N1, N2 = G::N2, T = G::T, S1 = G::S1;
    constexpr int C1 = 16 / N2;          // pass-1 columns per thread (both polarizations)
    constexpr int C2 = 16 / N1;          // pass-2 columns per thread (both polarizations)

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4 *xs = reinterpret_cast<float4 *>(smem_raw);
    float2 *sH = reinterpret_cast<float2 *>(smem_raw + G::OFF_H);
    float2 *sA = reinterpret_cast<float2 *>(smem_raw + G::OFF_TWA);
    float2 *sB = reinterpret_cast<float2 *>(smem_raw + G::OFF_TWB);
    float2 *s2 = reinterpret_cast<float2 *>(smem_raw + G::OFF_TW2);
    float *sP = reinterpret_cast<float *>(smem_raw);   // ESSFM: aliases the block buffer
    float *sT = sP + G::PADP;

    const int t = threadIdx.x;
    const int w = blockIdx.x / p.n_blocks;
    const int b = blockIdx.x - w * p.n_blocks;
    const long long n = p.n;
    const float2 *__restrict__ in = p.in + (size_t)w * 2 * n;
    float2 *__restrict__ out = p.out + (size_t)w * 2 * n;
    const long long win0 = (long long)b * p.valid - p.half_overlap;

    prefetch_h<N>(sH, p.H, t);
    for (int i = t; i < G::TWA; i += T) sA[i] = __ldg(p.twA + i);
    for (int i = t; i < G::TWB; i += T) sB[i] = __ldg(p.twB + i);
    for (int i = t; i < G::TW2; i += T) s2[i] = __ldg(p.tw2 + i);

    float2 v[2][C1][N2];

    // ---- load the block window in the pass-1 layout (coalesced across threads)
    if (win0 >= 0 && win0 + N <= n) {
#pragma unroll
        for (int pol = 0; pol < 2; ++pol)
#pragma unroll
            for (int i = 0; i < C1; ++i)
#pragma unroll
                for (int j = 0; j < N2; ++j)
                    v[pol][i][j] = __ldg(in + pol * n + win0 + (t + T * i) + S1 * j);
    } else {
#pragma unroll
        for (int pol = 0; pol < 2; ++pol)
#pragma unroll
            for (int i = 0; i < C1; ++i)
#pragma unroll
                for (int j = 0; j < N2; ++j) {
                    long long idx = win0 + (t + T * i) + S1 * j;
                    float2 val = make_float2(0.f, 0.f);
                    if (p.boundary == DBP_PERIODIC) {
                        idx %= n;
                        if (idx < 0) idx += n;
                        val = __ldg(in + pol * n + idx);
                    } else if (idx >= 0 && idx < n) {
                        val = __ldg(in + pol * n + idx);
                    }
                    v[pol][i][j] = val;
                }
    }
    __syncthreads();   // twiddle tables visible

    for (int s = 0; s < p.n_steps; ++s) {
        if (ESSFM && s > 0) __syncthreads();   // previous step's theta reads are done

        // ---- pass 1 (forward): DFT over the top digit, twiddle, to shared memory
#pragma unroll
        for (int i = 0; i < C1; ++i) {
            const int c = t + T * i;
            const float2 *ta = sA + (c & 15);
            const float2 *tb = sB + (c >> 4);
            Dft<N2, false>::run(v[0][i]);
            Dft<N2, false>::run(v[1][i]);
#pragma unroll
            for (int k = 1; k < N2; ++k) {
                const float2 wk = cmul(ta[16 * k], tb[(S1 / 16) * k]);
                v[0][i][k] = cmul(v[0][i][k], wk);
                v[1][i][k] = cmul(v[1][i][k], wk);
            }
#pragma unroll
            for (int k = 0; k < N2; ++k)
                xs[xphys<N0>(c + S1 * k)] = make_float4(v[0][i][k].x, v[0][i][k].y, v[1][i][k].x, v[1][i][k].y);
        }
        __syncthreads();

        // ---- pass 2 (forward): radix N1, stride N0
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            const int c2 = t + T * i;
            const int n0 = c2 % N0, k0 = c2 / N0;
            const int base = n0 + S1 * k0;
            float2 u0[N1], u1[N1];
#pragma unroll
            for (int j = 0; j < N1; ++j) {
                const float4 f = xs[xphys<N0>(base + N0 * j)];
                u0[j] = make_float2(f.x, f.y);
                u1[j] = make_float2(f.z, f.w);
            }
            Dft<N1, false>::run(u0);
            Dft<N1, false>::run(u1);
            const float2 *tw = s2 + n0;
#pragma unroll
            for (int k = 1; k < N1; ++k) {
                const float2 wk = tw[N0 * k];
                u0[k] = cmul(u0[k], wk);
                u1[k] = cmul(u1[k], wk);
            }
#pragma unroll
            for (int k = 0; k < N1; ++k)
                xs[xphys<N0>(base + N0 * k)] = make_float4(u0[k].x, u0[k].y, u1[k].x, u1[k].y);
        }
        cp_async_wait_all();
        __syncthreads();   // pass-2 results and H_s visible

        // ---- pass 3: contiguous radix-N0 DFT, x H_s, inverse DFT (registers only)
        if constexpr (N0 == 16) {
            const int base = 16 * t;
            float2 u0[16], u1[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float4 f = xs[xphys<16>(base + j)];
                u0[j] = make_float2(f.x, f.y);
                u1[j] = make_float2(f.z, f.w);
            }
            Dft<16, false>::run(u0);
            Dft<16, false>::run(u1);
            const float4 *hrow = reinterpret_cast<const float4 *>(sH + hphys<16>(base));
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 h = hrow[j];
                u0[2 * j] = cmul(u0[2 * j], make_float2(h.x, h.y));
                u1[2 * j] = cmul(u1[2 * j], make_float2(h.x, h.y));
                u0[2 * j + 1] = cmul(u0[2 * j + 1], make_float2(h.z, h.w));
                u1[2 * j + 1] = cmul(u1[2 * j + 1], make_float2(h.z, h.w));
            }
            Dft<16, true>::run(u0);
            Dft<16, true>::run(u1);
#pragma unroll
            for (int j = 0; j < 16; ++j) xs[xphys<16>(base + j)] = make_float4(u0[j].x, u0[j].y, u1[j].x, u1[j].y);
        } else {
            const int c3 = t >> 1, pol = t & 1;
            const int base = N0 * c3;
            float2 *xh = reinterpret_cast<float2 *>(xs);
            float2 u[N0];
#pragma unroll
            for (int j = 0; j < N0; ++j) u[j] = xh[2 * xphys<N0>(base + j) + pol];
            Dft<N0, false>::run(u);
            const float4 *hrow = reinterpret_cast<const float4 *>(sH + hphys<N0>(base));
#pragma unroll
            for (int j = 0; j < N0 / 2; ++j) {
                const float4 h = hrow[j];
                u[2 * j] = cmul(u[2 * j], make_float2(h.x, h.y));
                u[2 * j + 1] = cmul(u[2 * j + 1], make_float2(h.z, h.w));
            }
            Dft<N0, true>::run(u);
#pragma unroll
            for (int j = 0; j < N0; ++j) xh[2 * xphys<N0>(base + j) + pol] = u[j];
        }
        __syncthreads();
        if (p.h_stride != 0 && s + 1 < p.n_steps) prefetch_h<N>(sH, p.H + p.h_stride * (s + 1), t);

        // ---- pass 2' (inverse): conjugate twiddle, inverse radix-N1 DFT
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            const int c2 = t + T * i;
            const int n0 = c2 % N0, k0 = c2 / N0;
            const int base = n0 + S1 * k0;
            float2 u0[N1], u1[N1];
#pragma unroll
            for (int j = 0; j < N1; ++j) {
                const float4 f = xs[xphys<N0>(base + N0 * j)];
                u0[j] = make_float2(f.x, f.y);
                u1[j] = make_float2(f.z, f.w);
            }
            const float2 *tw = s2 + n0;
#pragma unroll
            for (int k = 1; k < N1; ++k) {
                const float2 wk = tw[N0 * k];
                u0[k] = cmulc(u0[k], wk);
                u1[k] = cmulc(u1[k], wk);
            }
            Dft<N1, true>::run(u0);
            Dft<N1, true>::run(u1);
#pragma unroll
            for (int k = 0; k < N1; ++k)
                xs[xphys<N0>(base + N0 * k)] = make_float4(u0[k].x, u0[k].y, u1[k].x, u1[k].y);
        }
        __syncthreads();

        // ---- pass 1' (inverse): conjugate twiddle, inverse radix-N2 DFT, into registers
#pragma unroll
        for (int i = 0; i < C1; ++i) {
            const int c = t + T * i;
            const float2 *ta = sA + (c & 15);
            const float2 *tb = sB + (c >> 4);
#pragma unroll
            for (int j = 0; j < N2; ++j) {
                const float4 f = xs[xphys<N0>(c + S1 * j)];
                v[0][i][j] = make_float2(f.x, f.y);
                v[1][i][j] = make_float2(f.z, f.w);
            }
#pragma unroll
            for (int k = 1; k < N2; ++k) {
                const float2 wk = cmul(ta[16 * k], tb[(S1 / 16) * k]);
                v[0][i][k] = cmulc(v[0][i][k], wk);
                v[1][i][k] = cmulc(v[1][i][k], wk);
            }
            Dft<N2, true>::run(v[0][i]);
            Dft<N2, true>::run(v[1][i]);
        }

        // ---- nonlinear sub-step
        const float *__restrict__ a = p.taps + p.taps_stride * s;
        if constexpr (ESSFM) {
            __syncthreads();   // block buffer free: P and theta reuse it
#pragma unroll
            for (int i = 0; i < C1; ++i)
#pragma unroll
                for (int j = 0; j < N2; ++j) {
                    const float2 y0 = v[0][i][j], y1 = v[1][i][j];
                    sP[pphys((t + T * i) + S1 * j)] =
                        fmaf(y0.x, y0.x, fmaf(y0.y, y0.y, fmaf(y1.x, y1.x, y1.y * y1.y)));
                }
            __syncthreads();
            // symmetric filter over 16 consecutive positions per thread, circular in the block
            {
                const int k0 = 16 * t;
                float th[16];
                {
                    const float4 *pc = reinterpret_cast<const float4 *>(sP + pphys(k0));
                    const float a0 = __ldg(a);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float4 f = pc[q];
                        th[4 * q + 0] = a0 * f.x;
                        th[4 * q + 1] = a0 * f.y;
                        th[4 * q + 2] = a0 * f.z;
                        th[4 * q + 3] = a0 * f.w;
                    }
                }
                for (int blk = 0; blk < p.n_tapblk; ++blk) {
                    const int i0 = 8 * blk;
                    float lw[24], rw[24];
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const int el = (k0 - i0 - 8 + 4 * q) & (N - 1);
                        const int er = (k0 + i0 + 4 * q) & (N - 1);
                        const float4 fl = *reinterpret_cast<const float4 *>(sP + pphys(el));
                        const float4 fr = *reinterpret_cast<const float4 *>(sP + pphys(er));
                        lw[4 * q + 0] = fl.x; lw[4 * q + 1] = fl.y; lw[4 * q + 2] = fl.z; lw[4 * q + 3] = fl.w;
                        rw[4 * q + 0] = fr.x; rw[4 * q + 1] = fr.y; rw[4 * q + 2] = fr.z; rw[4 * q + 3] = fr.w;
                    }
#pragma unroll
                    for (int ii = 1; ii <= 8; ++ii) {
                        const float ai = __ldg(a + i0 + ii);
#pragma unroll
                        for (int r = 0; r < 16; ++r) th[r] = fmaf(ai, lw[r - ii + 8] + rw[r + ii], th[r]);
                    }
                }
                float4 *pt = reinterpret_cast<float4 *>(sT + pphys(k0));
#pragma unroll
                for (int q = 0; q < 4; ++q) pt[q] = make_float4(th[4 * q], th[4 * q + 1], th[4 * q + 2], th[4 * q + 3]);
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < C1; ++i)
#pragma unroll
                for (int j = 0; j < N2; ++j) {
                    const float2 e = expj(sT[pphys((t + T * i) + S1 * j)]);
                    v[0][i][j] = cmul(v[0][i][j], e);
                    v[1][i][j] = cmul(v[1][i][j], e);
                }
        } else {
            const float a0 = __ldg(a);
#pragma unroll
            for (int i = 0; i < C1; ++i)
#pragma unroll
                for (int j = 0; j < N2; ++j) {
                    const float2 y0 = v[0][i][j], y1 = v[1][i][j];
                    const float2 e = expj(a0 * fmaf(y0.x, y0.x, fmaf(y0.y, y0.y, fmaf(y1.x, y1.x, y1.y * y1.y))));
                    v[0][i][j] = cmul(y0, e);
                    v[1][i][j] = cmul(y1, e);
                }
        }
    }

    // ---- overlap-and-save: keep the central V samples
    const int h = p.half_overlap;
    const long long obase = (long long)b * p.valid - h;
#pragma unroll
    for (int i = 0; i < C1; ++i)
#pragma unroll
        for (int j = 0; j < N2; ++j) {
            const int e = (t + T * i) + S1 * j;
            const long long g = obase + e;
            if (e >= h && e < h + p.valid && g < n) {
                __stcs(out + g, v[0][i][j]);
                __stcs(out + n + g, v[1][i][j]);
            }
        }
}

// Opt a kernel into more than 48 KB of dynamic shared memory, once per device.
template <typename K>
inline bool set_smem_once(K kernel, size_t bytes, unsigned long long &done_mask) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    const unsigned long long bit = 1ull << dev;
    if (done_mask & bit) return true;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
        return false;
    done_mask |= bit;
    return true;
}

template <int N>
int launch_fwd_n(const FwdParams &p, int n_wave, bool essfm, cudaStream_t st) {
    using G = Geo<N>;
    static unsigned long long done_essfm = 0, done_ssfm = 0;
    const long long grid = (long long)p.n_blocks * n_wave;
    if (grid <= 0 || grid > 0x7fffffffLL) return DBP_ERR_ARG;
    if (essfm) {
        if (!set_smem_once(dbp_fwd_kernel<N, true>, G::SMEM, done_essfm)) return DBP_ERR_CUDA;
        dbp_fwd_kernel<N, true><<<(unsigned)grid, G::T, G::SMEM, st>>>(p);
    } else {
        if (!set_smem_once(dbp_fwd_kernel<N, false>, G::SMEM, done_ssfm)) return DBP_ERR_CUDA;
        dbp_fwd_kernel<N, false><<<(unsigned)grid, G::T, G::SMEM, st>>>(p);
    }
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

}  // namespace dbp
