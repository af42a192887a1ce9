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
// The block lives in registers in the pass-1 layout between steps, so a step costs
// four shared-memory exchanges (plus two for the ESSFM filter).  Overlap-and-save
// (Section III): the block reads input window [b V - O/2, b V - O/2 + N) and writes its
// central V = N - O samples.
#pragma once
#include "dbp_internal.cuh"
#include "dft_regs.cuh"

namespace dbp {

template <int N0>
__device__ __forceinline__ int xphys(int e) { return e + 2 * (e / N0); }
__device__ __forceinline__ int pphys(int e) { return e + 4 * (e >> 4); }

template <int N, bool ESSFM>
__global__ void __launch_bounds__(Geo<N>::T, Geo<N>::MINB) dbp_fwd_kernel(const FwdParams p) {
    using G = Geo<N>;
    constexpr int N0 = G::N0, N1 = G::N1, N2 = G::N2, T = G::T, S1 = G::S1;
    constexpr int C1 = 16 / N2;          // pass-1 columns per polarization per thread
    constexpr int C2 = 16 / N1;          // pass-2 columns per polarization per thread
    constexpr int C3 = 32 / N0;          // pass-3 columns per thread (both polarizations)

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *sx = reinterpret_cast<float2 *>(smem_raw);            // [2][PADN]
    float *sP = reinterpret_cast<float *>(sx + 2 * G::PADN);       // [PADP]
    float *sT = sP + G::PADP;                                       // [PADP]

    const int t = threadIdx.x;
    const int w = blockIdx.x / p.n_blocks;
    const int b = blockIdx.x - w * p.n_blocks;
    const long long n = p.n;
    const float2 *__restrict__ in = p.in + (size_t)w * 2 * n;
    float2 *__restrict__ out = p.out + (size_t)w * 2 * n;
    const long long win0 = (long long)b * p.valid - p.half_overlap;

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

    for (int s = 0; s < p.n_steps; ++s) {
        const float2 *__restrict__ Hs = p.H + p.h_stride * s;

        // ---- pass 1 (forward): DFT over the top digit, twiddle, to shared memory
#pragma unroll
        for (int i = 0; i < C1; ++i) {
            const int c = t + T * i;
            const float2 *tw = p.tw1 + c * N2;
#pragma unroll
            for (int pol = 0; pol < 2; ++pol) Dft<N2, false>::run(v[pol][i]);
#pragma unroll
            for (int k = 1; k < N2; ++k) {
                const float2 wk = __ldg(tw + k);
                v[0][i][k] = cmul(v[0][i][k], wk);
                v[1][i][k] = cmul(v[1][i][k], wk);
            }
#pragma unroll
            for (int pol = 0; pol < 2; ++pol)
#pragma unroll
                for (int k = 0; k < N2; ++k) sx[pol * G::PADN + xphys<N0>(c + S1 * k)] = v[pol][i][k];
        }
        __syncthreads();

        // ---- pass 2 (forward): radix N1, stride N0
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            const int c2 = t + T * i;
            const int n0 = c2 % N0, k0 = c2 / N0;
            const int base = n0 + S1 * k0;
            float2 u[2][N1];
#pragma unroll
            for (int pol = 0; pol < 2; ++pol) {
#pragma unroll
                for (int j = 0; j < N1; ++j) u[pol][j] = sx[pol * G::PADN + xphys<N0>(base + N0 * j)];
                Dft<N1, false>::run(u[pol]);
            }
            const float2 *tw = p.tw2 + n0 * N1;
#pragma unroll
            for (int k = 1; k < N1; ++k) {
                const float2 wk = __ldg(tw + k);
                u[0][k] = cmul(u[0][k], wk);
                u[1][k] = cmul(u[1][k], wk);
            }
#pragma unroll
            for (int pol = 0; pol < 2; ++pol)
#pragma unroll
                for (int k = 0; k < N1; ++k) sx[pol * G::PADN + xphys<N0>(base + N0 * k)] = u[pol][k];
        }
        __syncthreads();

        // ---- pass 3: contiguous radix-N0 DFT, x H_s, inverse DFT (registers only)
#pragma unroll
        for (int i = 0; i < C3; ++i) {
            const int q = t + T * i;
            const int pol = q / (N / N0);
            const int c3 = q - pol * (N / N0);
            const int base = N0 * c3;
            float2 u[N0];
            float4 *row = reinterpret_cast<float4 *>(sx + pol * G::PADN + xphys<N0>(base));
#pragma unroll
            for (int j = 0; j < N0 / 2; ++j) {
                float4 f = row[j];
                u[2 * j] = make_float2(f.x, f.y);
                u[2 * j + 1] = make_float2(f.z, f.w);
            }
            Dft<N0, false>::run(u);
            const float4 *hrow = reinterpret_cast<const float4 *>(Hs + base);
#pragma unroll
            for (int j = 0; j < N0 / 2; ++j) {
                float4 h = __ldg(hrow + j);
                u[2 * j] = cmul(u[2 * j], make_float2(h.x, h.y));
                u[2 * j + 1] = cmul(u[2 * j + 1], make_float2(h.z, h.w));
            }
            Dft<N0, true>::run(u);
#pragma unroll
            for (int j = 0; j < N0 / 2; ++j)
                row[j] = make_float4(u[2 * j].x, u[2 * j].y, u[2 * j + 1].x, u[2 * j + 1].y);
        }
        __syncthreads();

        // ---- pass 2' (inverse): conjugate twiddle, inverse radix-N1 DFT
#pragma unroll
        for (int i = 0; i < C2; ++i) {
            const int c2 = t + T * i;
            const int n0 = c2 % N0, k0 = c2 / N0;
            const int base = n0 + S1 * k0;
            float2 u[2][N1];
            const float2 *tw = p.tw2 + n0 * N1;
#pragma unroll
            for (int pol = 0; pol < 2; ++pol)
#pragma unroll
                for (int j = 0; j < N1; ++j) u[pol][j] = sx[pol * G::PADN + xphys<N0>(base + N0 * j)];
#pragma unroll
            for (int k = 1; k < N1; ++k) {
                const float2 wk = __ldg(tw + k);
                u[0][k] = cmulc(u[0][k], wk);
                u[1][k] = cmulc(u[1][k], wk);
            }
#pragma unroll
            for (int pol = 0; pol < 2; ++pol) {
                Dft<N1, true>::run(u[pol]);
#pragma unroll
                for (int k = 0; k < N1; ++k) sx[pol * G::PADN + xphys<N0>(base + N0 * k)] = u[pol][k];
            }
        }
        __syncthreads();

        // ---- pass 1' (inverse): conjugate twiddle, inverse radix-N2 DFT, into registers
#pragma unroll
        for (int i = 0; i < C1; ++i) {
            const int c = t + T * i;
            const float2 *tw = p.tw1 + c * N2;
#pragma unroll
            for (int pol = 0; pol < 2; ++pol)
#pragma unroll
                for (int j = 0; j < N2; ++j) v[pol][i][j] = sx[pol * G::PADN + xphys<N0>(c + S1 * j)];
#pragma unroll
            for (int k = 1; k < N2; ++k) {
                const float2 wk = __ldg(tw + k);
                v[0][i][k] = cmulc(v[0][i][k], wk);
                v[1][i][k] = cmulc(v[1][i][k], wk);
            }
#pragma unroll
            for (int pol = 0; pol < 2; ++pol) Dft<N2, true>::run(v[pol][i]);
        }

        // ---- nonlinear sub-step
        const float *__restrict__ a = p.taps + p.taps_stride * s;
        if constexpr (ESSFM) {
            // joint intensity to shared memory (natural order)
#pragma unroll
            for (int i = 0; i < C1; ++i)
#pragma unroll
                for (int j = 0; j < N2; ++j) {
                    const float2 y0 = v[0][i][j], y1 = v[1][i][j];
                    sP[pphys((t + T * i) + S1 * j)] = fmaf(y0.x, y0.x, fmaf(y0.y, y0.y, fmaf(y1.x, y1.x, y1.y * y1.y)));
                }
            __syncthreads();
            // symmetric FIR over 16 consecutive positions per thread, circular in the block
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
                    const float th = sT[pphys((t + T * i) + S1 * j)];
                    float sn, cs;
                    sincosf(th, &sn, &cs);
                    const float2 e = make_float2(cs, sn);
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
                    const float th = a0 * fmaf(y0.x, y0.x, fmaf(y0.y, y0.y, fmaf(y1.x, y1.x, y1.y * y1.y)));
                    float sn, cs;
                    sincosf(th, &sn, &cs);
                    const float2 e = make_float2(cs, sn);
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
        if (!set_smem_once(dbp_fwd_kernel<N, true>, G::SMEM_ESSFM, done_essfm)) return DBP_ERR_CUDA;
        dbp_fwd_kernel<N, true><<<(unsigned)grid, G::T, G::SMEM_ESSFM, st>>>(p);
    } else {
        if (!set_smem_once(dbp_fwd_kernel<N, false>, G::SMEM_SSFM, done_ssfm)) return DBP_ERR_CUDA;
        dbp_fwd_kernel<N, false><<<(unsigned)grid, G::T, G::SMEM_SSFM, st>>>(p);
    }
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

}  // namespace dbp
