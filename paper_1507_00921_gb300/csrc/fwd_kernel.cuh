// Fused overlap-save DBP kernel: one CTA per block of N vector samples, all N_s steps
// in shared memory / registers, FP32.
//
// Per step s (Section II, operations (i)-(iv), inverted for backpropagation): FFT of
// both polarizations, x H_s (Eq. 1 inverse, 1/N folded in) fused into the contiguous
// FFT pass, IFFT, then the nonlinear sub-step
//   theta_k = gamma_eff_s (c_0 P_k + sum_i c_i (P_{k-i} + P_{k+i})),
//   P_k = |y_k,1|^2 + |y_k,2|^2          (Eq. 3; Eq. 2 when N_c = 0)
// and both polarizations rotated by exp(+j theta_k).  Between steps the block stays in
// registers in the pass-1 layout, so a step costs four shared-memory exchanges (plus two
// for the ESSFM filter).  The next step's H table is prefetched into shared memory with
// cp.async while passes 1-2 run.  Overlap-and-save (Section III): the block reads input
// window [b V - O/2, b V - O/2 + N) and writes its central V = N - O samples.
#pragma once
#include "block_fft.cuh"

namespace dbp {

template <int N, bool ESSFM>
__global__ void __launch_bounds__(Geo<N>::T, Geo<N>::MINB) dbp_fwd_kernel(const FwdParams p) {
    using B = Blk<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    B blk(smem_raw, threadIdx.x);

    const int w = blockIdx.x / p.n_blocks;
    const int b = blockIdx.x - w * p.n_blocks;
    const long long n = p.n;
    const float2 *__restrict__ in = p.in + (size_t)w * 2 * n;
    float2 *__restrict__ out = p.out + (size_t)w * 2 * n;
    const long long win0 = (long long)b * p.valid - p.half_overlap;

    blk.prefetch_h(p.H);
    blk.load_tables(p.twA, p.twB, p.tw2);
    typename B::Regs v;
    blk.load_window(v, in, n, win0, p.boundary);
    __syncthreads();   // twiddle tables visible

    MidMulH<N> mid{blk.sH};
    for (int s = 0; s < p.n_steps; ++s) {
        if (ESSFM && s > 0) __syncthreads();   // previous step's theta reads are done
        blk.pass1_fwd(v);
        __syncthreads();
        blk.template pass2<false>();
        cp_async_wait_all();
        __syncthreads();   // pass-2 results and H_s visible
        blk.pass3(mid);
        __syncthreads();
        if (p.h_stride != 0 && s + 1 < p.n_steps) blk.prefetch_h(p.H + p.h_stride * (s + 1));
        blk.template pass2<true>();
        __syncthreads();
        blk.pass1_inv(v);

        // ---- nonlinear sub-step
        const float *__restrict__ a = p.taps + p.taps_stride * s;
        if constexpr (ESSFM) {
            __syncthreads();   // block buffer free: P and theta reuse it
            blk.essfm_theta(v, a, p.n_tapblk);
            const float *sT = blk.farr(1);
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int j = 0; j < B::N2; ++j) {
                    const float2 e = expj(sT[pphys(blk.pos1(i, j))]);
                    v[0][i][j] = cmul(v[0][i][j], e);
                    v[1][i][j] = cmul(v[1][i][j], e);
                }
        } else {
            const float a0 = __ldg(a);
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int j = 0; j < B::N2; ++j) {
                    const float2 y0 = v[0][i][j], y1 = v[1][i][j];
                    const float2 e = expj(a0 * joint_intensity(y0, y1));
                    v[0][i][j] = cmul(y0, e);
                    v[1][i][j] = cmul(y1, e);
                }
        }
    }

    // ---- overlap-and-save: keep the central V samples
    const int h = p.half_overlap;
    const long long obase = (long long)b * p.valid - h;
#pragma unroll
    for (int i = 0; i < B::C1; ++i)
#pragma unroll
        for (int j = 0; j < B::N2; ++j) {
            const int e = blk.pos1(i, j);
            const long long g = obase + e;
            if (e >= h && e < h + p.valid && g < n) {
                __stcs(out + g, v[0][i][j]);
                __stcs(out + n + g, v[1][i][j]);
            }
        }
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
