// Coefficient-independent quantities of the Section IV least-squares fit of a
// single-step ESSFM (minimum MSE between the ESSFM output and a target waveform).
//
// With one step the linear sub-step output y of a block does not depend on c, and the
// ESSFM output is z_k = y_k exp(j theta_k), theta_k = gamma_eff sum_i c_i S_{k,i},
// S_{k,0} = P_k, S_{k,i} = P_{k-i} + P_{k+i} (P the joint intensity, indices circular
// inside the block, Eq. 3).  dbp_fitprep_kernel runs the linear sub-step of every
// overlap-save block (the same FFT, x H, IFFT as the forward kernel) and stores
//   Pb[item][e] = P_e                                for all N positions e of the block,
//   q[item][k]  = sum_p conj(y_{h+k,p}) t_{g,p}      for the V valid positions,
// g = b V + k the output position (q = 0 where g is outside the training range).
#pragma once
#include "block_fft.cuh"

namespace dbp {

template <int N>
__global__ void __launch_bounds__(Geo<N>::T, Geo<N>::MINB)
    dbp_fitprep_kernel(const FwdParams p, const float2 *__restrict__ target, long long limit, float *__restrict__ Pb,
                       float2 *__restrict__ q, int total) {
    using B = Blk<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    B blk(smem_raw, threadIdx.x);
    blk.load_tables(p.twA, p.twB, p.tw2);
    blk.prefetch_h(p.H);
    const long long n = p.n;
    const int h = p.half_overlap, V = p.valid;
    MidMulH<N> mid{blk.sH};
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int w = item / p.n_blocks;
        const int b = item - w * p.n_blocks;
        __syncthreads();   // tables visible; previous block's shared-memory use finished
        typename B::Regs v;
        blk.load_window(v, p.in + (size_t)w * 2 * n, n, (long long)b * V - h, p.boundary);
        blk.pass1_fwd(v);
        __syncthreads();
        blk.template pass2<false>();
        cp_async_wait_all();
        __syncthreads();
        blk.pass3(mid);
        __syncthreads();
        blk.template pass2<true>();
        __syncthreads();
        blk.pass1_inv(v);

        const float2 *tw = target + (size_t)w * 2 * n;
        float *pb = Pb + (size_t)item * N;
        float2 *qb = q + (size_t)item * V;
#pragma unroll
        for (int i = 0; i < B::C1; ++i)
#pragma unroll
            for (int j = 0; j < B::N2; ++j) {
                const int e = blk.pos1(i, j);
                const float2 y0 = v[0][i][j], y1 = v[1][i][j];
                pb[e] = joint_intensity(y0, y1);
                if (e >= h && e < h + V) {
                    const long long g = (long long)b * V + (e - h);
                    float2 r = make_float2(0.f, 0.f);
                    if (g < limit) {
                        const float2 t0 = __ldg(tw + g), t1 = __ldg(tw + n + g);
                        r = cadd(cmul(make_float2(y0.x, -y0.y), t0), cmul(make_float2(y1.x, -y1.y), t1));
                    }
                    qb[e - h] = r;
                }
            }
    }
}

template <int N>
int launch_fitprep_n(const FwdParams &p, int n_wave, const float2 *target, long long limit, float *Pb, float2 *q,
                     cudaStream_t st) {
    using G = Geo<N>;
    static unsigned long long done = 0;
    const long long total = (long long)p.n_blocks * n_wave;
    if (total <= 0 || total > 0x7fffffffLL) return DBP_ERR_ARG;
    if (!set_smem_once(dbp_fitprep_kernel<N>, G::SMEM, done)) return DBP_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dbp_fitprep_kernel<N>, G::T, G::SMEM))
        return DBP_ERR_CUDA;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > total) grid = total;
    dbp_fitprep_kernel<N><<<(int)grid, G::T, G::SMEM, st>>>(p, target, limit, Pb, q, (int)total);
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

}  // namespace dbp
