// Fused overlap-save DBP kernel: persistent CTAs, each taking one block of N vector
// samples at a time through all N_s steps in shared memory / registers, FP32.
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
// window [b V - O/2, b V - O/2 + N) and writes its central V = N - O samples.  In the
// ESSFM kernels the next block's window is prefetched into L2 by bulk prefetches and
// the outputs leave through the block buffer by bulk shared-to-global copies.  At
// N = 8192 the inter-pass twiddles of each thread sit in tensor memory (tcgen05).
#pragma once
#include "block_fft.cuh"

namespace dbp {

// Input window of overlap-save block (waveform w, block b) into registers (global
// loads only, no shared memory).  SINGLE: a one-polarization waveform [n]; the two
// polarization lanes carry blocks b and b + 1.
template <int N, bool SINGLE = false, class BK = Blk<N>>
__device__ __forceinline__ void load_block(const FwdParams &p, const BK &blk, int w, int b,
                                           typename Blk<N>::Regs &v) {
    const long long n = p.n;
    const float2 *__restrict__ in = p.in + (size_t)w * (SINGLE ? 1 : 2) * n;
    blk.template load_window<SINGLE>(v, in, n, (long long)b * p.valid - p.half_overlap, p.boundary, p.valid);
}

// All steps and the overlap-save output of block (w, b), loaded into v, with the
// twiddle tables in shared memory, p.H (step 0) prefetch committed and a barrier since
// the previous block's last shared-memory access (and, with bulk stores, since its
// output copy finished reading the staging buffer).  SINGLE: each lane has its own
// intensity P = |y|^2, filter and phase.
template <int N, bool ESSFM, bool SINGLE = false, bool FAST = false, bool TM = false, class BK = Blk<N>>
__device__ __forceinline__ void compute_block(const FwdParams &p, BK &blk, int w, int b,
                                              typename Blk<N>::Regs &v) {
    using B = Blk<N>;
    const long long n = p.n;
    float2 *__restrict__ out = p.out + (size_t)w * (SINGLE ? 1 : 2) * n;

    MidMulH<N> mid{blk.sH};
    for (int s = 0; s < p.n_steps; ++s) {
        if (ESSFM && s > 0) blk.sync();   // previous step's theta and tap reads are done
        if (ESSFM) blk.stage_taps(p.taps + p.taps_stride * s, p.taps_stride);
        blk.template pass1_fwd<TM>(v);
        blk.sync();
        blk.template pass2<false, TM && ESSFM>();
        cp_async_wait_all();
        // Passes 2 -> 3 -> 2' stay inside a warp: warp w's pass-2 columns write, and its
        // pass-3 threads read, positions [512 w, 512 w + 512), and warp w copied the H_s
        // entries of those positions itself.  A warp barrier orders them.
        __syncwarp();
        blk.pass3(mid);
        __syncwarp();
        if (p.h_stride != 0 && s + 1 < p.n_steps) blk.prefetch_h(p.H + p.h_stride * (s + 1));
        blk.template pass2<true, TM && ESSFM>();
        blk.sync();
        blk.template pass1_inv<TM>(v);
        if (p.linear_only) continue;   // FFE: dispersion compensation only

        // ---- nonlinear sub-step
        const float *__restrict__ a = p.taps + p.taps_stride * s;
        if constexpr (ESSFM && !SINGLE) {
            blk.sync();   // block buffer free: P and theta reuse it
            blk.essfm_theta_fwd(v, blk.sa, p.n_tapblk);
            const float *sT = blk.tharr();
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int j = 0; j < B::N2; ++j) {
                    const float2 e = expj<FAST>(sT[pphys(blk.pos1(i, j))]);
                    v[0][i][j] = cmul(v[0][i][j], e);
                    v[1][i][j] = cmul(v[1][i][j], e);
                }
        } else if constexpr (ESSFM) {
            const float *sT = blk.tharr();
            blk.sync();   // block buffer free
            blk.template essfm_theta_fwd<0>(v, blk.sa, p.n_tapblk);
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int j = 0; j < B::N2; ++j) v[0][i][j] = cmul(v[0][i][j], expj<FAST>(sT[pphys(blk.pos1(i, j))]));
            // lane 1: its P may overwrite lane 0's (the filter is done); the barrier inside
            // essfm_theta orders the lane-0 theta reads before lane 1's theta is written
            blk.template essfm_theta_fwd<1>(v, blk.sa, p.n_tapblk);
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int j = 0; j < B::N2; ++j) v[1][i][j] = cmul(v[1][i][j], expj<FAST>(sT[pphys(blk.pos1(i, j))]));
        } else if constexpr (SINGLE) {
            const float a0 = __ldg(a);
#pragma unroll
            for (int l = 0; l < 2; ++l)
#pragma unroll
                for (int i = 0; i < B::C1; ++i)
#pragma unroll
                    for (int j = 0; j < B::N2; ++j) {
                        const float2 y = v[l][i][j];
                        v[l][i][j] = cmul(y, expj<FAST>(a0 * fmaf(y.x, y.x, y.y * y.y)));
                    }
        } else {
            const float a0 = __ldg(a);
#pragma unroll
            for (int i = 0; i < B::C1; ++i)
#pragma unroll
                for (int j = 0; j < B::N2; ++j) {
                    const float2 y0 = v[0][i][j], y1 = v[1][i][j];
                    const float2 e = expj<FAST>(a0 * joint_intensity(y0, y1));
                    v[0][i][j] = cmul(y0, e);
                    v[1][i][j] = cmul(y1, e);
                }
        }
    }

    // ---- overlap-and-save: keep the central V samples
    const int h = p.half_overlap;
    const long long obase = (long long)b * p.valid - h;
    if (ESSFM && p.bulk_store) {
        // stage [2][V] (polarizations, or the two blocks of a one-polarization pair) in
        // the block buffer, then one thread copies each half to its place in `out`
        const int V = p.valid;
        float2 *stage = reinterpret_cast<float2 *>(blk.xs);
        blk.sync();   // all reads of P / theta / the block buffer are done
#pragma unroll
        for (int i = 0; i < B::C1; ++i)
#pragma unroll
            for (int j = 0; j < B::N2; ++j) {
                const int e = blk.pos1(i, j);
                if (e < h || e >= h + V) continue;
                stage[e - h] = v[0][i][j];
                stage[V + e - h] = v[1][i][j];
            }
        fence_proxy_async_smem();
        blk.sync();
        if (blk.t == 0) {
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                const long long g0 = (long long)(b + (SINGLE ? l : 0)) * V;
                const long long cnt = n - g0 < V ? n - g0 : V;
                if (cnt > 0)
                    bulk_store(out + (SINGLE ? 0 : l * n) + g0, stage + l * V, (unsigned)(cnt * sizeof(float2)));
            }
            bulk_commit();
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < B::C1; ++i)
#pragma unroll
        for (int j = 0; j < B::N2; ++j) {
            const int e = blk.pos1(i, j);
            if (e < h || e >= h + p.valid) continue;
            const long long g = obase + e;
            if constexpr (SINGLE) {
                if (g < n) __stcs(out + g, v[0][i][j]);
                if (g + p.valid < n) __stcs(out + g + p.valid, v[1][i][j]);
            } else if (g < n) {
                __stcs(out + g, v[0][i][j]);
                __stcs(out + n + g, v[1][i][j]);
            }
        }
}

// One block from load to output (batched launches): load, then compute.  FAST: the
// hardware exponential, as dbp_run takes it for ESSFM plans of at most two steps.
template <int N, bool ESSFM, bool SINGLE = false, bool FAST = false, class BK = Blk<N>>
__device__ __forceinline__ void process_block(const FwdParams &p, BK &blk, int w, int b) {
    typename Blk<N>::Regs v;
    load_block<N, SINGLE>(p, blk, w, b, v);
    if (ESSFM && p.bulk_store) {   // the previous block's output copy must have read shared memory
        if (blk.t == 0) bulk_wait_read_all();
        blk.sync();
    }
    compute_block<N, ESSFM, SINGLE, FAST, false, BK>(p, blk, w, b, v);
}

// Persistent over blocks: CTA c processes blocks c, c + gridDim.x, ...  The twiddle
// tables (and H when all steps share it) are loaded into shared memory once per CTA, and
// at N = 8192 each thread's inter-pass twiddles once into tensor memory; the input
// window of the block this CTA runs next is prefetched into L2 while the current one is
// processed.  One barrier per block boundary: the steps' own barriers already separate
// the last reads of H and of the taps from the next block's writes.  SINGLE: an item is
// a pair of consecutive blocks of a one-polarization waveform.
template <int N, bool ESSFM, bool SINGLE = false, bool FAST = false>
__global__ void __launch_bounds__(Geo<N>::T, Geo<N>::MINB) dbp_fwd_kernel(const FwdParams p, int total) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // N = 8192 (one CTA per SM, one pass-1 and one pass-2 column per thread): each
    // thread's inter-pass twiddles live in TMEM, 64 columns of its lane; 16 warps = 4 per
    // lane quarter, so 4 x 64 = 256 columns.  Pass 1 reads them in every kernel, pass 2 in
    // the ESSFM kernels (in the SSFM/FFE kernels the pass-2 table reads measured faster:
    // their register allocation spills more with the TMEM reads).
    constexpr bool TM = (N == 8192);
    constexpr uint32_t TM_COLS = 4 * Blk<N>::TW_COLS;
    __shared__ uint32_t s_tmem;
    Blk<N> blk(smem_raw, threadIdx.x);
    blk.load_tables(p.twA, p.twB, p.tw2);
    if constexpr (TM) {
        static_assert(Geo<N>::T == 512, "16 warps: 4 per TMEM lane quarter");
        if (threadIdx.x < 32) {
            tmem_alloc(&s_tmem, TM_COLS);
            tmem_relinquish();
        }
        tmem_fence_before_sync();
        __syncthreads();   // tables and the TMEM address visible
        tmem_fence_after_sync();
        const uint32_t warp = threadIdx.x >> 5;
        blk.twt = s_tmem + (((warp & 3u) * 32u) << 16) + Blk<N>::TW_COLS * (warp >> 2);
        blk.twiddles_to_tmem();
    }
    const int per_wave = SINGLE ? (p.n_blocks + 1) / 2 : p.n_blocks;
    const int bstep = SINGLE ? 2 : 1;
    const long long wstride = (SINGLE ? 1 : 2) * p.n;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int w = item / per_wave;
        const int b = (item - w * per_wave) * bstep;
        if (item == (int)blockIdx.x || p.h_stride != 0) blk.prefetch_h(p.H);
        const int next = item + (int)gridDim.x;
        if (p.prefetch_ahead != 0 && next < total) {
            const int w2 = next / per_wave, b2 = (next - w2 * per_wave) * bstep;
            blk.template prefetch_window_l2<SINGLE, ESSFM>(p.in + (size_t)w2 * wstride, p.n,
                                                    (long long)b2 * p.valid - p.half_overlap, p.valid);
        }
        // The loads go out before the barrier: they touch registers only.  The barrier then
        // orders every shared-memory access of the previous block (the last ones: theta reads
        // or the output staging, whose bulk copy thread 0 waits for) before this block's.
        typename Blk<N>::Regs v;
        load_block<N, SINGLE>(p, blk, w, b, v);
        if (ESSFM && p.bulk_store && threadIdx.x == 0) bulk_wait_read_all();
        __syncthreads();   // tables visible; previous block's shared-memory use finished
        compute_block<N, ESSFM, SINGLE, FAST, TM>(p, blk, w, b, v);
    }
    if (ESSFM && p.bulk_store && threadIdx.x == 0) bulk_wait_all();
    if constexpr (TM) {   // every tcgen05.ld has been waited for; free the columns
        tmem_fence_before_sync();
        __syncthreads();
        tmem_fence_after_sync();
        if (threadIdx.x < 32) tmem_dealloc(s_tmem, TM_COLS);
    }
}

// SMs x resident CTAs per SM for a kernel configuration (at least 1).
template <typename K>
inline int resident_ctas(K kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess)
        return 1;
    const int r = sms * per_sm;
    return r > 0 ? r : 1;
}

template <int N, bool ESSFM, bool SINGLE, bool FAST = false>
int launch_fwd_variant(const FwdParams &p, long long grid, cudaStream_t st) {
    using G = Geo<N>;
    static unsigned long long done = 0;
    static int resident[64];   // CTAs resident per GPU (SMs x CTAs per SM), per device
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DBP_ERR_CUDA;
    if (!set_smem_once(dbp_fwd_kernel<N, ESSFM, SINGLE, FAST>, G::SMEM, done)) return DBP_ERR_CUDA;
    if (!resident[dev]) resident[dev] = resident_ctas(dbp_fwd_kernel<N, ESSFM, SINGLE, FAST>, G::T, G::SMEM);
    const int ctas = (int)(grid < resident[dev] ? grid : resident[dev]);
    dbp_fwd_kernel<N, ESSFM, SINGLE, FAST><<<(unsigned)ctas, G::T, G::SMEM, st>>>(p, (int)grid);
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

// ESSFM plans of at most two steps take the hardware exponential (expj<true>).
template <int N>
int launch_fwd_n(const FwdParams &p, int n_wave, bool essfm, cudaStream_t st) {
    const long long per_wave = p.single_pol ? (p.n_blocks + 1) / 2 : p.n_blocks;
    const long long grid = per_wave * n_wave;
    if (grid <= 0 || grid > 0x7fffffffLL) return DBP_ERR_ARG;
    const bool fast = essfm && p.fast_exp;
    if (p.single_pol) {
        if (fast) return launch_fwd_variant<N, true, true, true>(p, grid, st);
        return essfm ? launch_fwd_variant<N, true, true>(p, grid, st) : launch_fwd_variant<N, false, true>(p, grid, st);
    }
    if (fast) return launch_fwd_variant<N, true, false, true>(p, grid, st);
    return essfm ? launch_fwd_variant<N, true, false>(p, grid, st) : launch_fwd_variant<N, false, false>(p, grid, st);
}

}  // namespace dbp


