// dbp_grad and dbp_set_steps: the reverse-mode gradient of the fused DBP and the update
// of the step table it is usually paired with (fitting step lengths / nonlinear
// strengths by gradient descent).
//
// dbp_grad launches, on the caller's stream:
//   1. dbp_adj_kernel: one CTA per overlap-save block; block input gradients and
//      per-warp partial sums of R_{s,i} = sum_k s_k S_{k,i} and dL/ddz_s to scratch;
//   2. gather_kernel: overlap-add of the block input gradients (Section III's
//      overlap-and-save transposed), each input sample summing its covering blocks in
//      block order;
//   3. reduce_kernel, reduce_segments_kernel: FP64 sums of the partials over all warp
//      rows (segment sums, then the sum of the segments), in a fixed order;
//   4. finalize_kernel: dL/dc_{s,i} = gamma_eff_s R_{s,i} (summed over steps when the
//      coefficients are shared), dL/dgamma_eff_s = sum_i c_{s,i} R_{s,i}, dL/ddz_s.
// Kernels 2-4 are programmatic dependent launches (each waits for its predecessor's end
// before reading its output).  No floating-point atomics: results are bitwise
// reproducible.
#include <math.h>
#include <stdlib.h>

#include "adj_kernel.cuh"

namespace dbp {

// Programmatic dependent launch: dbp_grad launches the kernels that follow the adjoint
// kernel with programmatic stream serialization, so each is scheduled while its
// predecessor drains; griddepcontrol.wait then blocks until the predecessor grid has
// completed and its memory is visible (a no-op in a kernel launched the ordinary way).
__device__ __forceinline__ void wait_for_predecessor() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... Params, typename... Args>
static cudaError_t launch_dependent(void (*kernel)(Params...), dim3 grid, dim3 block, cudaStream_t st,
                                    Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__global__ void gather_kernel(const float4 *__restrict__ gblk, float2 *__restrict__ gin, long long n, int nb, int V,
                              int half, int N, int boundary, int n_wave) {
    wait_for_predecessor();
    allow_dependents();
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n_wave) return;
    const long long w = idx / n, j = idx - w * n;
    const float4 *gw = gblk + (size_t)w * nb * N;
    float sx = 0.f, sy = 0.f, sz = 0.f, sw = 0.f;
    if (n >= N) {
        const int m0 = boundary == DBP_PERIODIC ? -1 : 0, m1 = boundary == DBP_PERIODIC ? 1 : 0;
        for (int m = m0; m <= m1; ++m) {
            const long long jp = j + m * n;                 // position in unwrapped block coordinates
            long long blo = jp + half - N + 1;              // st_b <= jp < st_b + N, st_b = b V - half
            blo = blo <= 0 ? 0 : (blo + V - 1) / V;
            long long bhi = jp + half < 0 ? -1 : (jp + half) / V;
            if (bhi > nb - 1) bhi = nb - 1;
            for (long long b = blo; b <= bhi; ++b) {
                const long long e = jp - (b * V - half);
                if (e < 0 || e >= N) continue;
                const float4 g = gw[(size_t)b * N + e];
                sx += g.x; sy += g.y; sz += g.z; sw += g.w;
            }
        }
    } else {
        for (int b = 0; b < nb; ++b) {
            const long long st = (long long)b * V - half;
            if (boundary == DBP_PERIODIC) {
                long long e = (j - st) % n;
                if (e < 0) e += n;
                for (; e < N; e += n) {
                    const float4 g = gw[(size_t)b * N + e];
                    sx += g.x; sy += g.y; sz += g.z; sw += g.w;
                }
            } else {
                const long long e = j - st;
                if (e >= 0 && e < N) {
                    const float4 g = gw[(size_t)b * N + e];
                    sx += g.x; sy += g.y; sz += g.z; sw += g.w;
                }
            }
        }
    }
    float2 *gp = gin + (size_t)w * 2 * n;
    gp[j] = make_float2(sx, sy);
    gp[n + j] = make_float2(sz, sw);
}

// gather_kernel for waveforms short enough for 32-bit positions (n + nb V + N < 2^30):
// one waveform per grid row, one division per unwrapped position, the periodic copies
// (the blocks at the waveform ends wrap around) only where they reach.  Sums the covering
// blocks in increasing block order, as gather_kernel does.
__global__ void gather32_kernel(const float4 *__restrict__ gblk, float2 *__restrict__ gin, int n, int nb, int V,
                                int half, int N, int boundary) {
    wait_for_predecessor();
    allow_dependents();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int w = blockIdx.y;
    const float4 *gw = gblk + (size_t)w * nb * N;
    float sx = 0.f, sy = 0.f, sz = 0.f, sw = 0.f;
    const int end = (nb - 1) * V - half + N;            // unwrapped end of the last window
    const bool per = boundary == DBP_PERIODIC;
    // m = +1, 0, -1 in order of increasing block index: jp = j - n (first blocks), j, j + n (last blocks)
#pragma unroll
    for (int m = -1; m <= 1; ++m) {
        if (m != 0 && !per) continue;
        const int jp = j + m * n;
        if (jp < -half || jp >= end) continue;
        int bhi = (jp + half) / V;                       // last block whose window starts at or before jp
        if (bhi > nb - 1) bhi = nb - 1;
        int blo = bhi;
        while (blo > 0 && (blo - 1) * V - half + N > jp) --blo;
        for (int b = blo; b <= bhi; ++b) {
            const int e = jp - (b * V - half);
            const float4 g = gw[(size_t)b * N + e];
            sx += g.x; sy += g.y; sz += g.z; sw += g.w;
        }
    }
    float2 *gp = gin + (size_t)w * 2 * n;
    gp[j] = make_float2(sx, sy);
    gp[n + j] = make_float2(sz, sw);
}

// Two-stage FP64 sum over the rows of partial sums (one row per warp of each block):
// seg_sum[q * segs + g] = sum of part[b * stride + q] over the rows b of contiguous
// segment g, then out[q] = sum of the segment sums in segment order.  The grid and the
// order of every addition depend only on (rows, stride, segs), so the result is bitwise
// reproducible.
__global__ void reduce_kernel(const float *__restrict__ part, long long rows, int stride, int segs,
                              double *__restrict__ seg_sum) {
    wait_for_predecessor();
    allow_dependents();
    __shared__ double sm[256];
    const int q = blockIdx.x, g = blockIdx.y;
    const long long per = (rows + segs - 1) / segs;
    const long long b0 = (long long)g * per;
    const long long b1 = b0 + per < rows ? b0 + per : rows;
    double acc = 0.0;
    for (long long b = b0 + threadIdx.x; b < b1; b += blockDim.x) acc += (double)part[(size_t)b * stride + q];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) seg_sum[(size_t)q * segs + g] = sm[0];
}

__global__ void reduce_segments_kernel(const double *__restrict__ seg_sum, int stride, int segs, double *out) {
    wait_for_predecessor();
    allow_dependents();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= stride) return;
    double acc = 0.0;
    for (int g = 0; g < segs; ++g) acc += seg_sum[(size_t)q * segs + g];
    out[q] = acc;
}

__global__ void finalize_kernel(const double *sums, const float *craw, const double *geff, int ns, int nt, int nr,
                                int per_step, float *d_coeffs, float *d_gamma, float *d_dz) {
    wait_for_predecessor();
    allow_dependents();
    const int t = threadIdx.x;
    const double *R = sums, *DZ = sums + (size_t)ns * nr;
    for (int q = t; q < ns * (nt + 1); q += blockDim.x) {
        const int s = q / (nt + 1), i = q % (nt + 1);
        if (d_coeffs && per_step) d_coeffs[q] = (float)(geff[s] * R[s * nr + i]);
    }
    if (d_coeffs && !per_step)
        for (int i = t; i <= nt; i += blockDim.x) {
            double acc = 0.0;
            for (int s = 0; s < ns; ++s) acc += geff[s] * R[s * nr + i];
            d_coeffs[i] = (float)acc;
        }
    for (int s = t; s < ns; s += blockDim.x) {
        if (d_gamma) {
            double acc = 0.0;
            for (int i = 0; i <= nt; ++i) acc += (double)craw[s * (nt + 1) + i] * R[s * nr + i];
            d_gamma[s] = (float)acc;
        }
        if (d_dz) d_dz[s] = (float)DZ[s];
    }
}

static int launch_adj(const PlanImpl &P, const AdjParams &q, int n_wave, cudaStream_t st) {
    const bool essfm = P.method == DBP_ESSFM;
    switch (P.info.fft_size) {
        case 512: return launch_adj_512(q, n_wave, essfm, st);
        case 1024: return launch_adj_1024(q, n_wave, essfm, st);
        case 2048: return launch_adj_2048(q, n_wave, essfm, st);
        case 4096: return launch_adj_4096(q, n_wave, essfm, st);
        case 8192: return launch_adj_8192(q, n_wave, essfm, st);
        default: return DBP_ERR_INFEASIBLE;
    }
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace dbp

using namespace dbp;

extern "C" int dbp_grad(dbp_plan_t *plan, const void *in, const void *grad_out, void *grad_in, float *d_coeffs,
                        float *d_gamma_eff, float *d_step_len, dbp_stream_t stream) {
    if (!plan || !in || !grad_out) return DBP_ERR_ARG;
    PlanImpl &P = plan->impl;
    if (P.precision != DBP_FP32 || P.scheme != DBP_SCHEME_FUSED || P.signal.n_pols == 1)
        return DBP_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = P.info.fft_size, ns = P.info.n_steps, nt = P.info.n_taps;
    const int nw = P.signal.n_waveforms;
    const long long blocks = (long long)P.info.n_blocks * nw;
    const int nr = 1 + 8 * P.n_tapblk;
    const int stride = ns * nr + ns;
    const size_t wbytes = (size_t)2 * P.signal.n_samples * sizeof(float2) * nw;
    if (grad_in && (overlaps(grad_in, in, wbytes) || overlaps(grad_in, grad_out, wbytes))) return DBP_ERR_ALIAS;

    // scratch: gblk, uscr, yscr, checkpoints, partials, sums
    const size_t fld = (size_t)blocks * N * sizeof(float4);
    const size_t o_g = 0, o_u = al256(fld), o_y = o_u + al256(fld);
    const size_t o_c = o_y + al256(fld);
    const size_t o_p = o_c + al256(fld * (ns > 1 ? ns - 1 : 1));
    const long long rows = blocks * (N / 512);   // one row of partial sums per warp of each block
    const size_t o_s = o_p + al256(sizeof(float) * (size_t)rows * stride);
    // segments of the first reduction stage: about 1024 rows each, at most 64
    const int segs = (int)(rows / 1024 + 1 < 64 ? rows / 1024 + 1 : 64);
    const size_t o_seg = o_s + al256(sizeof(double) * stride);
    const size_t total = o_seg + al256(sizeof(double) * (size_t)stride * segs);
    if (P.adj_bytes < total) {
        if (P.d_adj) cudaFree(P.d_adj);
        P.d_adj = nullptr;
        P.adj_bytes = 0;
        if (dev_alloc(&P.d_adj, total)) return DBP_ERR_ALLOC;
        P.adj_bytes = total;
    }
    unsigned char *sc = (unsigned char *)P.d_adj;
    AdjParams q;
    fill_fwd_params(P, q.f);
    q.f.in = (const float2 *)in;
    q.f.out = nullptr;
    q.gout = (const float2 *)grad_out;
    q.gblk = (float4 *)(sc + o_g);
    q.uscr = (float4 *)(sc + o_u);
    q.yscr = (float4 *)(sc + o_y);
    q.ckpt = (float4 *)(sc + o_c);
    q.part = (float *)(sc + o_p);
    q.nr = nr;
    const double fsn = P.signal.sample_rate_hz / N;
    q.cphi = (float)(2.0 * M_PI * M_PI * P.info.beta2_s2_per_m * fsn * fsn);
    int rc = launch_adj(P, q, nw, st);
    if (rc) return rc;
    if (grad_in) {
        const long long n = P.signal.n_samples;
        const long long span = n + (long long)P.info.n_blocks * P.info.valid + N;
        if (n >= N && span < (1LL << 30) && nw <= 65535) {
            if (launch_dependent(gather32_kernel, dim3((unsigned)((n + 255) / 256), (unsigned)nw), dim3(256), st,
                                 (const float4 *)q.gblk, (float2 *)grad_in, (int)n, (int)P.info.n_blocks,
                                 (int)P.info.valid, (int)(P.info.overlap / 2), N, (int)P.signal.boundary) != cudaSuccess)
                return DBP_ERR_CUDA;
        } else {
            const long long total_s = n * nw;
            if (launch_dependent(gather_kernel, dim3((unsigned)((total_s + 255) / 256)), dim3(256), st,
                                 (const float4 *)q.gblk, (float2 *)grad_in, (long long)n, (int)P.info.n_blocks,
                                 (int)P.info.valid, (int)(P.info.overlap / 2), N, (int)P.signal.boundary,
                                 nw) != cudaSuccess)
                return DBP_ERR_CUDA;
        }
    }
    double *sums = (double *)(sc + o_s);
    double *seg_sum = (double *)(sc + o_seg);
    if (launch_dependent(reduce_kernel, dim3((unsigned)stride, (unsigned)segs), dim3(256), st, (const float *)q.part,
                         rows, stride, segs, seg_sum) != cudaSuccess ||
        launch_dependent(reduce_segments_kernel, dim3((unsigned)((stride + 127) / 128)), dim3(128), st,
                         (const double *)seg_sum, stride, segs, sums) != cudaSuccess ||
        launch_dependent(finalize_kernel, dim3(1), dim3(256), st, (const double *)sums, (const float *)P.d_craw,
                         (const double *)P.d_geff, ns, nt, nr, (int)P.coeffs_per_step, d_coeffs, d_gamma_eff,
                         d_step_len) != cudaSuccess)
        return DBP_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

extern "C" int dbp_set_steps(dbp_plan_t *plan, const double *step_len_m, const double *gamma_eff) {
    if (!plan) return DBP_ERR_ARG;
    PlanImpl &P = plan->impl;
    const int ns = P.info.n_steps;
    if (step_len_m)
        for (int s = 0; s < ns; ++s)
            if (!(step_len_m[s] >= 0) || !isfinite(step_len_m[s])) return DBP_ERR_ARG;
    if (gamma_eff)
        for (int s = 0; s < ns; ++s)
            if (!isfinite(gamma_eff[s])) return DBP_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return DBP_ERR_CUDA;
    if (step_len_m) {
        for (int s = 0; s < ns; ++s) P.step_dz[s] = step_len_m[s];
        const int rc = build_h_tables(P);
        if (rc) return rc;
    }
    if (gamma_eff) {
        for (int s = 0; s < ns; ++s) P.step_geff[s] = gamma_eff[s];
    }
    return upload_taps(P, P.coeffs);
}
