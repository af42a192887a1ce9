// dbp_fit_coeffs: the Section IV least-squares fit of a single-step ESSFM's
// coefficients c_0..c_Nc against a target waveform, by Gauss-Newton on the complex
// residual t - z.
//
// With a_i = gamma_eff c_i, z_k = y_k exp(j theta_k), theta_k = sum_i a_i S_{k,i}, the
// Jacobian of the residual is -j S_{k,i} z_{k,p}; stacked as real and imaginary parts,
//   J^T J  = sum_k P_k S_{k,i} S_{k,j}                      (|z_{k,p}| = |y_{k,p}|)
//   J^T r  = sum_k S_{k,i} Im(exp(-j theta_k) q_k),  q_k = sum_p conj(y_{k,p}) t_{k,p}
//   |r|^2  = sum_k (|t_k|^2 + P_k) - 2 sum_k Re(exp(-j theta_k) q_k).
// J^T J does not depend on c, so it is accumulated once and factored once (Cholesky,
// FP64, on the host: at most 65 x 65); each iteration is one pass over the training
// samples for J^T r.  Device passes:
//   1. dbp_fitprep_kernel: linear sub-step per block -> P (whole block) and q (valid);
//   2. fit_gram_kernel: per-block partial sums of P S_i S_j and of |t|^2 + P;
//   3. per iteration, fit_grad_kernel: per-block partial sums of J^T r and Re(e^{-j theta} q);
//   4. fit_reduce_kernel: FP64 sums over blocks in a fixed order.
// Products and sums of the regressors are formed in FP64 from the FP32 intensities, so
// J^T J is the Gram matrix of the FP32 regressors to FP64 rounding.  No floating-point
// atomics: results are bitwise reproducible.
#include <math.h>

#include <vector>

#include "fit_kernel.cuh"

namespace dbp {

// S_{k,i} (i < kc), or 1 for the common-phase regressor i == kc (kc < 0: none)
__device__ __forceinline__ double regressor(const float *sP, int e, int i, int mask, int kc) {
    if (i == kc) return 1.0;
    return i == 0 ? (double)sP[e] : (double)sP[(e - i) & mask] + (double)sP[(e + i) & mask];
}

// Training positions of block b: output samples b V + k, 0 <= k < kv.
__device__ __forceinline__ int training_count(int b, int V, long long limit) {
    const long long r = limit - (long long)b * V;
    return r <= 0 ? 0 : (r >= V ? V : (int)r);
}

// part[item][pair] (pairs i <= j of K regressors, row-major upper triangle) =
// sum_k P_k S_{k,i} S_{k,j}; part[item][npair] = sum_k (P_k + |t_k,1|^2 + |t_k,2|^2).
// Regressor kc (if >= 0) is the constant 1 of a common phase.
__global__ void fit_gram_kernel(const float *__restrict__ Pb, const float2 *__restrict__ target, long long n, int N,
                                int V, int half, int n_blocks, long long limit, int K, int kc,
                                double *__restrict__ part) {
    extern __shared__ __align__(16) double dsm[];
    double *red = dsm;
    float *sP = reinterpret_cast<float *>(dsm + blockDim.x);
    const int item = blockIdx.x, tid = threadIdx.x;
    const int w = item / n_blocks, b = item - w * n_blocks;
    for (int e = tid; e < N; e += blockDim.x) sP[e] = Pb[(size_t)item * N + e];
    __syncthreads();
    const int kv = training_count(b, V, limit), mask = N - 1;
    const int npair = K * (K + 1) / 2, stride = npair + 1;
    for (int pair = tid; pair < npair; pair += blockDim.x) {
        int i = 0, r = pair;
        while (r >= K - i) {
            r -= K - i;
            ++i;
        }
        const int j = i + r;
        double acc = 0.0;
        for (int k = 0; k < kv; ++k) {
            const int e = half + k;
            acc += (double)sP[e] * (regressor(sP, e, i, mask, kc) * regressor(sP, e, j, mask, kc));
        }
        part[(size_t)item * stride + pair] = acc;
    }
    const float2 *tw = target + (size_t)w * 2 * n;
    double en = 0.0;
    for (int k = tid; k < kv; k += blockDim.x) {
        const long long g = (long long)b * V + k;
        const float2 t0 = tw[g], t1 = tw[n + g];
        en += (double)sP[half + k] + (double)t0.x * t0.x + (double)t0.y * t0.y + (double)t1.x * t1.x +
              (double)t1.y * t1.y;
    }
    red[tid] = en;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    if (tid == 0) part[(size_t)item * stride + npair] = red[0];
}

// part[item][i] = sum_k S_{k,i} Im(e^{-j theta_k} q_k), part[item][K] = sum_k Re(e^{-j theta_k} q_k),
// theta_k = sum_i a_i S_{k,i} (S_{k,kc} = 1 if kc >= 0).
__global__ void fit_grad_kernel(const float *__restrict__ Pb, const float2 *__restrict__ q, int N, int V, int half,
                                int n_blocks, long long limit, int K, int kc, const double *__restrict__ a,
                                double *__restrict__ part) {
    extern __shared__ __align__(16) double dsm[];
    double *red = dsm;                    // [blockDim.x]
    double *sa = red + blockDim.x;        // [K]
    double *sw = sa + K;                  // [V]
    float *sP = reinterpret_cast<float *>(sw + V);
    const int item = blockIdx.x, tid = threadIdx.x;
    const int b = item % n_blocks;
    for (int e = tid; e < N; e += blockDim.x) sP[e] = Pb[(size_t)item * N + e];
    for (int i = tid; i < K; i += blockDim.x) sa[i] = a[i];
    __syncthreads();
    const int kv = training_count(b, V, limit), mask = N - 1;
    double racc = 0.0;
    for (int k = tid; k < kv; k += blockDim.x) {
        const int e = half + k;
        double th = 0.0;
        for (int i = 0; i < K; ++i) th += sa[i] * regressor(sP, e, i, mask, kc);
        double s, c;
        sincos(th, &s, &c);
        const float2 qk = q[(size_t)item * V + k];
        sw[k] = c * qk.y - s * qk.x;
        racc += c * qk.x + s * qk.y;
    }
    red[tid] = racc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (tid < o) red[tid] += red[tid + o];
        __syncthreads();
    }
    const int warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
    for (int i = warp; i < K; i += nwarps) {
        double acc = 0.0;
        for (int k = lane; k < kv; k += 32) acc += regressor(sP, half + k, i, mask, kc) * sw[k];
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) part[(size_t)item * (K + 1) + i] = acc;
    }
    if (tid == 0) part[(size_t)item * (K + 1) + K] = red[0];
}

// out[c] = sum over items (fixed order) of part[item * stride + c].
__global__ void fit_reduce_kernel(const double *__restrict__ part, long long items, int stride, double *out) {
    __shared__ double sm[256];
    const int c = blockIdx.x;
    double acc = 0.0;
    for (long long it = threadIdx.x; it < items; it += blockDim.x) acc += part[(size_t)it * stride + c];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = sm[0];
}

static int launch_fitprep(int N, const FwdParams &p, int n_wave, const float2 *target, long long limit, float *Pb,
                          float2 *q, cudaStream_t st) {
    switch (N) {
        case 512: return launch_fitprep_n<512>(p, n_wave, target, limit, Pb, q, st);
        case 1024: return launch_fitprep_n<1024>(p, n_wave, target, limit, Pb, q, st);
        case 2048: return launch_fitprep_n<2048>(p, n_wave, target, limit, Pb, q, st);
        case 4096: return launch_fitprep_n<4096>(p, n_wave, target, limit, Pb, q, st);
        case 8192: return launch_fitprep_n<8192>(p, n_wave, target, limit, Pb, q, st);
        default: return DBP_ERR_INFEASIBLE;
    }
}

// Cholesky factor L (lower, row-major K x K) of the symmetric matrix g; false unless
// every pivot is positive and above 1e-14 of the largest diagonal entry.
static bool cholesky(const std::vector<double> &g, int K, std::vector<double> &L) {
    double dmax = 0.0;
    for (int i = 0; i < K; ++i) dmax = fmax(dmax, g[(size_t)i * K + i]);
    if (!(dmax > 0.0)) return false;
    L.assign((size_t)K * K, 0.0);
    for (int j = 0; j < K; ++j) {
        double d = g[(size_t)j * K + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * K + k] * L[(size_t)j * K + k];
        if (!(d > 1e-14 * dmax)) return false;
        const double ljj = sqrt(d);
        L[(size_t)j * K + j] = ljj;
        for (int i = j + 1; i < K; ++i) {
            double s = g[(size_t)i * K + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * K + k] * L[(size_t)j * K + k];
            L[(size_t)i * K + j] = s / ljj;
        }
    }
    return true;
}

// Solves L L^T x = r in place.
static void cholesky_solve(const std::vector<double> &L, int K, std::vector<double> &r) {
    for (int i = 0; i < K; ++i) {
        double s = r[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * K + k] * r[k];
        r[i] = s / L[(size_t)i * K + i];
    }
    for (int i = K - 1; i >= 0; --i) {
        double s = r[i];
        for (int k = i + 1; k < K; ++k) s -= L[(size_t)k * K + i] * r[k];
        r[i] = s / L[(size_t)i * K + i];
    }
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace dbp

using namespace dbp;

extern "C" int dbp_fit_coeffs(dbp_plan_t *plan, const void *x, const void *target, long long n_train, int max_iter,
                              double tol, double *coeffs, double *phase, double *loss, int *n_iter,
                              dbp_stream_t stream) {
    if (!plan || !x || !target || !coeffs || max_iter < 0 || !(tol >= 0.0)) return DBP_ERR_ARG;
    PlanImpl &P = plan->impl;
    if (P.method != DBP_ESSFM || P.info.n_steps != 1 || P.precision != DBP_FP32 ||
        P.scheme != DBP_SCHEME_FUSED || P.signal.n_pols == 1)
        return DBP_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = P.info.fft_size, V = P.info.valid, half = P.info.overlap / 2;
    const int KC = P.info.n_taps + 1;             // coefficients
    const int K = KC + (phase ? 1 : 0);           // parameters: coefficients, then the common phase
    const int kc = phase ? KC : -1;
    const int nw = P.signal.n_waveforms, nb = P.info.n_blocks;
    const long long n = P.signal.n_samples;
    const long long limit = (n_train <= 0 || n_train > n) ? n : n_train;
    const long long items = (long long)nb * nw;
    if (items > 0x7fffffffLL) return DBP_ERR_ARG;
    const int npair = K * (K + 1) / 2;

    // scratch (shared with dbp_grad): P blocks, q, Gram partials and sums, gradient
    // partials and sums, a = gamma_eff c (and the phase)
    const size_t o_p = 0, o_q = o_p + al256(sizeof(float) * (size_t)items * N);
    const size_t o_gp = o_q + al256(sizeof(float2) * (size_t)items * V);
    const size_t o_gs = o_gp + al256(sizeof(double) * (size_t)items * (npair + 1));
    const size_t o_rp = o_gs + al256(sizeof(double) * (npair + 1));
    const size_t o_rs = o_rp + al256(sizeof(double) * (size_t)items * (K + 1));
    const size_t o_a = o_rs + al256(sizeof(double) * (K + 1));
    const size_t total = o_a + al256(sizeof(double) * K);
    if (P.adj_bytes < total) {
        if (P.d_adj) cudaFree(P.d_adj);
        P.d_adj = nullptr;
        P.adj_bytes = 0;
        if (dev_alloc(&P.d_adj, total)) return DBP_ERR_ALLOC;
        P.adj_bytes = total;
    }
    unsigned char *sc = (unsigned char *)P.d_adj;
    float *Pb = (float *)(sc + o_p);
    float2 *q = (float2 *)(sc + o_q);
    double *gpart = (double *)(sc + o_gp), *gsum = (double *)(sc + o_gs);
    double *rpart = (double *)(sc + o_rp), *rsum = (double *)(sc + o_rs), *d_a = (double *)(sc + o_a);

    FwdParams p;
    fill_fwd_params(P, p);
    p.in = (const float2 *)x;
    p.out = nullptr;
    int rc = launch_fitprep(N, p, nw, (const float2 *)target, limit, Pb, q, st);
    if (rc) return rc;

    const int threads = 256;
    const size_t gram_smem = sizeof(double) * threads + sizeof(float) * N;
    const size_t grad_smem = sizeof(double) * (threads + K + V) + sizeof(float) * N;
    if (cudaFuncSetAttribute(fit_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_smem) ||
        cudaFuncSetAttribute(fit_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem))
        return DBP_ERR_CUDA;
    fit_gram_kernel<<<(int)items, threads, gram_smem, st>>>(Pb, (const float2 *)target, n, N, V, half, nb, limit, K,
                                                             kc, gpart);
    fit_reduce_kernel<<<npair + 1, 256, 0, st>>>(gpart, items, npair + 1, gsum);
    std::vector<double> hg(npair + 1);
    if (cudaMemcpyAsync(hg.data(), gsum, sizeof(double) * (npair + 1), cudaMemcpyDeviceToHost, st) ||
        cudaStreamSynchronize(st))
        return DBP_ERR_CUDA;

    // theta = gamma_eff sum_i c_i S_i (+ phase): parameter i scales its regressor by s_i
    const double ge = P.step_geff[0];
    std::vector<double> sfac(K, ge);
    if (phase) sfac[KC] = 1.0;
    const double m = (double)limit * nw;   // training vector samples
    std::vector<double> G((size_t)K * K), L;
    for (int i = 0, pr = 0; i < K; ++i)
        for (int j = i; j < K; ++j, ++pr) G[(size_t)i * K + j] = G[(size_t)j * K + i] = sfac[i] * sfac[j] * hg[pr];
    const double energy = hg[npair];
    if (!cholesky(G, K, L)) return DBP_ERR_SINGULAR;

    std::vector<double> c(K), a(K), r(K + 1);
    for (int i = 0; i < KC; ++i) c[i] = coeffs[i];
    if (phase) c[KC] = *phase;
    int updates = 0;
    bool done = false;
    for (int it = 0;; ++it) {
        for (int i = 0; i < K; ++i) a[i] = sfac[i] * c[i];
        if (cudaMemcpyAsync(d_a, a.data(), sizeof(double) * K, cudaMemcpyHostToDevice, st)) return DBP_ERR_CUDA;
        fit_grad_kernel<<<(int)items, threads, grad_smem, st>>>(Pb, q, N, V, half, nb, limit, K, kc, d_a, rpart);
        fit_reduce_kernel<<<K + 1, 256, 0, st>>>(rpart, items, K + 1, rsum);
        if (cudaMemcpyAsync(r.data(), rsum, sizeof(double) * (K + 1), cudaMemcpyDeviceToHost, st) ||
            cudaStreamSynchronize(st))
            return DBP_ERR_CUDA;
        if (loss) loss[it] = (energy - 2.0 * r[K]) / m;
        if (done || it == max_iter) break;
        std::vector<double> delta(r.begin(), r.begin() + K);
        for (int i = 0; i < K; ++i) delta[i] *= sfac[i];
        cholesky_solve(L, K, delta);
        double dmax = 0.0, cmax = 1.0;
        for (int i = 0; i < K; ++i) {
            c[i] += delta[i];
            dmax = fmax(dmax, fabs(delta[i]));
            cmax = fmax(cmax, fabs(c[i]));
        }
        ++updates;
        done = dmax <= tol * cmax;
    }
    for (int i = 0; i < KC; ++i) coeffs[i] = c[i];
    if (phase) *phase = c[KC];
    if (n_iter) *n_iter = updates;
    return DBP_OK;
}
