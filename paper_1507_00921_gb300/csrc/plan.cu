// Planner, FP64 table builders and C-ABI entry points of libdbp.
//
// The planner turns the paper's link / signal / step parameters into the geometry of
// the overlap-and-save scheme (Section III) and the per-step constants of Section II:
//   beta2 = -D lambda^2 / (2 pi c)
//   dz_s: step lengths, step 0 next to the receiver
//   gamma_eff_s = gamma * manakov * integral over step s of exp(-alpha (z - z_span))
//                 (= (1 - exp(-alpha dz)) / alpha for a one-span step, Section II)
//   M = 2 pi |beta2| L f_s^2 (Section III, B = sampling rate), O = ceil(M) + 2 N_s N_c
//       rounded up to a multiple of 8 unless given.
// Tables built on the GPU in FP64 and rounded once to FP32:
//   H_s at digit-reversed position p: exp(+j 2 pi^2 beta2 f_k^2 dz_s) / N, with the
//   phase reduced modulo 2 pi in FP64 first (it reaches ~10^3 rad over 3200 km);
//   FFT twiddles W_N^{c k} (split as W_N^{(c mod 16) k} W_{N/16}^{(c div 16) k}) and
//   W_{N0 N1}^{n0 k1}.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "dbp_internal.cuh"

namespace dbp {

static const double kPi = 3.14159265358979323846;
static const double kC = 299792458.0;

// ------------------------------------------------------------------ FP64 table kernels
// FP32 pair for the complex value (c, s) of magnitude m (FP64): among the 3 x 3 FP32
// values within one unit in the last place of (c, s), the one whose magnitude is
// closest to m (ties: the nearest rounding).  Tables applied at every step and their
// conjugates in the inverse transform then do not drift in magnitude over many steps.
__device__ float2 round_unit(double c, double s, double m) {
    const float c0 = (float)c, s0 = (float)s;
    float bc = c0, bs = s0;
    double best = fabs(sqrt((double)c0 * c0 + (double)s0 * s0) - m);
    for (int i = -1; i <= 1; ++i)
        for (int j = -1; j <= 1; ++j) {
            if (i == 0 && j == 0) continue;
            const float cc = i < 0 ? nextafterf(c0, -INFINITY) : (i > 0 ? nextafterf(c0, INFINITY) : c0);
            const float ss = j < 0 ? nextafterf(s0, -INFINITY) : (j > 0 ? nextafterf(s0, INFINITY) : s0);
            const double e = fabs(sqrt((double)cc * cc + (double)ss * ss) - m);
            if (e < best) {
                best = e;
                bc = cc;
                bs = ss;
            }
        }
    return make_float2(bc, bs);
}

__global__ void build_h_kernel(float2 *H, int N, int n0, int n1, int n2, double beta2, double fs,
                               const double *dz, int n_tables) {
    const int pidx = blockIdx.x * blockDim.x + threadIdx.x;
    const int tbl = blockIdx.y;
    if (pidx >= N || tbl >= n_tables) return;
    const int k2 = pidx % n0;
    const int k1 = (pidx / n0) % n1;
    const int k0 = pidx / (n0 * n1);
    const int k = k0 + n2 * k1 + n2 * n1 * k2;
    const int kk = (k < N / 2) ? k : k - N;
    const double f = (double)kk * fs / (double)N;
    const double phi = 2.0 * kPi * kPi * beta2 * f * f * dz[tbl];
    const double two_pi = 2.0 * kPi;
    const double red = phi - two_pi * rint(phi / two_pi);
    double s, c;
    sincos(red, &s, &c);
    H[(size_t)tbl * N + pidx] = round_unit(c / N, s / N, 1.0 / N);
}

// Twiddle tables, stored k-major so that lanes reading consecutive rows for one k hit
// consecutive shared-memory banks.
__global__ void build_twiddle_kernel(float2 *twA, float2 *twB, float2 *tw2, int N, int n0, int n1, int n2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double s, co;
    if (i < 16 * n2) {                  // A[k][cl] = exp(-j 2 pi cl k / N), cl < 16
        const int k = i / 16, cl = i % 16;
        sincospi(-2.0 * (double)((cl * k) % N) / (double)N, &s, &co);
        twA[i] = round_unit(co, s, 1.0);
    }
    const int nb = n0 * n1 / 16;
    if (i < nb * n2) {                  // B[k][ch] = exp(-j 2 pi 16 ch k / N), ch < n0 n1 / 16
        const int k = i / nb, ch = i % nb;
        const long long m = (16LL * ch * k) % N;
        sincospi(-2.0 * (double)m / (double)N, &s, &co);
        twB[i] = round_unit(co, s, 1.0);
    }
    if (i < n0 * n1) {                  // W2[k1][a] = exp(-j 2 pi a k1 / (n0 n1)), a < n0
        const int k = i / n0, a = i % n0;
        sincospi(-2.0 * (double)((a * k) % (n0 * n1)) / (double)(n0 * n1), &s, &co);
        tw2[i] = round_unit(co, s, 1.0);
    }
}

// ------------------------------------------------------------------ host physics
static double beta2_of(const dbp_link &l) {
    const double D = l.D_ps_per_nm_km * 1e-12 / (1e-9 * 1e3);      // s/m^2
    return -D * l.lambda_m * l.lambda_m / (2.0 * kPi * kC);
}
static double alpha_of(const dbp_link &l) { return l.alpha_db_per_km * log(10.0) / 10.0 / 1e3; }

static double leff(double alpha, double dz) {
    return alpha == 0.0 ? dz : (1.0 - exp(-alpha * dz)) / alpha;
}

// integral over [a, b] of exp(-alpha (z - z_span_start(z)))
static double profile_integral(double alpha, double span, double a, double b) {
    if (b <= a) return 0.0;
    double total = 0.0;
    const long j0 = (long)floor(a / span), j1 = (long)ceil(b / span);
    for (long j = j0; j < j1; ++j) {
        const double s0 = (double)j * span;
        const double lo = a > s0 ? a : s0;
        const double hi = b < s0 + span ? b : s0 + span;
        if (hi <= lo) continue;
        total += leff(alpha, hi - s0) - leff(alpha, lo - s0);
    }
    return total;
}

static bool supported_n(int n) { return n == 512 || n == 1024 || n == 2048 || n == 4096 || n == 8192; }

static int validate(const dbp_link *link, const dbp_signal *sig, const dbp_steps *st) {
    if (!link || !sig || !st) return DBP_ERR_ARG;
    if (link->n_spans < 1 || !(link->span_len_m > 0) || !(link->lambda_m > 0) || !(link->alpha_db_per_km >= 0) ||
        !isfinite(link->D_ps_per_nm_km) || !isfinite(link->gamma_per_W_km) || !isfinite(link->manakov_factor))
        return DBP_ERR_ARG;
    if (!(sig->sample_rate_hz > 0) || sig->n_samples < 1 || sig->n_waveforms < 1) return DBP_ERR_ARG;
    if (sig->boundary != DBP_PERIODIC && sig->boundary != DBP_ZERO) return DBP_ERR_ARG;
    if (sig->n_pols != 0 && sig->n_pols != 1 && sig->n_pols != 2) return DBP_ERR_ARG;
    if (st->method != DBP_SSFM && st->method != DBP_ESSFM && st->method != DBP_FFE) return DBP_ERR_ARG;
    if (st->scheme != DBP_SCHEME_FUSED && st->scheme != DBP_SCHEME_PER_STEP) return DBP_ERR_ARG;
    if (st->n_steps < 1 || st->n_steps > DBP_MAX_STEPS) return DBP_ERR_ARG;
    if (st->n_taps < 0 || st->n_taps > DBP_MAX_TAPS) return DBP_ERR_ARG;
    if (st->method != DBP_ESSFM && st->n_taps != 0) return DBP_ERR_ARG;
    if (st->coeffs_per_step != 0 && st->coeffs_per_step != 1) return DBP_ERR_ARG;
    if (st->precision != DBP_FP32 && st->precision != DBP_SPLIT_BF16 && st->precision != DBP_SPLIT_FP16)
        return DBP_ERR_ARG;
    if (st->fft_size != 0 && !supported_n(st->fft_size)) return DBP_ERR_INFEASIBLE;
    if (st->fft_size == 0 && st->precision != DBP_FP32) return DBP_ERR_UNSUPPORTED;
    if (st->precision != DBP_FP32) {
        const int N = st->fft_size, NA = st->dft_block;
        if (N < 1024 || N > 4096 || (NA != 64 && NA != 128 && NA != 256) || N / NA < 4 || N / NA > 32)
            return DBP_ERR_UNSUPPORTED;
    }
    if (sig->n_pols == 1 && st->precision != DBP_FP32) return DBP_ERR_UNSUPPORTED;
    if (st->overlap < 0 || (st->overlap % 4) != 0) return DBP_ERR_ARG;
    if (st->step_len_m)
        for (int s = 0; s < st->n_steps; ++s)
            if (!(st->step_len_m[s] >= 0) || !isfinite(st->step_len_m[s])) return DBP_ERR_ARG;
    if (st->gamma_eff)
        for (int s = 0; s < st->n_steps; ++s)
            if (!isfinite(st->gamma_eff[s])) return DBP_ERR_ARG;
    return DBP_OK;
}

int describe(const dbp_link *link, const dbp_signal *sig, const dbp_steps *st, dbp_plan_info *info,
                    double *dz, double *geff) {
    int rc = validate(link, sig, st);
    if (rc) return rc;
    const int ns = st->n_steps;
    const double L = link->n_spans * link->span_len_m;
    const double alpha = alpha_of(*link);
    const double gamma = link->gamma_per_W_km * 1e-3 * link->manakov_factor;
    double total = 0.0;
    double top = L;
    for (int s = 0; s < ns; ++s) {
        const double d = st->step_len_m ? st->step_len_m[s] : L / ns;
        const double bot = top - d;
        double g = st->gamma_eff ? st->gamma_eff[s] : gamma * profile_integral(alpha, link->span_len_m, bot, top);
        if (st->method == DBP_FFE) g = 0.0;   // linear sub-step only
        if (dz) dz[s] = d;
        if (geff) geff[s] = g;
        total += d;
        top = bot;
    }
    const double b2 = beta2_of(*link);
    const double mem = 2.0 * kPi * fabs(b2) * total * sig->sample_rate_hz * sig->sample_rate_hz;
    int o = st->overlap;
    if (o == 0) {
        long long need;
        if (st->scheme == DBP_SCHEME_PER_STEP) {   // largest per-step overlap ceil(M_s) + 2 N_c
            need = 0;
            for (int s = 0; s < ns; ++s) {
                const double d = st->step_len_m ? st->step_len_m[s] : L / ns;
                const double ms = 2.0 * kPi * fabs(b2) * d * sig->sample_rate_hz * sig->sample_rate_hz;
                const long long q = (long long)ceil(ms - 1e-9) + 2LL * st->n_taps;
                if (q > need) need = q;
            }
        } else {
            need = (long long)ceil(mem - 1e-9) + 2LL * ns * st->n_taps;
        }
        if (need > 0x3fffffff) return DBP_ERR_INFEASIBLE;
        o = (int)(((need + 7) / 8) * 8);
    }
    int fft = st->fft_size;
    if (fft == 0) {
        // Section III: the block length minimising the operation count per output
        // sample, N (8 log2 N + 21 + N_c) / (N - O) (FFE: 8 log2 N + 8), over the
        // supported lengths that exceed the overlap
        const double extra = st->method == DBP_FFE ? 8.0 : 21.0 + (st->method == DBP_ESSFM ? st->n_taps : 0);
        double best = 0.0;
        for (int cand = 512; cand <= 8192; cand *= 2) {
            if (o >= cand) continue;
            const double cost = cand * (8.0 * log2((double)cand) + extra) / (double)(cand - o);
            if (fft == 0 || cost < best) {
                fft = cand;
                best = cost;
            }
        }
        if (fft == 0) return DBP_ERR_INFEASIBLE;
    }
    if (o >= fft) return DBP_ERR_INFEASIBLE;
    const int valid = fft - o;
    const long long nb = (sig->n_samples + valid - 1) / valid;
    if (nb * sig->n_waveforms > 0x7fffffffLL) return DBP_ERR_ARG;
    if (info) {
        info->fft_size = fft;
        info->overlap = o;
        info->valid = valid;
        info->n_blocks = (int32_t)nb;
        info->n_steps = ns;
        info->n_taps = st->n_taps;
        info->beta2_s2_per_m = b2;
        info->memory_samples = mem;
        info->link_len_m = total;
    }
    return DBP_OK;
}

int upload_taps(PlanImpl &P, const float *host_coeffs) {
    const int ns = P.info.n_steps, nt = P.info.n_taps;
    float *h = (float *)calloc((size_t)ns * P.taps_stride, sizeof(float));
    if (!h) return DBP_ERR_ALLOC;
    for (int s = 0; s < ns; ++s) {
        const float *c = host_coeffs ? host_coeffs + (P.coeffs_per_step ? (size_t)s * (nt + 1) : 0) : nullptr;
        for (int i = 0; i <= nt; ++i) {
            const float ci = c ? c[i] : (i == 0 ? 1.0f : 0.0f);
            P.coeffs[(size_t)s * (nt + 1) + i] = ci;
            h[(size_t)s * P.taps_stride + i] = (float)(P.step_geff[s] * (double)ci);
        }
    }
    cudaError_t e = cudaMemcpy(P.d_taps, h, (size_t)ns * P.taps_stride * sizeof(float), cudaMemcpyHostToDevice);
    free(h);
    if (e == cudaSuccess)
        e = cudaMemcpy(P.d_craw, P.coeffs, sizeof(float) * (size_t)ns * (nt + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(P.d_geff, P.step_geff, sizeof(double) * ns, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

static void release(PlanImpl &P) {
    if (P.d_H) cudaFree(P.d_H);
    if (P.d_taps) cudaFree(P.d_taps);
    if (P.d_twA) cudaFree(P.d_twA);
    if (P.d_twB) cudaFree(P.d_twB);
    if (P.d_tw2) cudaFree(P.d_tw2);
    if (P.d_stage_in) cudaFree(P.d_stage_in);
    if (P.d_stage_out) cudaFree(P.d_stage_out);
    for (auto &s : P.aux)
        if (s) cudaStreamDestroy(s);
    for (auto &e : P.ev)
        if (e) cudaEventDestroy(e);
    if (P.d_craw) cudaFree(P.d_craw);
    if (P.d_geff) cudaFree(P.d_geff);
    if (P.d_adj) cudaFree(P.d_adj);
    if (P.d_Hn) cudaFree(P.d_Hn);
    if (P.d_Wn) cudaFree(P.d_Wn);
    if (P.d_F) cudaFree(P.d_F);
    if (P.d_Fu) cudaFree(P.d_Fu);
    if (P.d_err) cudaFree(P.d_err);
    if (P.d_pp) cudaFree(P.d_pp);
    free(P.step_dz);
    free(P.step_geff);
    free(P.coeffs);
}

static bool fault_inject_alloc() {
    const char *f = getenv("DBP_FAULT_INJECT");
    return f && strcmp(f, "alloc") == 0;
}

int dev_alloc(void **p, size_t bytes) {
    if (fault_inject_alloc()) return DBP_ERR_ALLOC;
    return cudaMalloc(p, bytes) == cudaSuccess ? DBP_OK : DBP_ERR_ALLOC;
}

// (Re)builds the H_s tables from P.step_dz on the GPU in FP64, synchronously; one table
// when all steps have the same length.
int build_h_tables(PlanImpl &P) {
    const int ns = P.info.n_steps, N = P.info.fft_size;
    bool shared = true;
    for (int s = 1; s < ns; ++s)
        if (P.step_dz[s] != P.step_dz[0]) shared = false;
    const int n_tables = shared ? 1 : ns;
    const int had = P.d_H ? (P.h_shared ? 1 : ns) : 0;
    if (had < n_tables) {
        if (P.d_H) cudaFree(P.d_H);
        P.d_H = nullptr;
        if (dev_alloc((void **)&P.d_H, sizeof(float2) * (size_t)N * n_tables)) return DBP_ERR_ALLOC;
    }
    P.h_shared = shared;
    int n0, n1, n2;
    host_geo(N, n0, n1, n2);
    double *d_dz = nullptr;
    int rc = dev_alloc((void **)&d_dz, sizeof(double) * n_tables);
    if (!rc && cudaMemcpy(d_dz, P.step_dz, sizeof(double) * n_tables, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = DBP_ERR_CUDA;
    if (!rc) {
        dim3 g((N + 255) / 256, n_tables);
        build_h_kernel<<<g, 256>>>(P.d_H, N, n0, n1, n2, P.info.beta2_s2_per_m, P.signal.sample_rate_hz, d_dz,
                                   n_tables);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) rc = DBP_ERR_CUDA;
    }
    if (!rc && P.precision != DBP_FP32) {
        // natural frequency order for the DFT-GEMM path (the digit map with n0 = N is the identity)
        if (P.d_Hn && had < n_tables) {
            cudaFree(P.d_Hn);
            P.d_Hn = nullptr;
        }
        if (!P.d_Hn && dev_alloc((void **)&P.d_Hn, sizeof(float2) * (size_t)N * n_tables)) rc = DBP_ERR_ALLOC;
        if (!rc) {
            dim3 g((N + 255) / 256, n_tables);
            build_h_kernel<<<g, 256>>>(P.d_Hn, N, N, 1, 1, P.info.beta2_s2_per_m, P.signal.sample_rate_hz, d_dz,
                                       n_tables);
            if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) rc = DBP_ERR_CUDA;
        }
    }
    if (d_dz) cudaFree(d_dz);
    return rc;
}

static int make_plan(const dbp_link *link, const dbp_signal *sig, const dbp_steps *st, dbp_plan_t **out) {
    if (!out) return DBP_ERR_ARG;
    *out = nullptr;
    dbp_plan_info info;
    int rc = describe(link, sig, st, &info, nullptr, nullptr);
    if (rc) return rc;
    dbp_plan_t *plan = new (std::nothrow) dbp_plan_t();
    if (!plan) return DBP_ERR_ALLOC;
    PlanImpl &P = plan->impl;
    P.link = *link;
    P.signal = *sig;
    if (P.signal.n_pols == 0) P.signal.n_pols = 2;
    P.info = info;
    P.method = st->method;
    P.coeffs_per_step = st->coeffs_per_step;
    P.precision = st->precision;
    P.scheme = st->scheme;
    P.user_overlap = st->overlap;
    P.dft_block = st->precision == DBP_FP32 ? 0 : st->dft_block;
    P.n_tapblk = st->method == DBP_ESSFM ? tap_blocks(st->n_taps) : 0;
    P.taps_stride = 1 + 8 * P.n_tapblk;
    const int ns = st->n_steps, N = info.fft_size;
    P.step_dz = (double *)malloc(sizeof(double) * ns);
    P.step_geff = (double *)malloc(sizeof(double) * ns);
    P.coeffs = (float *)malloc(sizeof(float) * (size_t)ns * (st->n_taps + 1));
    if (!P.step_dz || !P.step_geff || !P.coeffs) {
        release(P);
        delete plan;
        return DBP_ERR_ALLOC;
    }
    describe(link, sig, st, nullptr, P.step_dz, P.step_geff);
    if (cudaGetDevice(&P.device) != cudaSuccess) {
        release(P);
        delete plan;
        return DBP_ERR_CUDA;
    }
    int n0, n1, n2;
    host_geo(N, n0, n1, n2);
    rc = build_h_tables(P);
    if (!rc) rc = dev_alloc((void **)&P.d_taps, sizeof(float) * (size_t)ns * P.taps_stride);
    if (!rc) rc = dev_alloc((void **)&P.d_craw, sizeof(float) * (size_t)ns * (st->n_taps + 1));
    if (!rc) rc = dev_alloc((void **)&P.d_geff, sizeof(double) * ns);
    if (!rc) rc = dev_alloc((void **)&P.d_twA, sizeof(float2) * (size_t)16 * n2);
    if (!rc) rc = dev_alloc((void **)&P.d_twB, sizeof(float2) * (size_t)(n0 * n1 / 16) * n2);
    if (!rc) rc = dev_alloc((void **)&P.d_tw2, sizeof(float2) * (size_t)n0 * n1);
    if (!rc) {
        build_twiddle_kernel<<<(N + 255) / 256, 256>>>(P.d_twA, P.d_twB, P.d_tw2, N, n0, n1, n2);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(0) != cudaSuccess) rc = DBP_ERR_CUDA;
    }
    if (!rc) rc = upload_taps(P, st->coeffs);
    if (!rc && P.precision != DBP_FP32) rc = build_gemm_tables(P);
    if (rc) {
        release(P);
        delete plan;
        return rc;
    }
    *out = plan;
    return DBP_OK;
}

bool overlaps(const void *a, const void *b, size_t bytes) {
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + bytes && y < x + bytes;
}

void fill_fwd_params(const PlanImpl &P, FwdParams &p) {
    p.in = nullptr;
    p.out = nullptr;
    p.n = P.signal.n_samples;
    p.n_blocks = P.info.n_blocks;
    p.valid = P.info.valid;
    p.half_overlap = P.info.overlap / 2;
    p.boundary = P.signal.boundary;
    p.n_steps = P.info.n_steps;
    p.n_tapblk = P.n_tapblk;
    p.taps_stride = P.taps_stride;
    p.h_stride = P.h_shared ? 0 : P.info.fft_size;
    p.H = P.d_H;
    p.taps = P.d_taps;
    p.twA = P.d_twA;
    p.twB = P.d_twB;
    p.tw2 = P.d_tw2;
    p.prefetch_ahead = P.prefetch_ahead;
    p.linear_only = P.method == DBP_FFE ? 1 : 0;
    p.single_pol = P.signal.n_pols == 1 ? 1 : 0;
    p.bulk_store = 0;
    p.fast_exp = (P.method == DBP_ESSFM && P.info.n_steps <= 2) ? 1 : 0;
}

// Outputs can be written by bulk copies when every waveform's polarization rows start
// on 16-byte boundaries.
static int bulk_ok(const void *out, long long n) {
    return ((uintptr_t)out % 16 == 0 && n % 2 == 0) ? 1 : 0;
}

static int launch_fwd(const FwdParams &p, int N, int n_wave, bool essfm, cudaStream_t st) {
    switch (N) {
        case 512: return launch_fwd_512(p, n_wave, essfm, st);
        case 1024: return launch_fwd_1024(p, n_wave, essfm, st);
        case 2048: return launch_fwd_2048(p, n_wave, essfm, st);
        case 4096: return launch_fwd_4096(p, n_wave, essfm, st);
        case 8192: return launch_fwd_8192(p, n_wave, essfm, st);
        default: return DBP_ERR_INFEASIBLE;
    }
}

// Per-step scheme: one single-step pass per step, each through HBM with the step's own
// overlap, ping-ponging between `out` and one plan-owned buffer so the last step writes
// `out`.
static int launch_per_step(const PlanImpl &P, const void *in, void *out, int n_wave, cudaStream_t st) {
    const int N = P.info.fft_size, ns = P.info.n_steps;
    const size_t bytes = (size_t)P.signal.n_pols * P.signal.n_samples * sizeof(float2) * n_wave;
    PlanImpl &M = const_cast<PlanImpl &>(P);
    if (ns > 1 && M.pp_bytes < bytes) {
        if (M.d_pp) cudaFree(M.d_pp);
        M.d_pp = nullptr;
        M.pp_bytes = 0;
        if (dev_alloc(&M.d_pp, bytes)) return DBP_ERR_ALLOC;
        M.pp_bytes = bytes;
    }
    const double fs = P.signal.sample_rate_hz;
    const void *src = in;
    for (int s = 0; s < ns; ++s) {
        void *dst = ((ns - 1 - s) % 2 == 0) ? out : M.d_pp;
        FwdParams p;
        fill_fwd_params(P, p);
        int o = P.user_overlap;
        if (o == 0) {
            const double ms = 2.0 * M_PI * fabs(P.info.beta2_s2_per_m) * P.step_dz[s] * fs * fs;
            const long long q = (long long)ceil(ms - 1e-9) + 2LL * P.info.n_taps;
            o = (int)(((q + 7) / 8) * 8);
        }
        p.in = (const float2 *)src;
        p.out = (float2 *)dst;
        p.bulk_store = bulk_ok(dst, P.signal.n_samples);
        p.n_steps = 1;
        p.valid = N - o;
        p.half_overlap = o / 2;
        p.n_blocks = (int)((P.signal.n_samples + p.valid - 1) / p.valid);
        p.H = P.d_H + (P.h_shared ? 0 : (size_t)N * s);
        p.h_stride = 0;
        p.taps = P.d_taps + (size_t)P.taps_stride * s;
        const int rc = launch_fwd(p, N, n_wave, P.method == DBP_ESSFM, st);
        if (rc) return rc;
        src = dst;
    }
    return DBP_OK;
}

int launch(const PlanImpl &P, const void *in, void *out, int n_wave, cudaStream_t st) {
    if (P.precision != DBP_FP32) return launch_gemm_plan(P, in, out, n_wave, st);
    if (P.scheme == DBP_SCHEME_PER_STEP) return launch_per_step(P, in, out, n_wave, st);
    FwdParams p;
    fill_fwd_params(P, p);
    p.in = (const float2 *)in;
    p.out = (float2 *)out;
    p.bulk_store = bulk_ok(out, P.signal.n_samples);
    const bool essfm = P.method == DBP_ESSFM;
    switch (P.info.fft_size) {
        case 512: return launch_fwd_512(p, n_wave, essfm, st);
        case 1024: return launch_fwd_1024(p, n_wave, essfm, st);
        case 2048: return launch_fwd_2048(p, n_wave, essfm, st);
        case 4096: return launch_fwd_4096(p, n_wave, essfm, st);
        case 8192: return launch_fwd_8192(p, n_wave, essfm, st);
        default: return DBP_ERR_INFEASIBLE;
    }
}

static size_t waveform_bytes(const PlanImpl &P) {
    return (size_t)P.signal.n_pols * P.signal.n_samples * sizeof(float2);
}

}  // namespace dbp

using namespace dbp;

extern "C" {

int dbp_plan_describe(const dbp_link *link, const dbp_signal *signal, const dbp_steps *steps, dbp_plan_info *info,
                      double *step_dz, double *step_gamma_eff) {
    return describe(link, signal, steps, info, step_dz, step_gamma_eff);
}

int dbp_plan(const dbp_link *link, const dbp_signal *signal, const dbp_steps *steps, dbp_plan_t **out) {
    return make_plan(link, signal, steps, out);
}

int dbp_plan_get_info(const dbp_plan_t *plan, dbp_plan_info *info) {
    if (!plan || !info) return DBP_ERR_ARG;
    *info = plan->impl.info;
    return DBP_OK;
}

int dbp_set_coeffs(dbp_plan_t *plan, const float *host_coeffs) {
    if (!plan || !host_coeffs) return DBP_ERR_ARG;
    if (plan->impl.method != DBP_ESSFM) return DBP_ERR_ARG;
    return upload_taps(plan->impl, host_coeffs);
}

int dbp_run(dbp_plan_t *plan, const void *in, void *out, dbp_stream_t stream) {
    if (!plan || !in || !out) return DBP_ERR_ARG;
    const PlanImpl &P = plan->impl;
    const size_t bytes = waveform_bytes(P) * P.signal.n_waveforms;
    if (overlaps(in, out, bytes)) return DBP_ERR_ALIAS;
    return launch(P, in, out, P.signal.n_waveforms, (cudaStream_t)stream);
}

int dbp_run_host(dbp_plan_t *plan, const void *in, void *out, dbp_stream_t stream) {
    if (!plan || !in || !out) return DBP_ERR_ARG;
    PlanImpl &P = plan->impl;
    const size_t wb = waveform_bytes(P);
    const int nw = P.signal.n_waveforms;
    const size_t bytes = wb * nw;
    if (overlaps(in, out, bytes)) return DBP_ERR_ALIAS;
    cudaStream_t st = (cudaStream_t)stream;
    if (P.stage_bytes < bytes) {
        if (P.d_stage_in) cudaFree(P.d_stage_in);
        if (P.d_stage_out) cudaFree(P.d_stage_out);
        P.d_stage_in = P.d_stage_out = nullptr;
        P.stage_bytes = 0;
        if (dev_alloc(&P.d_stage_in, bytes) || dev_alloc(&P.d_stage_out, bytes)) return DBP_ERR_ALLOC;
        P.stage_bytes = bytes;
    }
    if (!P.aux[0]) {
        for (auto &s : P.aux)
            if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return DBP_ERR_CUDA;
        for (auto &e : P.ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return DBP_ERR_CUDA;
    }
    // Pipeline: chunks of waveforms rotate over three streams, so that the copy in of one
    // chunk, the kernel of the previous one and the copy out of the one before overlap.
    const int chunks = nw >= 24 ? 24 : nw;
    if (cudaEventRecord(P.ev[0], st) != cudaSuccess) return DBP_ERR_CUDA;
    for (auto &s : P.aux)
        if (cudaStreamWaitEvent(s, P.ev[0], 0) != cudaSuccess) return DBP_ERR_CUDA;
    int w0 = 0;
    for (int c = 0; c < chunks; ++c) {
        const int w1 = (int)(((long long)nw * (c + 1)) / chunks);
        const int cnt = w1 - w0;
        if (cnt <= 0) continue;
        cudaStream_t s = P.aux[c % 3];
        const size_t off = wb * w0, len = wb * cnt;
        if (cudaMemcpyAsync((char *)P.d_stage_in + off, (const char *)in + off, len, cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
            return DBP_ERR_CUDA;
        int rc = launch(P, (char *)P.d_stage_in + off, (char *)P.d_stage_out + off, cnt, s);
        if (rc) return rc;
        if (cudaMemcpyAsync((char *)out + off, (char *)P.d_stage_out + off, len, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess)
            return DBP_ERR_CUDA;
        w0 = w1;
    }
    for (int k = 0; k < 3; ++k) {
        if (cudaEventRecord(P.ev[1 + k], P.aux[k]) != cudaSuccess) return DBP_ERR_CUDA;
        if (cudaStreamWaitEvent(st, P.ev[1 + k], 0) != cudaSuccess) return DBP_ERR_CUDA;
    }
    return cudaStreamSynchronize(st) == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

int dbp_plan_status(dbp_plan_t *plan) {
    if (!plan) return DBP_ERR_ARG;
    PlanImpl &P = plan->impl;
    if (cudaDeviceSynchronize() != cudaSuccess) return DBP_ERR_CUDA;
    if (!P.d_err) return DBP_OK;
    int e = 0;
    if (cudaMemcpy(&e, P.d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DBP_ERR_CUDA;
    if (e && cudaMemset(P.d_err, 0, sizeof(int)) != cudaSuccess) return DBP_ERR_CUDA;
    return e;
}

void dbp_destroy(dbp_plan_t *plan) {
    if (!plan) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(plan->impl.device);
    cudaDeviceSynchronize();
    release(plan->impl);
    cudaSetDevice(cur);
    delete plan;
}

const char *dbp_strerror(int code) {
    switch (code) {
        case DBP_OK: return "ok";
        case DBP_ERR_ARG: return "invalid argument";
        case DBP_ERR_INFEASIBLE: return "infeasible plan: block length must exceed the overlap and be supported";
        case DBP_ERR_ALLOC: return "allocation failed";
        case DBP_ERR_CUDA: return "CUDA runtime error";
        case DBP_ERR_TIMEOUT: return "bounded device wait timed out";
        case DBP_ERR_ALIAS: return "output buffer overlaps input buffer";
        case DBP_ERR_UNSUPPORTED: return "unsupported option";
        case DBP_ERR_SCRATCH: return "problem exceeds the fixed scratch of dbp_run_noalloc";
        case DBP_ERR_SINGULAR: return "normal equations of the fit are not positive definite";
        default: return "unknown error";
    }
}

const char *dbp_version(void) { return "libdbp 0.1 (sm_103a)"; }

}  // extern "C"
