/*
 * libdbp -- digital backpropagation (DBP) of polarization-multiplexed optical
 * signals with the split-step Fourier method (SSFM) and the enhanced SSFM (ESSFM),
 * on one NVIDIA GB300 (sm_103a).
 *
 * Method: Secondini et al., "Coherent 100G Nonlinear Compensation with Single-Step
 * Digital Backpropagation", arXiv:1507.00921.
 *   - Section II, Eq. 1:  linear sub-step  Y_k = X_k exp(-j 2 pi^2 beta2 f_k^2 dz)
 *   - Section II, Eq. 2:  SSFM nonlinear sub-step  z_k = y_k exp(-j gamma dz_eff |y_k|^2)
 *   - Section II, Eq. 3:  ESSFM nonlinear sub-step, a real symmetric filter c_0..c_Nc
 *     over the joint intensity |y_k|^2 = |y_k,1|^2 + |y_k,2|^2 of both polarizations
 *   - Section II, after Eq. 2:  dz_eff = (1 - exp(-alpha dz)) / alpha, steps chained
 *   - Section III:  overlap-and-save blocks of N samples, overlap >= channel memory
 *     M ~= 2 pi |beta2| L B^2 with B equal to the sampling rate
 * Backpropagation applies the inverse operators (+j phases), steps running from the
 * receiver back to the transmitter, each step linear sub-step first.
 *
 * Data layout: a waveform is complex64 (interleaved float re, im), polarization-major:
 * [n_waveforms][2][n_samples].  All device buffers are owned by the caller; the plan
 * owns its tables and scratch.  Every call returns 0 (DBP_OK) or a negative DBP_ERR_*
 * code; nothing is printed and no call aborts the process.  Calls on one plan are not
 * thread-safe; different plans may be used from different host threads.
 */
#ifndef DBP_H
#define DBP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define DBP_OK               0
#define DBP_ERR_ARG         -1   /* null pointer, non-positive size, bad enum value    */
#define DBP_ERR_INFEASIBLE  -2   /* block length <= overlap, or unsupported fft_size  */
#define DBP_ERR_ALLOC       -3   /* device or host allocation failed                  */
#define DBP_ERR_CUDA        -4   /* a CUDA runtime call failed                        */
#define DBP_ERR_TIMEOUT     -5   /* a bounded device wait gave up (batched launch)    */
#define DBP_ERR_ALIAS       -6   /* output buffer overlaps the input buffer           */
#define DBP_ERR_UNSUPPORTED -7   /* option not supported for this plan or call         */
#define DBP_ERR_SCRATCH     -8   /* dbp_run_noalloc: problem exceeds its fixed scratch */
#define DBP_ERR_SINGULAR    -9   /* dbp_fit_coeffs: normal equations not positive definite */

/* Enumerations. */
#define DBP_PERIODIC   0   /* waveform is periodic outside [0, n) (circular channel)  */
#define DBP_ZERO       1   /* waveform is zero outside [0, n)                          */
#define DBP_SSFM       0   /* Eq. 2 nonlinear sub-step (n_taps must be 0)               */
#define DBP_ESSFM      1   /* Eq. 3 nonlinear sub-step with n_taps = N_c coefficients   */
#define DBP_FFE        2   /* linear sub-step only: bulk dispersion compensation, the
                              feed-forward equaliser of Section III (n_taps must be 0)  */
#define DBP_SCHEME_FUSED    0   /* all N_s steps on chip per block; overlap covers the whole link */
#define DBP_SCHEME_PER_STEP 1   /* one pass per step through HBM; per-step overlap
                                   ceil(M_s) + 2 N_c, so short blocks suit long links  */
#define DBP_FP32       0   /* FFT linear sub-step in FP32                               */
#define DBP_SPLIT_BF16 1   /* linear sub-step as DFT-matrix GEMMs on the tensor cores,
                              BF16 hi/lo split operands, FP32 accumulation; dft_block
                              64 with fft_size 1024 or 2048 runs on tcgen05 (5th-gen
                              tensor cores, accumulators in tensor memory), the other
                              sizes on warp-level mma.sync                              */
#define DBP_SPLIT_FP16 2   /* the same with FP16 hi/lo split operands                  */

/* Opaque stream handle: a cudaStream_t (NULL = legacy default stream). */
typedef void *dbp_stream_t;

/* The fibre link (Section II parameters; Section IV link: spans of SMF + EDFAs). */
typedef struct {
    int32_t n_spans;            /* number of amplified spans, >= 1                       */
    double  span_len_m;         /* span length (m), > 0                                  */
    double  alpha_db_per_km;    /* power attenuation (dB/km), >= 0                       */
    double  D_ps_per_nm_km;     /* dispersion parameter D; beta2 = -D lambda^2/(2 pi c)  */
    double  lambda_m;           /* carrier wavelength (m), > 0                           */
    double  gamma_per_W_km;     /* Kerr coefficient gamma (1/(W km))                     */
    double  manakov_factor;     /* multiplies gamma (8/9 for the Manakov equation)       */
} dbp_link;

/* The received signal. */
typedef struct {
    double  sample_rate_hz;     /* f_s; also the bandwidth B of the memory rule          */
    int64_t n_samples;          /* samples per polarization per waveform, >= 1           */
    int32_t n_waveforms;        /* independent waveforms in one call, >= 1               */
    int32_t boundary;           /* DBP_PERIODIC or DBP_ZERO                              */
    int32_t n_pols;             /* 2 (or 0): polarization-multiplexed, complex64 [2][n]
                                   per waveform, P_k = |y_k,1|^2 + |y_k,2|^2 (Eq. 3);
                                   1: one polarization, complex64 [n] per waveform, the
                                   scalar form P_k = |y_k|^2 that Eq. 3 extends (gamma_eff
                                   uses the link's manakov_factor as given: 1 for a scalar
                                   link).  n_pols = 1 runs dbp_run, dbp_run_host and both
                                   schemes at FP32; dbp_grad, dbp_fit_coeffs, the batch calls
                                   and dbp_run_noalloc return DBP_ERR_UNSUPPORTED for it.  */
} dbp_signal;

/* The backpropagation steps. */
typedef struct {
    int32_t method;             /* DBP_SSFM, DBP_ESSFM or DBP_FFE                        */
    int32_t n_steps;            /* N_s >= 1; step 0 is next to the receiver              */
    int32_t n_taps;             /* N_c, 0..DBP_MAX_TAPS (0 for DBP_SSFM)                 */
    const float  *coeffs;       /* host; c_0..c_Nc: [n_steps][n_taps+1] if
                                   coeffs_per_step else [n_taps+1]; NULL -> c_0 = 1, rest 0 */
    int32_t coeffs_per_step;    /* 0 or 1                                                */
    const double *step_len_m;   /* host [n_steps] step lengths (sum should be the link
                                   length) or NULL for uniform L / N_s                   */
    const double *gamma_eff;    /* host [n_steps] gamma*manakov*dz_eff overrides or NULL  */
    int32_t fft_size;           /* N in {512,1024,2048,4096,8192}, or 0 (FP32 only): the
                                   supported N minimising Section III's operation count
                                   per output sample, N (8 log2 N + 21 + N_c) / (N - O)
                                   (FFE: 8 log2 N + 8), among those above the overlap O;
                                   dbp_plan_info.fft_size reports the choice            */
    int32_t overlap;            /* O: 0 = rule ceil(M) + 2 N_s N_c rounded up to a
                                   multiple of 8; else a multiple of 4 in [0, N)        */
    int32_t precision;          /* DBP_FP32, DBP_SPLIT_BF16 or DBP_SPLIT_FP16            */
    int32_t dft_block;          /* split precisions: DFT-GEMM size N_a in {64,128,256}
                                   with fft_size in {1024,2048,4096} and 4 <= N/N_a <= 32  */
    int32_t scheme;             /* DBP_SCHEME_FUSED or DBP_SCHEME_PER_STEP               */
} dbp_steps;

#define DBP_MAX_TAPS  64
#define DBP_MAX_STEPS 1024

/* Geometry and step table of a plan, computed on the host. */
typedef struct {
    int32_t fft_size;           /* N                                                     */
    int32_t overlap;            /* O (even); O/2 samples discarded at each block end
                                   (per-step scheme: the largest per-step overlap)       */
    int32_t valid;              /* N - O output samples per block                        */
    int32_t n_blocks;           /* blocks per waveform = ceil(n_samples / valid)         */
    int32_t n_steps;
    int32_t n_taps;
    double  beta2_s2_per_m;     /* beta2                                                 */
    double  memory_samples;     /* M = 2 pi |beta2| L f_s^2 (Section III)                */
    double  link_len_m;         /* L                                                     */
} dbp_plan_info;

typedef struct dbp_plan dbp_plan_t;

/*
 * Computes the plan geometry and per-step table on the host only (no CUDA call):
 * dz_s (step lengths) and gamma_eff_s = gamma * manakov * integral over step s of the
 * forward power profile exp(-alpha (z - z_span_start)) (equal to Section II's
 * dz_eff = (1 - exp(-alpha dz))/alpha for a one-span step).  step_dz / step_gamma_eff
 * may be NULL; otherwise they receive n_steps values.
 */
int dbp_plan_describe(const dbp_link *link, const dbp_signal *signal, const dbp_steps *steps,
                      dbp_plan_info *info, double *step_dz, double *step_gamma_eff);

/*
 * Creates a plan on the current CUDA device: validates the parameters, computes the
 * step table, and builds on the GPU, in FP64, the dispersion transfer functions
 * H_s(f_k) = exp(+j 2 pi^2 beta2 f_k^2 dz_s) / N (inverse of Eq. 1, phase reduced mod
 * 2 pi before rounding to FP32) and the FFT twiddles; uploads gamma_eff_s * c_{s,i}.
 * Synchronizes the legacy default stream before returning.  *out is owned by the
 * caller and released with dbp_destroy.
 */
int dbp_plan(const dbp_link *link, const dbp_signal *signal, const dbp_steps *steps,
             dbp_plan_t **out);

/* Geometry of an existing plan. */
int dbp_plan_get_info(const dbp_plan_t *plan, dbp_plan_info *info);

/*
 * Replaces the ESSFM coefficients (host array laid out as dbp_steps.coeffs, with the
 * plan's coeffs_per_step).  Takes effect for work enqueued after the call; the upload
 * is synchronous.
 */
int dbp_set_coeffs(dbp_plan_t *plan, const float *host_coeffs);

/*
 * Backpropagates n_waveforms waveforms: in and out are DEVICE pointers to
 * complex64 [n_waveforms][2][n_samples]; out must not overlap in (DBP_ERR_ALIAS).
 * One fused kernel per call: each thread block takes one overlap-save block of N
 * vector samples and runs all N_s steps (FFT, x H_s, IFFT, nonlinear sub-step) in
 * shared memory, writing its N - O central samples.  Asynchronous on `stream`.
 */
int dbp_run(dbp_plan_t *plan, const void *in, void *out, dbp_stream_t stream);

/*
 * Reverse-mode gradient of dbp_run (no counterpart in the paper's experiment, which fits
 * the coefficients by MSE, Section IV; derived from Eqs. 1-3 and Section III).  For a
 * real loss L with grad_out = dL/dRe(out) + j dL/dIm(out) (DEVICE complex64, same layout
 * as out), writes (each pointer may be NULL to skip; values are overwritten):
 *   grad_in      DEVICE complex64 [n_waveforms][2][n_samples]: dL/dRe(in) + j dL/dIm(in)
 *   d_coeffs     DEVICE float: dL/dc_{s,i}, [n_steps][n_taps+1] if coeffs_per_step, else
 *                [n_taps+1] summed over steps (c unscaled: theta = gamma_eff_s sum c_i S_i)
 *   d_gamma_eff  DEVICE float [n_steps]: dL/dgamma_eff_s
 *   d_step_len   DEVICE float [n_steps]: dL/ddz_s through H_s (gamma_eff_s held fixed)
 * for the plan's current coefficients and steps, on `stream`.  The plan allocates its
 * scratch (per-block gradients, spectra, step checkpoints, partial sums) on the first
 * call.  Deterministic: no floating-point atomics.  grad_in must not overlap in or
 * grad_out (DBP_ERR_ALIAS).
 */
int dbp_grad(dbp_plan_t *plan, const void *in, const void *grad_out, void *grad_in, float *d_coeffs,
             float *d_gamma_eff, float *d_step_len, dbp_stream_t stream);

/*
 * Replaces the step lengths dz_s (host [n_steps], rebuilds H_s on the GPU in FP64) and/or
 * the nonlinear strengths gamma_eff_s (host [n_steps]); NULL keeps the current values.
 * The overlap and block geometry are not changed.  Synchronizes the device.
 */
int dbp_set_steps(dbp_plan_t *plan, const double *step_len_m, const double *gamma_eff);

/*
 * Least-squares fit of a single-step ESSFM's coefficients (Section IV: the coefficients
 * minimise the mean square error between the ESSFM output and a target, e.g. the output
 * of a many-step SSFM, over a training part of the waveform).  The plan must be ESSFM
 * with n_steps = 1, FP32 precision, the fused scheme and two polarizations (else
 * DBP_ERR_UNSUPPORTED); its block geometry, H and gamma_eff are used as they are, its
 * coefficients are not changed (apply the result with dbp_set_coeffs).
 *   x, target  DEVICE complex64 [n_waveforms][2][n_samples]: the received waveforms and
 *              the targets for the plan's outputs.
 *   n_train    output samples [0, n_train) of every waveform enter the fit (<= 0: all).
 *   max_iter   Gauss-Newton updates at most (>= 0); tol: stop once every update of the
 *              parameters is at most tol * max(1, max |parameter|).
 *   coeffs     HOST double [n_taps + 1]: the start point on entry (c = 1, 0, ..., 0 is
 *              the SSFM, c = 0 the linear-only compensation), the fitted c_0..c_Nc on
 *              return (unscaled: theta = gamma_eff * sum_i c_i S_i).
 *   phase      HOST double or NULL.  Non-NULL: a common phase phi is fitted with the
 *              coefficients (theta + phi), start value on entry, fitted value on return;
 *              a receiver's carrier-phase recovery removes such a phase, so the
 *              coefficients are then not spent on matching the mean nonlinear phase.
 *   loss       HOST double [max_iter + 1] or NULL: mean over training vector samples of
 *              |t_k - z_k|^2 (both polarizations) at the start and after each update.
 *   n_iter     HOST int or NULL: updates made.
 * Uses the scratch of dbp_grad (allocated on first use); synchronizes `stream`.  The
 * normal matrix sum_k P_k S_k S_k^T does not depend on the parameters: it is built once
 * on the GPU and factored once; each iteration is one GPU pass over the training
 * samples.  Deterministic (fixed-order FP64 reductions).  DBP_ERR_SINGULAR when the
 * normal matrix is not positive definite (e.g. an all-zero input).  The objective is
 * not convex: different start points can end in different minima.
 */
int dbp_fit_coeffs(dbp_plan_t *plan, const void *x, const void *target, long long n_train, int max_iter,
                   double tol, double *coeffs, double *phase, double *loss, int *n_iter, dbp_stream_t stream);

/*
 * As dbp_run, but in and out are HOST pointers (pinned or pageable).  The plan
 * stages the data through device buffers it allocates on first use; copies and
 * compute are pipelined over chunks of waveforms.  Returns after the result is in
 * `out` (synchronizes `stream`).
 */
int dbp_run_host(dbp_plan_t *plan, const void *in, void *out, dbp_stream_t stream);

/*
 * Backpropagation for callers that cannot allocate device memory (no counterpart in
 * the paper).  Some callers cannot call cudaMalloc: a host that must keep to
 * pre-reserved device memory, an application whose allocator must not be re-entered
 * from a library, or a real-time receiver loop that cannot afford the device-wide
 * synchronisation an allocation or a free may bring.  This call takes the same link /
 * signal / step parameters as dbp_plan and the same DEVICE in/out buffers as dbp_run,
 * and computes exactly what dbp_plan + dbp_run compute (bit for bit), but it allocates
 * nothing: its tables (H_s, twiddles, filter taps) are rebuilt on every call in one
 * fixed scratch area of DBP_NOALLOC_SCRATCH_BYTES that lives in the library's device
 * image, so every GPU that loads the library holds it until the process exits.
 * Limits: at most DBP_NOALLOC_MAX_STEPS steps and tables that fit the scratch (for
 * example N = 8192 with equal step lengths, or up to 15 distinct step lengths at
 * N = 8192); beyond them it returns DBP_ERR_SCRATCH and does nothing.  Two
 * polarizations, FP32, fused scheme only (else DBP_ERR_UNSUPPORTED).
 * All calls share the one scratch area, which keeps the last call's tables (every entry
 * a call reads is rewritten by that call): calls that overlap on the GPU (different
 * streams, or different host threads) race on it and must be serialized by the caller.
 * The first call on each device looks up the scratch address with that device current
 * (a one-time set-up); make that first call before any stream capture.  Asynchronous on
 * `stream`: the host-side values of a call (taps, step lengths) travel as kernel
 * arguments, no host memory is copied.
 */
#define DBP_NOALLOC_SCRATCH_BYTES (1u << 20)
#define DBP_NOALLOC_MAX_STEPS 64
int dbp_run_noalloc(const dbp_link *link, const dbp_signal *signal, const dbp_steps *steps,
                    const void *in, void *out, dbp_stream_t stream);

/*
 * Batched launch of many jobs of uneven size (plans of any block length, link length,
 * step count and filter length, each with its own DEVICE in/out buffers; two
 * polarizations, FP32, fused scheme).  A batch is built once and replayed: the blocks
 * of all jobs are cut into work units (several blocks side by side for the shorter
 * block lengths), one persistent kernel pops the units of every block length from one
 * device counter, longest blocks first, and that kernel is captured in a CUDA graph.
 * Every job's output is bitwise equal to what dbp_run of its plan writes.
 * Plans and buffers must stay alive and unchanged in place while the batch exists.
 * flags: 0, or DBP_BATCH_STREAMING: every job's input is read only after
 * dbp_batch_publish(job) (a producer may fill inputs while the batch runs).  A job that
 * is not published within timeout_us microseconds (0 = 1 s) is skipped and the batch
 * reports DBP_ERR_TIMEOUT; the wait never hangs.
 */
#define DBP_BATCH_STREAMING 1
typedef struct dbp_batch dbp_batch_t;
int dbp_batch_create(dbp_plan_t *const *plans, const void *const *ins, void *const *outs, int n_jobs, int flags,
                     int timeout_us, dbp_batch_t **out);
/* Resets the work counters (and, when streaming, clears the publish flags) on `stream`,
 * then launches the batch graph after them.  Asynchronous. */
int dbp_batch_run(dbp_batch_t *batch, dbp_stream_t stream);
/* Streaming batches: marks job `job` (index into the create-time lists) as ready, on
 * `stream`, ordered after the flag reset of the latest dbp_batch_run.  Uses a copy, not
 * a kernel, so it proceeds while the batch occupies the SMs. */
int dbp_batch_publish(dbp_batch_t *batch, int job, dbp_stream_t stream);
/* Waits for the device and returns the batch status: DBP_OK or DBP_ERR_TIMEOUT. */
int dbp_batch_status(dbp_batch_t *batch);
void dbp_batch_destroy(dbp_batch_t *batch);
/* One-shot: create, run on `stream`, wait, destroy.  Returns the batch status. */
int dbp_run_batch(dbp_plan_t *const *plans, const void *const *ins, void *const *outs, int n_jobs,
                  dbp_stream_t stream);

/*
 * Waits for the device, then returns DBP_ERR_TIMEOUT if a bounded wait inside one of
 * the plan's tensor-core kernels (the split precisions' tcgen05 path) gave up since the
 * last call (its outputs are then incomplete), else DBP_OK; clears the record.
 */
int dbp_plan_status(dbp_plan_t *plan);

/* Frees the plan's device tables and scratch (synchronizes the device first). */
void dbp_destroy(dbp_plan_t *plan);

/* Static description of an error code. */
const char *dbp_strerror(int code);

/* Library version string. */
const char *dbp_version(void);

/*
 * Diagnostic (no counterpart in the paper): launches n_blocks x 256 threads that each
 * run iters x 128 independent FP32 FMAs (256 flop), for measuring the FP32-pipe peak the
 * DBP kernels are compared against.  `out` is a device buffer of n_blocks * 256 floats
 * that is normally left untouched.  Asynchronous on `stream`.
 */
int dbp_diag_fma(void *out, int n_blocks, int iters, dbp_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* DBP_H */
