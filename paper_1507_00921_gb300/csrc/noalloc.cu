// dbp_run_noalloc: backpropagation without any device allocation.
//
// Some callers cannot allocate device memory at all: a host that hands the library
// pre-reserved buffers under a fixed memory budget, an application whose allocator must
// not be re-entered from a library, or a real-time receiver loop that cannot afford the
// device-wide synchronisation a cudaMalloc / cudaFree may bring.  This entry point serves
// them.  It needs no plan: every call computes the step table on the host and builds the
// dispersion transfer functions, twiddles and filter taps in one fixed scratch area, a
// file-scope __device__ array that every GPU loading the library holds until the process
// exits, then runs the same fused DBP kernel as dbp_run.  The caller still provides the
// input and output buffers.  The host-side per-call values (filter taps, step lengths)
// reach the device as kernel arguments, so no host memory is read by a copy.
#include <mutex>

#include "dbp_internal.cuh"

namespace dbp {

// Fixed scratch: H tables, filter taps, twiddles and step lengths of one call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DBP_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device, found once per device with that device
// current (in host code the symbol itself is only a host-side stand-in).  A
// cudaDeviceReset of the device invalidates it; the library does not support calls after
// one.
static void *g_scratch_addr[64];
static std::mutex g_scratch_mu;

static int scratch_for_current_device(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DBP_ERR_CUDA;
    if (dev < 0 || dev >= 64) return DBP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DBP_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DBP_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Host-computed values of one call, passed by value as the argument of the staging
// kernel (17 KB, within the 32 KB kernel-parameter limit of sm_70 and later).
constexpr int kNoallocTaps = DBP_NOALLOC_MAX_STEPS * (1 + 8 * ((DBP_MAX_TAPS + 7) / 8));
struct NoallocArgs {
    float taps[kNoallocTaps];            // gamma_eff_s * c_{s,i}, [n_steps][taps_stride]
    double dz[DBP_NOALLOC_MAX_STEPS];    // step lengths of the H tables
    int n_taps;                          // floats of taps in use
    int n_dz;                            // entries of dz in use
};
static_assert(sizeof(NoallocArgs) <= 32000, "kernel parameter limit");

__global__ void noalloc_stage_kernel(const NoallocArgs a, float *taps, double *dz) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n_taps; i += gridDim.x * blockDim.x) taps[i] = a.taps[i];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n_dz; i += gridDim.x * blockDim.x) dz[i] = a.dz[i];
}

}  // namespace dbp

using namespace dbp;

extern "C" int dbp_run_noalloc(const dbp_link *link, const dbp_signal *signal, const dbp_steps *steps,
                               const void *in, void *out, dbp_stream_t stream) {
    if (!link || !signal || !steps || !in || !out) return DBP_ERR_ARG;
    if (steps->n_steps < 1) return DBP_ERR_ARG;
    if (steps->n_steps > DBP_NOALLOC_MAX_STEPS) return DBP_ERR_SCRATCH;
    if (steps->precision != DBP_FP32 || steps->scheme != DBP_SCHEME_FUSED || signal->n_pols == 1)
        return DBP_ERR_UNSUPPORTED;
    double dz[DBP_NOALLOC_MAX_STEPS], geff[DBP_NOALLOC_MAX_STEPS];
    dbp_plan_info info;
    int rc = describe(link, signal, steps, &info, dz, geff);
    if (rc) return rc;
    const int ns = info.n_steps, nt = info.n_taps, N = info.fft_size;
    const size_t bytes_io = (size_t)2 * signal->n_samples * sizeof(float2) * signal->n_waveforms;
    if (overlaps(in, out, bytes_io)) return DBP_ERR_ALIAS;

    bool shared = true;
    for (int s = 1; s < ns; ++s)
        if (dz[s] != dz[0]) shared = false;
    const int n_tables = shared ? 1 : ns;
    const int n_tapblk = steps->method == DBP_ESSFM ? tap_blocks(nt) : 0;
    const int taps_stride = 1 + 8 * n_tapblk;
    int n0, n1, n2;
    host_geo(N, n0, n1, n2);

    // scratch layout (each piece 256-byte aligned)
    const size_t off_h = 0;
    const size_t off_taps = off_h + align256(sizeof(float2) * (size_t)N * n_tables);
    const size_t off_twa = off_taps + align256(sizeof(float) * (size_t)ns * taps_stride);
    const size_t off_twb = off_twa + align256(sizeof(float2) * (size_t)16 * n2);
    const size_t off_tw2 = off_twb + align256(sizeof(float2) * (size_t)(n0 * n1 / 16) * n2);
    const size_t off_dz = off_tw2 + align256(sizeof(float2) * (size_t)n0 * n1);
    const size_t total = off_dz + align256(sizeof(double) * (size_t)n_tables);
    if (total > DBP_NOALLOC_SCRATCH_BYTES) return DBP_ERR_SCRATCH;

    void *base = nullptr;
    rc = scratch_for_current_device(&base);
    if (rc) return rc;
    unsigned char *sc = (unsigned char *)base;
    cudaStream_t st = (cudaStream_t)stream;

    // taps gamma_eff_s * c_{s,i}, zero padded to whole 8-tap blocks (every entry written),
    // and the step lengths, staged into the scratch by a kernel that takes them as its
    // argument
    NoallocArgs args;
    args.n_taps = ns * taps_stride;
    args.n_dz = n_tables;
    for (int s = 0; s < ns; ++s) {
        const float *c = steps->coeffs ? steps->coeffs + (steps->coeffs_per_step ? (size_t)s * (nt + 1) : 0) : nullptr;
        for (int i = 0; i < taps_stride; ++i) {
            double ci = 0.0;
            if (i <= nt) ci = c ? (double)c[i] : (i == 0 ? 1.0 : 0.0);
            args.taps[s * taps_stride + i] = (float)(geff[s] * ci);
        }
    }
    for (int s = 0; s < n_tables; ++s) args.dz[s] = dz[s];
    noalloc_stage_kernel<<<4, 256, 0, st>>>(args, (float *)(sc + off_taps), (double *)(sc + off_dz));
    float2 *H = (float2 *)(sc + off_h);
    build_h_kernel<<<dim3((N + 255) / 256, n_tables), 256, 0, st>>>(H, N, n0, n1, n2, info.beta2_s2_per_m,
                                                                     signal->sample_rate_hz,
                                                                     (const double *)(sc + off_dz), n_tables);
    build_twiddle_kernel<<<(N + 255) / 256, 256, 0, st>>>((float2 *)(sc + off_twa), (float2 *)(sc + off_twb),
                                                          (float2 *)(sc + off_tw2), N, n0, n1, n2);
    if (cudaGetLastError() != cudaSuccess) return DBP_ERR_CUDA;

    PlanImpl P;
    P.link = *link;
    P.signal = *signal;
    P.info = info;
    P.method = steps->method;
    P.coeffs_per_step = steps->coeffs_per_step;
    P.n_tapblk = n_tapblk;
    P.taps_stride = taps_stride;
    P.h_shared = shared;
    if (cudaGetDevice(&P.device) != cudaSuccess) return DBP_ERR_CUDA;
    P.d_H = H;
    P.d_taps = (float *)(sc + off_taps);
    P.d_twA = (float2 *)(sc + off_twa);
    P.d_twB = (float2 *)(sc + off_twb);
    P.d_tw2 = (float2 *)(sc + off_tw2);
    return launch(P, in, out, signal->n_waveforms, st);
}
