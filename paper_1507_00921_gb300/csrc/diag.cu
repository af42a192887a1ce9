// Diagnostics: an FP32 fused-multiply-add throughput kernel, used to measure the
// FP32-pipe peak that the DBP kernels are compared against.
#include "dbp_internal.cuh"

namespace dbp {

// Each thread runs 8 independent FMA chains, 16 FMAs per chain per iteration:
// 128 FMAs = 256 flop per thread per iteration.
__global__ void __launch_bounds__(256) fma_peak_kernel(float *out, int iters, float a, float b) {
    float x0 = threadIdx.x * 1e-3f, x1 = x0 + 1.f, x2 = x0 + 2.f, x3 = x0 + 3.f;
    float x4 = x0 + 4.f, x5 = x0 + 5.f, x6 = x0 + 6.f, x7 = x0 + 7.f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            x0 = fmaf(x0, a, b); x1 = fmaf(x1, a, b); x2 = fmaf(x2, a, b); x3 = fmaf(x3, a, b);
            x4 = fmaf(x4, a, b); x5 = fmaf(x5, a, b); x6 = fmaf(x6, a, b); x7 = fmaf(x7, a, b);
        }
    }
    const float s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

}  // namespace dbp

extern "C" int dbp_diag_fma(void *out, int n_blocks, int iters, dbp_stream_t stream) {
    if (!out || n_blocks < 1 || iters < 1) return DBP_ERR_ARG;
    dbp::fma_peak_kernel<<<n_blocks, 256, 0, (cudaStream_t)stream>>>((float *)out, iters, 0.999999f, 1e-6f);
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}
