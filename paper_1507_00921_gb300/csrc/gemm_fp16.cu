// Split-precision (fp16) DFT-as-GEMM DBP kernels and their DFT-matrix table builder.
#include "gemm_kernel.cuh"

namespace dbp {

// F[k][n] = exp(-j 2 pi k n / NA) in FP64, split into hi + lo parts of the 16-bit type and
// packed as pairs (k, k+1) for fixed n: tables [Fr hi, Fr lo, Fi hi, Fi lo][n][k/2].
__global__ void build_f_fp16(uint32_t *F, int NA) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NA * NA / 2) return;
    const int n = i / (NA / 2), kp = i % (NA / 2);
    float re[2], im[2];
    for (int d = 0; d < 2; ++d) {
        const int k = 2 * kp + d;
        double s, c;
        sincospi(-2.0 * (double)((k * n) % NA) / (double)NA, &s, &c);
        re[d] = (float)c;
        im[d] = (float)s;
    }
    uint32_t h, l;
    Split16<DBP_SPLIT_FP16>::split(re[0], re[1], h, l);
    F[i] = h;
    F[NA * NA / 2 + i] = l;
    Split16<DBP_SPLIT_FP16>::split(im[0], im[1], h, l);
    F[NA * NA + i] = h;
    F[3 * NA * NA / 2 + i] = l;
}

int build_f_tables_fp16(uint32_t *F, int NA) {
    build_f_fp16<<<(NA * NA / 2 + 255) / 256, 256>>>(F, NA);
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

int launch_gemm_fp16(const GemmParams &q, int N, int NA, int n_wave, bool essfm, cudaStream_t st) {
    if (N == 1024 && NA == 64) return launch_gemm_n<1024, 64, DBP_SPLIT_FP16>(q, n_wave, essfm, st);
    if (N == 1024 && NA == 128) return launch_gemm_n<1024, 128, DBP_SPLIT_FP16>(q, n_wave, essfm, st);
    if (N == 1024 && NA == 256) return launch_gemm_n<1024, 256, DBP_SPLIT_FP16>(q, n_wave, essfm, st);
    if (N == 2048 && NA == 64) return launch_gemm_n<2048, 64, DBP_SPLIT_FP16>(q, n_wave, essfm, st);
    if (N == 2048 && NA == 128) return launch_gemm_n<2048, 128, DBP_SPLIT_FP16>(q, n_wave, essfm, st);
    if (N == 2048 && NA == 256) return launch_gemm_n<2048, 256, DBP_SPLIT_FP16>(q, n_wave, essfm, st);
    if (N == 4096 && NA == 128) return launch_gemm_n<4096, 128, DBP_SPLIT_FP16>(q, n_wave, essfm, st);
    if (N == 4096 && NA == 256) return launch_gemm_n<4096, 256, DBP_SPLIT_FP16>(q, n_wave, essfm, st);
    return DBP_ERR_UNSUPPORTED;
}

}  // namespace dbp
