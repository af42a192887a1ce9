// Plan-level glue of the split-precision DFT-GEMM path: tables and dispatch.
#include "gemm_kernel.cuh"

namespace dbp {

__global__ void build_wn_kernel(float2 *Wn, int N) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double s, c;
    sincospi(-2.0 * (double)m / (double)N, &s, &c);
    Wn[m] = make_float2((float)c, (float)s);
}

int build_gemm_tables(PlanImpl &P) {
    const int N = P.info.fft_size, NA = P.dft_block;
    if (!P.d_Wn && dev_alloc((void **)&P.d_Wn, sizeof(float2) * (size_t)N)) return DBP_ERR_ALLOC;
    if (!P.d_F && dev_alloc((void **)&P.d_F, sizeof(uint32_t) * (size_t)2 * NA * NA)) return DBP_ERR_ALLOC;
    build_wn_kernel<<<(N + 255) / 256, 256>>>(P.d_Wn, N);
    int rc = P.precision == DBP_SPLIT_BF16 ? build_f_tables_bf16(P.d_F, NA) : build_f_tables_fp16(P.d_F, NA);
    if (rc) return rc;
    if (!P.d_err) {
        if (dev_alloc((void **)&P.d_err, sizeof(int))) return DBP_ERR_ALLOC;
        if (cudaMemset(P.d_err, 0, sizeof(int)) != cudaSuccess) return DBP_ERR_CUDA;
    }
    if (umma_supported(N, NA)) {
        if (!P.d_Fu && dev_alloc((void **)&P.d_Fu, 65536)) return DBP_ERR_ALLOC;
        rc = build_fu_tables(P.d_Fu, P.precision);
        if (rc) return rc;
    }
    return cudaStreamSynchronize(0) == cudaSuccess && cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

int launch_gemm_plan(const PlanImpl &P, const void *in, void *out, int n_wave, cudaStream_t st) {
    GemmParams q;
    fill_fwd_params(P, q.f);
    q.f.in = (const float2 *)in;
    q.f.out = (float2 *)out;
    q.Hn = P.d_Hn;
    q.Wn = P.d_Wn;
    q.F = P.d_F;
    const bool essfm = P.method == DBP_ESSFM;
    bool used = false;
    const int rc = launch_umma(q, P.d_Fu, P.d_err, P.precision, P.info.fft_size, n_wave, essfm, st, &used);
    if (rc || used) return rc;
    if (P.precision == DBP_SPLIT_BF16)
        return launch_gemm_bf16(q, P.info.fft_size, P.dft_block, n_wave, essfm, st);
    return launch_gemm_fp16(q, P.info.fft_size, P.dft_block, n_wave, essfm, st);
}

}  // namespace dbp
