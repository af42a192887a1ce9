// Tensor-core (tcgen05) split-precision DFT-GEMM path: the DFT-matrix tables in the
// canonical operand layout and the launchers of dbp_umma_kernel (N_a = 64).
#include <stdlib.h>
#include <string.h>

#include "umma_kernel.cuh"

namespace dbp {

// The real 128 x 128 matrix B of the 64-point DFT, B[k][n] = [[C, S], [-S, C]] with
// C = cos(2 pi na ka / 64), S = -sin(2 pi na ka / 64) (k = na or 64 + na: real or
// imaginary input part; n = ka or 64 + ka: real or imaginary output part), built in
// FP64, split into hi and lo parts of the 16-bit type (x = hi + lo), stored at the K-major
// canonical byte offsets of (row n, column k): hi in the first 32 KB, lo in the next.
template <int TY>
__global__ void build_fu_kernel(uint16_t *Fu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 128 * 128) return;
    const int nn = i / 128, k = i % 128;
    const int na = k % 64, ka = nn % 64;
    double s, c;
    sincospi(2.0 * (double)((na * ka) % 64) / 64.0, &s, &c);
    const double sm = -s;
    double val;
    if (k < 64) val = nn < 64 ? c : sm;
    else val = nn < 64 ? -sm : c;
    uint16_t hi, lo;
    if (TY == DBP_SPLIT_BF16) {
        const __nv_bfloat16 h = __double2bfloat16(val);
        const __nv_bfloat16 l = __double2bfloat16(val - (double)__bfloat162float(h));
        hi = *reinterpret_cast<const uint16_t *>(&h);
        lo = *reinterpret_cast<const uint16_t *>(&l);
    } else {
        const __half h = __double2half(val);
        const __half l = __double2half(val - (double)__half2float(h));
        hi = *reinterpret_cast<const uint16_t *>(&h);
        lo = *reinterpret_cast<const uint16_t *>(&l);
    }
    const uint32_t o = off_kmaj(nn, k) / 2;
    Fu[o] = hi;
    Fu[16384 + o] = lo;
}

int build_fu_tables(uint4 *Fu, int precision) {
    if (precision == DBP_SPLIT_BF16)
        build_fu_kernel<DBP_SPLIT_BF16><<<64, 256>>>(reinterpret_cast<uint16_t *>(Fu));
    else
        build_fu_kernel<DBP_SPLIT_FP16><<<64, 256>>>(reinterpret_cast<uint16_t *>(Fu));
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

template <int N, int TY>
static int launch_umma_n(const UmmaParams &u, cudaStream_t st) {
    using U = UGeo<N, TY>;
    static unsigned long long done = 0;
    static int sms[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DBP_ERR_CUDA;
    if (!set_smem_once(dbp_umma_kernel<N, TY>, U::SMEM, done)) return DBP_ERR_CUDA;
    if (!sms[dev] && cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return DBP_ERR_CUDA;
    const long long tiles = ((long long)u.total_blocks + U::G - 1) / U::G;
    const int grid = (int)(tiles < sms[dev] ? tiles : sms[dev]);
    dbp_umma_kernel<N, TY><<<grid, U::T, U::SMEM, st>>>(u);
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

bool umma_supported(int N, int NA) { return NA == 64 && (N == 1024 || N == 2048); }

// DBP_SPLIT_MMA_SYNC=1 selects the warp-level mma.sync kernel for N_a = 64 as well (for
// comparisons); by default N_a = 64 runs on tcgen05.
static bool legacy_forced() {
    const char *e = getenv("DBP_SPLIT_MMA_SYNC");
    return e && strcmp(e, "1") == 0;
}

int launch_umma(const GemmParams &q, const uint4 *Fu, int *err, int precision, int N, int n_wave, bool essfm,
                cudaStream_t st, bool *used) {
    *used = false;
    if (!Fu || !err || legacy_forced() || !umma_supported(N, 64)) return DBP_OK;
    UmmaParams u;
    u.g = q;
    u.Fu = Fu;
    u.err = err;
    const long long total = (long long)q.f.n_blocks * n_wave;
    if (total <= 0 || total > 0x7fffffffLL) return DBP_ERR_ARG;
    u.total_blocks = (int)total;
    u.essfm = essfm ? 1 : 0;
    *used = true;
    if (precision == DBP_SPLIT_BF16)
        return N == 1024 ? launch_umma_n<1024, DBP_SPLIT_BF16>(u, st) : launch_umma_n<2048, DBP_SPLIT_BF16>(u, st);
    return N == 1024 ? launch_umma_n<1024, DBP_SPLIT_FP16>(u, st) : launch_umma_n<2048, DBP_SPLIT_FP16>(u, st);
}

}  // namespace dbp
