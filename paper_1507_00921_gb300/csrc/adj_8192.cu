// Adjoint DBP kernels for block length N = 8192 (ESSFM and SSFM variants).
#include "adj_kernel.cuh"

namespace dbp {
int launch_adj_8192(const AdjParams &q, int n_wave, bool essfm, cudaStream_t st) {
    return launch_adj_n<8192>(q, n_wave, essfm, st);
}
}  // namespace dbp
