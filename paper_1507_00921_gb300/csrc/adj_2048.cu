// Adjoint DBP kernels for block length N = 2048 (ESSFM and SSFM variants).
#include "adj_kernel.cuh"

namespace dbp {
int launch_adj_2048(const AdjParams &q, int n_wave, bool essfm, cudaStream_t st) {
    return launch_adj_n<2048>(q, n_wave, essfm, st);
}
}  // namespace dbp
