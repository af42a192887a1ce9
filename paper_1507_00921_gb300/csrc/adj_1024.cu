// Adjoint DBP kernels for block length N = 1024 (ESSFM and SSFM variants).
#include "adj_kernel.cuh"

namespace dbp {
int launch_adj_1024(const AdjParams &q, int n_wave, bool essfm, cudaStream_t st) {
    return launch_adj_n<1024>(q, n_wave, essfm, st);
}
}  // namespace dbp
