// Adjoint DBP kernels for block length N = 512 (ESSFM and SSFM variants).
#include "adj_kernel.cuh"

namespace dbp {
int launch_adj_512(const AdjParams &q, int n_wave, bool essfm, cudaStream_t st) {
    return launch_adj_n<512>(q, n_wave, essfm, st);
}
}  // namespace dbp
