// Forward DBP kernels for block length N = 1024 (ESSFM and SSFM variants).
#include "fwd_kernel.cuh"

namespace dbp {
int launch_fwd_1024(const FwdParams &p, int n_wave, bool essfm, cudaStream_t st) {
    return launch_fwd_n<1024>(p, n_wave, essfm, st);
}
}  // namespace dbp
