// Forward DBP kernels for block length N = 4096 (ESSFM and SSFM variants).
#include "fwd_kernel.cuh"

namespace dbp {
int launch_fwd_4096(const FwdParams &p, int n_wave, bool essfm, cudaStream_t st) {
    return launch_fwd_n<4096>(p, n_wave, essfm, st);
}
}  // namespace dbp

namespace dbp {
int prepare_batch_4096(long long n_items, int *grid) { return prepare_batch_n<4096>(n_items, grid); }
int launch_batch_4096(const BatchJob *jobs, int n_jobs, long long n_items, unsigned long long *counter, int *error,
                  int max_spins, int grid, cudaStream_t st) {
    return launch_batch_n<4096>(jobs, n_jobs, n_items, counter, error, max_spins, grid, st);
}
}  // namespace dbp
