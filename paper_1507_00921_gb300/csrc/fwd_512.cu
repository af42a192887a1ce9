// Forward DBP kernels for block length N = 512 (ESSFM and SSFM variants).
#include "fwd_kernel.cuh"

namespace dbp {
int launch_fwd_512(const FwdParams &p, int n_wave, bool essfm, cudaStream_t st) {
    return launch_fwd_n<512>(p, n_wave, essfm, st);
}
}  // namespace dbp

namespace dbp {
int prepare_batch_512(long long n_items, int *grid) { return prepare_batch_n<512>(n_items, grid); }
int launch_batch_512(const BatchJob *jobs, int n_jobs, long long n_items, unsigned long long *counter, int *error,
                  int max_spins, int grid, cudaStream_t st) {
    return launch_batch_n<512>(jobs, n_jobs, n_items, counter, error, max_spins, grid, st);
}
}  // namespace dbp
