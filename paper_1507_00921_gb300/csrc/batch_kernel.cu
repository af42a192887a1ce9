// One persistent kernel for a whole batch of uneven jobs (plans of any block length,
// link length, step count and filter length).
//
// Every CTA has 512 threads and the largest shared-memory footprint of all block
// lengths.  It pops work units from one device counter; a unit is a run of up to
// K(N) overlap-save blocks of one block length N (K = 1 at N = 8192, 2 at 4096, 4 at
// 2048, 7 at 1024, 14 at 512: as many N / 16-thread sub-groups with their own
// shared-memory slice as fit), and the sub-groups backpropagate their blocks side by side,
// each synchronised with its own named barrier.  Units of the longest blocks come
// first, so the last units to finish are the short ones.  Each block waits for its
// job's publish flag with a bounded spin (nanosleep between polls, at most max_spins
// polls); a flag that never appears records DBP_ERR_TIMEOUT in *error and the block is
// skipped, so nothing hangs.
#include "fwd_kernel.cuh"

namespace dbp {

// A sub-group's shared-memory slice: the block's own layout (Geo<N>), then the job
// parameters of its current block.
template <int N>
struct UnitGeo {
    static constexpr int T = Geo<N>::T;
    static constexpr size_t OFF_P = (Geo<N>::SMEM + 15) / 16 * 16;
    static constexpr size_t SLICE = OFF_P + (sizeof(FwdParams) + 15) / 16 * 16;
    static constexpr int K_THREADS = 512 / T;
    static constexpr int K_SMEM = (int)((size_t)(227 * 1024 - 1024) / SLICE);
    static constexpr int K = K_THREADS < K_SMEM ? (K_THREADS < 15 ? K_THREADS : 15) : (K_SMEM < 15 ? K_SMEM : 15);
    static_assert(K >= 1, "at least one block per unit");
};

constexpr size_t umax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kUnifiedSmem =
    umax(umax(umax(UnitGeo<8192>::K * UnitGeo<8192>::SLICE, UnitGeo<4096>::K * UnitGeo<4096>::SLICE),
              umax(UnitGeo<2048>::K * UnitGeo<2048>::SLICE, UnitGeo<1024>::K * UnitGeo<1024>::SLICE)),
         UnitGeo<512>::K * UnitGeo<512>::SLICE);
static_assert(kUnifiedSmem <= 227 * 1024 - 1024, "shared memory budget of the unified batch kernel");

int batch_unit_blocks(int N) {
    switch (N) {
        case 8192: return UnitGeo<8192>::K;
        case 4096: return UnitGeo<4096>::K;
        case 2048: return UnitGeo<2048>::K;
        case 1024: return UnitGeo<1024>::K;
        case 512: return UnitGeo<512>::K;
        default: return 0;
    }
}

// One unit of block length N: sub-group `sub` of N / 16 threads takes item item0 + sub.
// Returns with every sub-group's shared-memory use of the unit finished (the caller
// follows with a CTA barrier).  Not inlined, so that each block length gets its own
// register allocation (as a dedicated kernel would).
template <int N>
__device__ __noinline__ void run_unit(unsigned char *smem, const BatchGroupDev &G, const BatchUnit &U,
                                         bool load_tables, int *error, int max_spins, int *s_job, int *s_ok) {
    using UG = UnitGeo<N>;
    const int sub = threadIdx.x / UG::T;
    if (sub >= UG::K) return;                       // threads beyond the K sub-groups idle
    const int lt = threadIdx.x - sub * UG::T;
    Blk<N, true> blk(smem + (size_t)sub * UG::SLICE, lt);
    blk.bar_id = 1 + sub;
    if (load_tables) blk.load_tables(G.jobs[0].p.twA, G.jobs[0].p.twB, G.jobs[0].p.tw2);
    if (sub >= U.count) return;
    const long long item = U.item0 + sub;
    if (lt == 0) {
        int lo = 0, hi = G.n_jobs - 1;              // last job with item0 <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (G.jobs[mid].item0 <= item) lo = mid; else hi = mid - 1;
        }
        int ok = 1;
        const volatile int *flag = G.jobs[lo].ready;
        for (int spins = 0; *flag == 0;) {
            if (*(volatile int *)error != 0 || ++spins > max_spins) {
                atomicCAS(error, 0, DBP_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(1000);
        }
        __threadfence();
        s_job[sub] = lo;
        s_ok[sub] = ok;
    }
    FwdParams *sp = reinterpret_cast<FwdParams *>(smem + (size_t)sub * UG::SLICE + UG::OFF_P);
    if (lt == 0) *sp = G.jobs[s_job[sub]].p;       // the leader wrote s_job just above
    blk.sync();                                     // tables, job, flag and parameters visible
    if (!s_ok[sub]) return;
    const BatchJob &J = G.jobs[s_job[sub]];
    const long long local = item - J.item0;
    const int w = (int)(local / sp->n_blocks);
    const int b = (int)(local - (long long)w * sp->n_blocks);
    blk.prefetch_h(sp->H);
    if (J.essfm && sp->fast_exp)   // the same exponential as the job's own dbp_run
        process_block<N, true, false, true>(*sp, blk, w, b);
    else if (J.essfm)
        process_block<N, true, false>(*sp, blk, w, b);
    else
        process_block<N, false, false>(*sp, blk, w, b);
    if (lt == 0) bulk_wait_read_all();              // the slice may be reused by another length
}

__global__ void __launch_bounds__(512, 1)
    dbp_batch_unified_kernel(const BatchGroupDev *__restrict__ groups, const BatchUnit *__restrict__ units,
                             long long n_units, unsigned long long *counter, int *error, int max_spins) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_unit;
    __shared__ int s_job[16], s_ok[16];
    int cur_n = 0;                                  // block length whose tables are in shared memory
    for (;;) {
        if (threadIdx.x == 0) s_unit = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long u = s_unit;
        if (u >= n_units) break;
        const BatchUnit U = units[u];
        const BatchGroupDev G = groups[U.group];
        const bool tables = G.N != cur_n;
        switch (G.N) {
            case 8192: run_unit<8192>(smem_raw, G, U, tables, error, max_spins, s_job, s_ok); break;
            case 4096: run_unit<4096>(smem_raw, G, U, tables, error, max_spins, s_job, s_ok); break;
            case 2048: run_unit<2048>(smem_raw, G, U, tables, error, max_spins, s_job, s_ok); break;
            case 1024: run_unit<1024>(smem_raw, G, U, tables, error, max_spins, s_job, s_ok); break;
            default: run_unit<512>(smem_raw, G, U, tables, error, max_spins, s_job, s_ok); break;
        }
        cur_n = G.N;
        __syncthreads();                            // unit done: s_unit and the slices free
    }
    if (threadIdx.x % 32 == 0) bulk_wait_all();     // output copies complete before exit
}

// Grid of the unified kernel (one CTA per SM) and its shared-memory opt-in; call before
// any stream capture.
int prepare_batch_unified(int *grid) {
    static unsigned long long done = 0;
    if (!set_smem_once(dbp_batch_unified_kernel, kUnifiedSmem, done)) return DBP_ERR_CUDA;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dbp_batch_unified_kernel, 512, kUnifiedSmem) !=
            cudaSuccess)
        return DBP_ERR_CUDA;
    *grid = sms * (per_sm > 0 ? per_sm : 1);
    return DBP_OK;
}

int launch_batch_unified(const BatchGroupDev *groups, const BatchUnit *units, long long n_units,
                         unsigned long long *counter, int *error, int max_spins, int grid, cudaStream_t st) {
    dbp_batch_unified_kernel<<<(unsigned)grid, 512, kUnifiedSmem, st>>>(groups, units, n_units, counter, error,
                                                                        max_spins);
    return cudaGetLastError() == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

}  // namespace dbp
