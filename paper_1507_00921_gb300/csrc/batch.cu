// Batched launch of many DBP jobs of uneven size in one CUDA graph.
//
// A batch is built once from a list of plans and their device buffers.  Jobs are
// grouped by block length N; each group is served by one persistent kernel whose CTAs
// pop (job, waveform, block) items from a device counter, so short and long waveforms,
// different link lengths, step counts and filter lengths share the GPU without one
// launch per job.  The group kernels run on parallel branches of one captured CUDA
// graph; dbp_batch_run replays it with a single graph launch.
//
// Streaming: with DBP_BATCH_STREAMING every job waits (bounded) for dbp_batch_publish
// before its input is read, so a producer can fill input buffers while the batch is
// already running.  A job that is never published makes the waiting CTAs give up after
// the batch's timeout and dbp_batch_status returns DBP_ERR_TIMEOUT; nothing hangs.
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "dbp_internal.cuh"

namespace dbp {

struct BatchGroupHost {
    int N;
    int n_jobs;
    long long n_items;
    BatchJob *d_jobs;        // device
    int grid;
    cudaStream_t stream;
    cudaEvent_t done;
};

struct BatchImpl {
    int device = 0;
    int n_jobs = 0;
    int streaming = 0;
    int max_spins = 0;
    std::vector<BatchGroupHost> groups;
    std::vector<int> job_group, job_index;    // per input job
    BatchJob *d_jobs = nullptr;               // all jobs, grouped
    int *d_ready = nullptr;                   // [n_jobs] publish flags (input order)
    unsigned long long *d_counters = nullptr; // [groups]
    int *d_error = nullptr;
    int *h_one = nullptr;                     // pinned constant 1 for publishing
    cudaStream_t cap = nullptr;
    cudaEvent_t fork = nullptr, reset_done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static int prepare_group(BatchGroupHost &g) {
    switch (g.N) {
        case 512: return prepare_batch_512(g.n_items, &g.grid);
        case 1024: return prepare_batch_1024(g.n_items, &g.grid);
        case 2048: return prepare_batch_2048(g.n_items, &g.grid);
        case 4096: return prepare_batch_4096(g.n_items, &g.grid);
        case 8192: return prepare_batch_8192(g.n_items, &g.grid);
        default: return DBP_ERR_INFEASIBLE;
    }
}

static int launch_group(const BatchGroupHost &g, unsigned long long *counter, int *error, int max_spins,
                        cudaStream_t st) {
    switch (g.N) {
        case 512: return launch_batch_512(g.d_jobs, g.n_jobs, g.n_items, counter, error, max_spins, g.grid, st);
        case 1024: return launch_batch_1024(g.d_jobs, g.n_jobs, g.n_items, counter, error, max_spins, g.grid, st);
        case 2048: return launch_batch_2048(g.d_jobs, g.n_jobs, g.n_items, counter, error, max_spins, g.grid, st);
        case 4096: return launch_batch_4096(g.d_jobs, g.n_jobs, g.n_items, counter, error, max_spins, g.grid, st);
        case 8192: return launch_batch_8192(g.d_jobs, g.n_jobs, g.n_items, counter, error, max_spins, g.grid, st);
        default: return DBP_ERR_INFEASIBLE;
    }
}

static void batch_release(BatchImpl *B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    for (auto &g : B->groups) {
        if (g.stream) cudaStreamDestroy(g.stream);
        if (g.done) cudaEventDestroy(g.done);
    }
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->reset_done) cudaEventDestroy(B->reset_done);
    if (B->d_jobs) cudaFree(B->d_jobs);
    if (B->d_ready) cudaFree(B->d_ready);
    if (B->d_counters) cudaFree(B->d_counters);
    if (B->d_error) cudaFree(B->d_error);
    if (B->h_one) cudaFreeHost(B->h_one);
    delete B;
}

}  // namespace dbp

struct dbp_batch {
    dbp::BatchImpl *impl;
};

using namespace dbp;

extern "C" int dbp_batch_create(dbp_plan_t *const *plans, const void *const *ins, void *const *outs, int n_jobs,
                                int flags, int timeout_us, dbp_batch_t **out) {
    if (!plans || !ins || !outs || !out || n_jobs < 1 || timeout_us < 0) return DBP_ERR_ARG;
    if (flags & ~DBP_BATCH_STREAMING) return DBP_ERR_ARG;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DBP_ERR_CUDA;
    for (int j = 0; j < n_jobs; ++j) {
        if (!plans[j] || !ins[j] || !outs[j]) return DBP_ERR_ARG;
        const PlanImpl &P = plans[j]->impl;
        if (P.device != dev) return DBP_ERR_ARG;
        if (P.precision != DBP_FP32 || P.scheme != DBP_SCHEME_FUSED || P.signal.n_pols == 1)
            return DBP_ERR_UNSUPPORTED;
        const size_t bytes = (size_t)2 * P.signal.n_samples * sizeof(float2) * P.signal.n_waveforms;
        if (overlaps(ins[j], outs[j], bytes)) return DBP_ERR_ALIAS;
    }
    BatchImpl *B = new (std::nothrow) BatchImpl();
    if (!B) return DBP_ERR_ALLOC;
    B->device = dev;
    B->n_jobs = n_jobs;
    B->streaming = (flags & DBP_BATCH_STREAMING) ? 1 : 0;
    B->max_spins = timeout_us > 0 ? timeout_us : 1000000;   // polls of ~1 us
    B->job_group.assign(n_jobs, -1);
    B->job_index.assign(n_jobs, -1);
    const int sizes[5] = {8192, 4096, 2048, 1024, 512};
    int rc = dev_alloc((void **)&B->d_ready, sizeof(int) * n_jobs);
    if (!rc) rc = dev_alloc((void **)&B->d_error, sizeof(int));
    if (!rc) rc = dev_alloc((void **)&B->d_jobs, sizeof(BatchJob) * n_jobs);
    if (!rc && cudaMallocHost((void **)&B->h_one, sizeof(int)) != cudaSuccess) rc = DBP_ERR_ALLOC;
    if (rc) {
        batch_release(B);
        return rc;
    }
    *B->h_one = 1;
    std::vector<BatchJob> host;
    host.reserve(n_jobs);
    for (int si = 0; si < 5; ++si) {
        BatchGroupHost g{};
        g.N = sizes[si];
        const size_t first = host.size();
        long long items = 0;
        for (int j = 0; j < n_jobs; ++j) {
            const PlanImpl &P = plans[j]->impl;
            if (P.info.fft_size != g.N) continue;
            BatchJob J;
            memset(&J, 0, sizeof(J));
            fill_fwd_params(P, J.p);
            J.p.in = (const float2 *)ins[j];
            J.p.out = (float2 *)outs[j];
            J.item0 = items;
            J.essfm = P.method == DBP_ESSFM;
            J.ready = B->d_ready + j;
            items += (long long)P.info.n_blocks * P.signal.n_waveforms;
            B->job_group[j] = (int)B->groups.size();
            B->job_index[j] = (int)(host.size() - first);
            host.push_back(J);
        }
        if (host.size() == first) continue;
        g.n_jobs = (int)(host.size() - first);
        g.n_items = items;
        g.d_jobs = B->d_jobs + first;
        B->groups.push_back(g);
    }
    if (cudaMemcpy(B->d_jobs, host.data(), sizeof(BatchJob) * host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = DBP_ERR_CUDA;
    if (!rc) rc = dev_alloc((void **)&B->d_counters, sizeof(unsigned long long) * B->groups.size());
    if (!rc && (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->reset_done, cudaEventDisableTiming) != cudaSuccess))
        rc = DBP_ERR_CUDA;
    for (auto &g : B->groups) {
        if (rc) break;
        rc = prepare_group(g);
        if (rc) break;
        if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess)
            rc = DBP_ERR_CUDA;
    }
    // capture: fork one branch per block-length group, join
    if (!rc && cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = DBP_ERR_CUDA;
    if (!rc) {
        int crc = cudaEventRecord(B->fork, B->cap) == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
        for (size_t gi = 0; gi < B->groups.size() && !crc; ++gi) {
            BatchGroupHost &g = B->groups[gi];
            if (cudaStreamWaitEvent(g.stream, B->fork, 0) != cudaSuccess) crc = DBP_ERR_CUDA;
            if (!crc) crc = launch_group(g, B->d_counters + gi, B->d_error, B->max_spins, g.stream);
            if (!crc && cudaEventRecord(g.done, g.stream) != cudaSuccess) crc = DBP_ERR_CUDA;
            if (!crc && cudaStreamWaitEvent(B->cap, g.done, 0) != cudaSuccess) crc = DBP_ERR_CUDA;
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(B->cap, &graph);
        if (!crc && ec != cudaSuccess) crc = DBP_ERR_CUDA;
        B->graph = graph;
        if (!crc && cudaGraphInstantiate(&B->exec, B->graph, 0) != cudaSuccess) crc = DBP_ERR_CUDA;
        rc = crc;
    }
    if (rc) {
        batch_release(B);
        return rc;
    }
    dbp_batch_t *b = new (std::nothrow) dbp_batch_t();
    if (!b) {
        batch_release(B);
        return DBP_ERR_ALLOC;
    }
    b->impl = B;
    *out = b;
    return DBP_OK;
}

extern "C" int dbp_batch_run(dbp_batch_t *batch, dbp_stream_t stream) {
    if (!batch || !batch->impl) return DBP_ERR_ARG;
    BatchImpl *B = batch->impl;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(B->d_counters, 0, sizeof(unsigned long long) * B->groups.size(), st) != cudaSuccess ||
        cudaMemsetAsync(B->d_error, 0, sizeof(int), st) != cudaSuccess)
        return DBP_ERR_CUDA;
    // publish flags (any non-zero value means published): all set now, or all cleared for
    // streaming batches (then set one by one by dbp_batch_publish)
    if (cudaMemsetAsync(B->d_ready, B->streaming ? 0 : 1, sizeof(int) * B->n_jobs, st) != cudaSuccess)
        return DBP_ERR_CUDA;
    if (cudaEventRecord(B->reset_done, st) != cudaSuccess) return DBP_ERR_CUDA;
    return cudaGraphLaunch(B->exec, st) == cudaSuccess ? DBP_OK : DBP_ERR_CUDA;
}

extern "C" int dbp_batch_publish(dbp_batch_t *batch, int job, dbp_stream_t stream) {
    if (!batch || !batch->impl || job < 0 || job >= batch->impl->n_jobs) return DBP_ERR_ARG;
    BatchImpl *B = batch->impl;
    cudaStream_t st = (cudaStream_t)stream;
    // after the flags were cleared by dbp_batch_run; a copy (no kernel) so that it
    // proceeds while the persistent kernels occupy the SMs
    if (cudaStreamWaitEvent(st, B->reset_done, 0) != cudaSuccess ||
        cudaMemcpyAsync(B->d_ready + job, B->h_one, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return DBP_ERR_CUDA;
    return DBP_OK;
}

extern "C" int dbp_batch_status(dbp_batch_t *batch) {
    if (!batch || !batch->impl) return DBP_ERR_ARG;
    BatchImpl *B = batch->impl;
    int err = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return DBP_ERR_CUDA;
    if (cudaMemcpy(&err, B->d_error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return DBP_ERR_CUDA;
    return err;
}

extern "C" void dbp_batch_destroy(dbp_batch_t *batch) {
    if (!batch) return;
    cudaDeviceSynchronize();
    batch_release(batch->impl);
    delete batch;
}

extern "C" int dbp_run_batch(dbp_plan_t *const *plans, const void *const *ins, void *const *outs, int n,
                             dbp_stream_t stream) {
    dbp_batch_t *b = nullptr;
    int rc = dbp_batch_create(plans, ins, outs, n, 0, 0, &b);
    if (rc) return rc;
    rc = dbp_batch_run(b, stream);
    if (!rc) rc = dbp_batch_status(b);
    dbp_batch_destroy(b);
    return rc;
}
