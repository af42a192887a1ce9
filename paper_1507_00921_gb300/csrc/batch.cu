// Batched launch of many DBP jobs of uneven size in one CUDA graph.
//
// A batch is built once from a list of plans and their device buffers.  Jobs are
// grouped by block length N and the blocks of every group are cut into work units of as
// many blocks as one 512-thread CTA runs side by side at that length (batch_kernel.cu);
// one persistent kernel pops the units of all groups from one device counter, longest
// blocks first, so short and long waveforms, different link lengths, step counts and
// filter lengths share the SMs dynamically without one launch per job.  The kernel is
// captured in a CUDA graph; dbp_batch_run replays it with a single graph launch.
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

struct BatchImpl {
    int device = 0;
    int n_jobs = 0;
    int streaming = 0;
    int max_spins = 0;
    int grid = 0;
    long long n_units = 0;
    BatchJob *d_jobs = nullptr;               // all jobs, grouped by block length
    BatchGroupDev *d_groups = nullptr;
    BatchUnit *d_units = nullptr;
    int *d_ready = nullptr;                   // [n_jobs] publish flags (input order)
    unsigned long long *d_counter = nullptr;  // unit counter
    int *d_error = nullptr;
    int *h_one = nullptr;                     // pinned constant 1 for publishing
    cudaStream_t cap = nullptr;
    cudaEvent_t reset_done = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

static void batch_release(BatchImpl *B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->reset_done) cudaEventDestroy(B->reset_done);
    if (B->d_jobs) cudaFree(B->d_jobs);
    if (B->d_groups) cudaFree(B->d_groups);
    if (B->d_units) cudaFree(B->d_units);
    if (B->d_ready) cudaFree(B->d_ready);
    if (B->d_counter) cudaFree(B->d_counter);
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
    const int sizes[5] = {8192, 4096, 2048, 1024, 512};
    int rc = dev_alloc((void **)&B->d_ready, sizeof(int) * n_jobs);
    if (!rc) rc = dev_alloc((void **)&B->d_error, sizeof(int));
    if (!rc) rc = dev_alloc((void **)&B->d_counter, sizeof(unsigned long long));
    if (!rc) rc = dev_alloc((void **)&B->d_jobs, sizeof(BatchJob) * n_jobs);
    if (!rc && cudaMallocHost((void **)&B->h_one, sizeof(int)) != cudaSuccess) rc = DBP_ERR_ALLOC;
    if (rc) {
        batch_release(B);
        return rc;
    }
    *B->h_one = 1;
    // jobs grouped by block length (longest first), units of up to K(N) blocks per group
    std::vector<BatchJob> host;
    std::vector<BatchGroupDev> groups;
    std::vector<BatchUnit> units;
    host.reserve(n_jobs);
    for (int si = 0; si < 5; ++si) {
        const int N = sizes[si];
        const size_t first = host.size();
        long long items = 0;
        for (int j = 0; j < n_jobs; ++j) {
            const PlanImpl &P = plans[j]->impl;
            if (P.info.fft_size != N) continue;
            BatchJob J;
            memset(&J, 0, sizeof(J));
            fill_fwd_params(P, J.p);
            J.p.in = (const float2 *)ins[j];
            J.p.out = (float2 *)outs[j];
            J.p.bulk_store = 0;
            J.item0 = items;
            J.essfm = P.method == DBP_ESSFM;
            J.ready = B->d_ready + j;
            items += (long long)P.info.n_blocks * P.signal.n_waveforms;
            host.push_back(J);
        }
        if (host.size() == first) continue;
        BatchGroupDev g;
        g.jobs = B->d_jobs + first;
        g.n_jobs = (int)(host.size() - first);
        g.N = N;
        const int k = batch_unit_blocks(N);
        for (long long i = 0; i < items; i += k) {
            BatchUnit u;
            u.item0 = i;
            u.group = (int)groups.size();
            u.count = (int)(items - i < k ? items - i : k);
            units.push_back(u);
        }
        groups.push_back(g);
    }
    B->n_units = (long long)units.size();
    if (!rc) rc = dev_alloc((void **)&B->d_groups, sizeof(BatchGroupDev) * groups.size());
    if (!rc) rc = dev_alloc((void **)&B->d_units, sizeof(BatchUnit) * units.size());
    if (!rc && (cudaMemcpy(B->d_jobs, host.data(), sizeof(BatchJob) * host.size(), cudaMemcpyHostToDevice) !=
                    cudaSuccess ||
                cudaMemcpy(B->d_groups, groups.data(), sizeof(BatchGroupDev) * groups.size(),
                           cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(B->d_units, units.data(), sizeof(BatchUnit) * units.size(), cudaMemcpyHostToDevice) !=
                    cudaSuccess))
        rc = DBP_ERR_CUDA;
    if (!rc && (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&B->reset_done, cudaEventDisableTiming) != cudaSuccess))
        rc = DBP_ERR_CUDA;
    if (!rc) rc = prepare_batch_unified(&B->grid);
    if (!rc && B->n_units < B->grid) B->grid = (int)(B->n_units > 0 ? B->n_units : 1);
    // capture the one kernel launch
    if (!rc && cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = DBP_ERR_CUDA;
    if (!rc) {
        int crc = launch_batch_unified(B->d_groups, B->d_units, B->n_units, B->d_counter, B->d_error, B->max_spins,
                                       B->grid, B->cap);
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
    if (cudaMemsetAsync(B->d_counter, 0, sizeof(unsigned long long), st) != cudaSuccess ||
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
    // proceeds while the persistent kernel occupies the SMs
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
