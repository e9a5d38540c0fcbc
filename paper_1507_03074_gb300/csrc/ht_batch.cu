// C ABI: batches of independent events (ht_batch_*).
//
// The paper runs its events one after another (Sec. 4).  A batch keeps the
// vote matrices of up to max_events events resident and runs steps 1 and 2
// for all of them in one launch sequence -- hit binning, the fill (fused
// with the maxima tests when it fits), and the ordering of the peaks -- so
// that the per-launch costs are paid once per batch.  The kernels read the
// hit offsets from device memory, so a sequence captured in a CUDA graph for
// an event count serves every later run with that count: hits are copied to
// fixed staging buffers before the graph and the results out after it.
#include "ht_engine.h"

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace hte {
ht_status report(ht_status s, const std::string &msg);   // ht_api.cu
}

struct ht_batch {
    hte::Engine E;
    cudaStream_t stream = nullptr;
    uint32_t capacity = 0;           // peaks over the whole batch
    float *d_xyz = nullptr;          // staging: x | y | z, max_hits each
    float *h_xyz = nullptr;          // pinned
    uint32_t *d_off = nullptr;       // max_events + 1 hit offsets
    uint32_t *h_off = nullptr;       // pinned
    htk::Peak *d_out = nullptr;      // capacity peaks
    htk::Peak *h_out = nullptr;      // pinned
    uint32_t *d_counts = nullptr;    // max_events
    uint32_t *h_counts = nullptr;    // pinned: max_events counts + status
    cudaEvent_t done = nullptr;      // end of the last run (orders runs on different streams)
    bool done_pending = false;
    struct Graph {
        uint32_t n_events;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    bool graphs_ok = true;           // capture works on this device / driver
    bool poisoned = false;
};

namespace {

constexpr size_t kMaxGraphs = 8;

ht_status cuda_fail(ht_batch *b, cudaError_t e, const char *what)
{
    if (b)
        b->poisoned = true;
    char buf[320];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return hte::report(HT_E_CUDA, buf);
}

#define BK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return cuda_fail(b, e_, #call);                                                        \
    } while (0)

ht_status check_batch(ht_batch *b)
{
    if (!b)
        return hte::report(HT_E_INVAL, "batch is NULL");
    if (b->poisoned)
        return hte::report(HT_E_STATE, "batch is in an error state after an earlier CUDA failure");
    return HT_OK;
}

void drop_graphs(ht_batch *b)
{
    for (auto &g : b->graphs)
        cudaGraphExecDestroy(g.exec);
    b->graphs.clear();
}

// The kernels of one run, enqueued on st (also what a graph captures).
cudaError_t enqueue_compute(ht_batch *b, uint32_t n_events, cudaStream_t st)
{
    hte::Engine &E = b->E;
    const uint32_t mh = E.max_hits;
    // offsets clamped to the staging size; n_total = max_hits: nothing the
    // kernels take as arguments depends on the run
    cudaError_t e = hte::engine_fill(E, b->d_xyz, b->d_xyz + mh, b->d_xyz + 2 * (size_t)mh, b->d_off, mh, n_events,
                                     mh, 0u, st);
    if (e != cudaSuccess)
        return e;
    return hte::engine_scan(E, n_events, b->d_out, b->capacity, b->d_counts, st, true);
}

// Run the kernels: replay the graph for n_events, or run them directly and
// capture a graph for the next run with this count.
cudaError_t run_compute(ht_batch *b, uint32_t n_events, cudaStream_t st)
{
    if (b->E.prof.on || !b->graphs_ok)
        return enqueue_compute(b, n_events, st);
    for (auto &g : b->graphs)
        if (g.n_events == n_events)
            return cudaGraphLaunch(g.exec, st);
    cudaError_t e = enqueue_compute(b, n_events, st);
    if (e != cudaSuccess)
        return e;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t ec = enqueue_compute(b, n_events, st);
        e = cudaStreamEndCapture(st, &graph);
        if (ec != cudaSuccess)
            e = ec;
    }
    if (e == cudaSuccess)
        e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph)
        cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        // no graphs here: keep launching directly
        cudaGetLastError();
        b->graphs_ok = false;
        return cudaSuccess;
    }
    if (b->graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(b->graphs.front().exec);
        b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back({n_events, exec});
    return cudaSuccess;
}

// Status word of the last run; resets the counters when a kernel flagged a failure.
ht_status check_status(ht_batch *b, uint32_t s, cudaStream_t st)
{
    if (!s)
        return HT_OK;
    BK(cudaMemsetAsync(b->E.d_ctr, 0, hte::engine_ctr_words(b->E) * 4, st));
    b->E.ctr_dirty = false;
    b->E.fused_valid = false;
    BK(cudaStreamSynchronize(st));
    if (s & htk::ST_WAIT_TIMEOUT)
        return hte::report(HT_E_TIMEOUT, "a bounded device-side wait gave up (scan pipeline)");
    if (s & htk::ST_SCRATCH_OVERFLOW)
        return hte::report(HT_E_NOMEM, "peak scratch overflow");
    return hte::report(HT_E_CUDA, "kernel reported an invalid argument");
}

} // namespace

extern "C" {

ht_status ht_batch_create(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                          uint32_t max_events, uint32_t max_hits, uint32_t capacity, ht_batch **out)
{
    if (!out)
        return hte::report(HT_E_INVAL, "out is NULL");
    *out = nullptr;
    if (max_hits < 1 || capacity < 1)
        return hte::report(HT_E_INVAL, "max_hits and capacity must be >= 1");
    ht_batch *b = new (std::nothrow) ht_batch();
    if (!b)
        return hte::report(HT_E_NOMEM, "host allocation failed");
    std::string why;
    ht_status s = hte::engine_create(b->E, binning, ranges, threshold, max_events, max_hits, nullptr, &why);
    if (s != HT_OK) {
        delete b;
        return hte::report(s, why);
    }
    b->capacity = capacity;
    const size_t xyz = (size_t)max_hits * 12 + 64, off = ((size_t)max_events + 1) * 4;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_xyz, xyz)) != cudaSuccess || (e = cudaMallocHost(&b->h_xyz, xyz)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_off, off)) != cudaSuccess || (e = cudaMallocHost(&b->h_off, off)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_out, (size_t)capacity * sizeof(htk::Peak))) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_out, (size_t)capacity * sizeof(htk::Peak))) != cudaSuccess ||
        (e = cudaMalloc(&b->d_counts, (size_t)max_events * 4)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_counts, ((size_t)max_events + 1) * 4)) != cudaSuccess) {
        cudaGetLastError();
        ht_batch_destroy(b);
        return hte::report(HT_E_NOMEM, std::string("allocation failed: ") + cudaGetErrorString(e));
    }
    *out = b;
    return HT_OK;
}

ht_status ht_batch_destroy(ht_batch *b)
{
    if (!b)
        return HT_OK;
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    if (b->done_pending)
        cudaEventSynchronize(b->done);
    drop_graphs(b);
    hte::engine_destroy(b->E);
    cudaFree(b->d_xyz);
    cudaFree(b->d_off);
    cudaFree(b->d_out);
    cudaFree(b->d_counts);
    cudaFreeHost(b->h_xyz);
    cudaFreeHost(b->h_off);
    cudaFreeHost(b->h_out);
    cudaFreeHost(b->h_counts);
    if (b->done)
        cudaEventDestroy(b->done);
    if (b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
    return HT_OK;
}

ht_status ht_batch_run(ht_batch *b, const float *x, const float *y, const float *z, const uint32_t *hit_off,
                       uint32_t n_events, uint32_t n_hits, ht_peak *out, uint32_t *counts, uint32_t flags,
                       void *stream)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    hte::Engine &E = b->E;
    if (flags & ~(uint32_t)HT_MEM_DEVICE)
        return hte::report(HT_E_INVAL, "unknown flag (batches take HT_MEM_DEVICE only)");
    if (n_events < 1 || n_events > E.max_events)
        return hte::report(HT_E_INVAL, "need 1 <= n_events <= max_events");
    if (n_hits > E.max_hits)
        return hte::report(HT_E_INVAL, "more hits than max_hits");
    if (!hit_off || !out || !counts || (n_hits && (!x || !y || !z)))
        return hte::report(HT_E_INVAL, "NULL array");
    const bool dev = (flags & HT_MEM_DEVICE) != 0;
    if (!dev) {
        if (hit_off[0] != 0 || hit_off[n_events] != n_hits)
            return hte::report(HT_E_INVAL, "hit_off must start at 0 and end at n_hits");
        for (uint32_t e = 0; e < n_events; ++e)
            if (hit_off[e + 1] < hit_off[e])
                return hte::report(HT_E_INVAL, "hit_off must be non-decreasing");
    }
    cudaStream_t st = stream ? (cudaStream_t)stream : b->stream;
    if (b->done_pending)
        BK(cudaStreamWaitEvent(st, b->done, 0));   // the staging of the last run is free

    // ---- hits in ---------------------------------------------------------
    const size_t mh = E.max_hits, bytes = (size_t)n_hits * 4, off_bytes = ((size_t)n_events + 1) * 4;
    if (!dev) {
        if (b->done_pending)
            BK(cudaEventSynchronize(b->done));      // pinned staging no longer read
        std::memcpy(b->h_xyz, x, bytes);
        std::memcpy(b->h_xyz + mh, y, bytes);
        std::memcpy(b->h_xyz + 2 * mh, z, bytes);
        std::memcpy(b->h_off, hit_off, off_bytes);
    }
    const cudaMemcpyKind kin = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const float *sx = dev ? x : b->h_xyz, *sy = dev ? y : b->h_xyz + mh, *sz = dev ? z : b->h_xyz + 2 * mh;
    if (n_hits) {
        BK(cudaMemcpyAsync(b->d_xyz, sx, bytes, kin, st));
        BK(cudaMemcpyAsync(b->d_xyz + mh, sy, bytes, kin, st));
        BK(cudaMemcpyAsync(b->d_xyz + 2 * mh, sz, bytes, kin, st));
    }
    BK(cudaMemcpyAsync(b->d_off, dev ? hit_off : b->h_off, off_bytes, kin, st));

    // ---- steps 1 + 2 -----------------------------------------------------
    BK(run_compute(b, n_events, st));
    E.last_hit_off = b->d_off;        // what a later autotune re-times (also after a replay)
    E.last_n_hits0 = (uint32_t)mh;
    E.last_n_events = n_events;
    E.last_accumulate = false;

    // ---- results out -----------------------------------------------------
    if (dev) {
        BK(cudaMemcpyAsync(counts, b->d_counts, (size_t)n_events * 4, cudaMemcpyDeviceToDevice, st));
        BK(cudaMemcpyAsync(out, b->d_out, (size_t)b->capacity * sizeof(htk::Peak), cudaMemcpyDeviceToDevice, st));
        BK(cudaEventRecord(b->done, st));
        b->done_pending = true;
        return HT_OK;
    }
    BK(cudaMemcpyAsync(b->h_counts, b->d_counts, (size_t)n_events * 4, cudaMemcpyDeviceToHost, st));
    BK(cudaMemcpyAsync(b->h_counts + E.max_events, hte::engine_status(E), 4, cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    b->done_pending = false;
    if ((s = check_status(b, b->h_counts[E.max_events], st)) != HT_OK)
        return s;
    uint64_t total = 0;
    for (uint32_t e = 0; e < n_events; ++e)
        total += b->h_counts[e];
    const uint32_t k = (uint32_t)(total < b->capacity ? total : b->capacity);
    if (k) {
        BK(cudaMemcpyAsync(b->h_out, b->d_out, (size_t)k * sizeof(htk::Peak), cudaMemcpyDeviceToHost, st));
        BK(cudaStreamSynchronize(st));
        std::memcpy(out, b->h_out, (size_t)k * sizeof(htk::Peak));
    }
    std::memcpy(counts, b->h_counts, (size_t)n_events * 4);
    return total > b->capacity ? HT_TRUNCATED : HT_OK;
}

ht_status ht_batch_sync(ht_batch *b, void *stream)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    cudaStream_t st = stream ? (cudaStream_t)stream : b->stream;
    if (b->done_pending)
        BK(cudaStreamWaitEvent(st, b->done, 0));
    BK(cudaMemcpyAsync(b->h_counts + b->E.max_events, hte::engine_status(b->E), 4, cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    b->done_pending = false;
    return check_status(b, b->h_counts[b->E.max_events], st);
}

ht_status ht_batch_copy_matrix(ht_batch *b, uint32_t event, uint32_t *dst, uint64_t n_cells)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    if (!dst || n_cells != b->E.n_cells || event >= b->E.max_events)
        return hte::report(HT_E_INVAL, "dst, n_cells (one event's matrix) or event out of range");
    if (b->done_pending)
        BK(cudaEventSynchronize(b->done));
    BK(cudaStreamSynchronize(b->stream));
    BK(cudaMemcpy(dst, b->E.d_M + (size_t)event * b->E.n_cells, n_cells * 4, cudaMemcpyDeviceToHost));
    return HT_OK;
}

ht_status ht_batch_set_tuning(ht_batch *b, const ht_tuning *t)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    if (!t)
        return hte::report(HT_E_INVAL, "tuning is NULL");
    BK(cudaStreamSynchronize(b->stream));
    if (b->done_pending)
        BK(cudaEventSynchronize(b->done));
    drop_graphs(b);
    std::string why;
    s = hte::engine_set_tuning(b->E, *t, &b->poisoned, &why);
    return s == HT_OK ? HT_OK : hte::report(s, why);
}

ht_status ht_batch_get_tuning(ht_batch *b, ht_tuning *t)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    if (!t)
        return hte::report(HT_E_INVAL, "tuning is NULL");
    hte::engine_get_tuning(b->E, t);
    return HT_OK;
}

ht_status ht_batch_autotune(ht_batch *b, uint32_t reps, ht_tuning *chosen, double *us_per_event)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    if (b->done_pending)
        BK(cudaEventSynchronize(b->done));
    drop_graphs(b);
    std::string why;
    s = hte::engine_autotune(b->E, reps, b->stream, us_per_event, &why);
    if (s == HT_E_CUDA)
        b->poisoned = true;
    if (s != HT_OK)
        return hte::report(s, why);
    if (chosen)
        hte::engine_get_tuning(b->E, chosen);
    return HT_OK;
}

ht_status ht_batch_profile(ht_batch *b, int enable)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    BK(hte::prof_enable(b->E, enable != 0));
    return HT_OK;
}

ht_status ht_batch_profile_read(ht_batch *b, ht_kernel_time *out, uint32_t cap, uint32_t *n)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    if (!n || (cap && !out))
        return hte::report(HT_E_INVAL, "NULL argument");
    BK(hte::prof_read(b->E, out, cap, n));
    return HT_OK;
}

} // extern "C"
