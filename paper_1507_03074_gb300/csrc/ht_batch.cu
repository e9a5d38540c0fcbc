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
#include "ht_runner.h"
#include "ht_trace.h"

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace hte {
ht_status report(ht_status s, const std::string &msg);   // ht_api.cu
}

struct ht_batch {
    hte::Runner R;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;      // end of the last run (orders runs on different streams)
    bool done_pending = false;
    bool poisoned = false;
};

namespace hte {

static constexpr size_t kMaxGraphs = 8;

ht_status runner_create(Runner &R, const ht_binning *b, const ht_ranges *r, uint32_t threshold, uint32_t max_events,
                        uint32_t max_hits, uint32_t capacity, std::string *why)
{
    if (max_hits < 1 || capacity < 1) {
        *why = "max_hits and capacity must be >= 1";
        return HT_E_INVAL;
    }
    ht_status s = engine_create(R.E, b, r, threshold, max_events, max_hits, nullptr, why);
    if (s != HT_OK)
        return s;
    R.capacity = capacity;
    const size_t xyz = (size_t)max_hits * 12 + 64, off = ((size_t)max_events + 1) * 4;
    const size_t out_b = (size_t)capacity * sizeof(htk::Peak), cnt_b = ((size_t)max_events + 1) * 4;
    cudaError_t e;
    if ((e = cudaMalloc(&R.d_xyz, xyz)) != cudaSuccess || (e = cudaMallocHost(&R.h_xyz, xyz)) != cudaSuccess ||
        (e = cudaMalloc(&R.d_off, off)) != cudaSuccess || (e = cudaMallocHost(&R.h_off, off)) != cudaSuccess ||
        (e = cudaMalloc(&R.d_out, out_b)) != cudaSuccess || (e = cudaMalloc(&R.d_counts, cnt_b)) != cudaSuccess ||
        (e = cudaHostAlloc(&R.h_out, out_b, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostAlloc(&R.h_counts, cnt_b, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer((void **)&R.h_out_dev, R.h_out, 0)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer((void **)&R.h_counts_dev, R.h_counts, 0)) != cudaSuccess) {
        cudaGetLastError();
        runner_destroy(R);
        *why = std::string("allocation failed: ") + cudaGetErrorString(e);
        return HT_E_NOMEM;
    }
    return HT_OK;
}

void runner_drop_graphs(Runner &R)
{
    for (auto &g : R.graphs)
        cudaGraphExecDestroy(g.exec);
    R.graphs.clear();
}

void runner_destroy(Runner &R)
{
    runner_drop_graphs(R);
    engine_destroy(R.E);
    cudaFree(R.d_xyz);
    cudaFree(R.d_off);
    cudaFree(R.d_out);
    cudaFree(R.d_counts);
    cudaFreeHost(R.h_xyz);
    cudaFreeHost(R.h_off);
    cudaFreeHost(R.h_out);
    cudaFreeHost(R.h_counts);
    R.d_xyz = R.h_xyz = nullptr;
    R.d_off = R.h_off = R.d_counts = R.h_counts = R.h_counts_dev = nullptr;
    R.d_out = R.h_out = R.h_out_dev = nullptr;
}

// The kernels of one run (also what a graph captures).
static cudaError_t enqueue_compute(Runner &R, uint32_t n_events, bool to_host, uint32_t fill_flags, cudaStream_t st)
{
    Engine &E = R.E;
    const uint32_t mh = E.max_hits;
    // offsets clamped to the staging size; n_total = max_hits: nothing the
    // kernels take as arguments depends on the run
    cudaError_t e = engine_fill(E, R.d_xyz, R.d_xyz + mh, R.d_xyz + 2 * (size_t)mh, R.d_off, mh, n_events, mh,
                                fill_flags, st);
    if (e != cudaSuccess)
        return e;
    return engine_scan(E, n_events, to_host ? R.h_out_dev : R.d_out, R.capacity, to_host ? R.h_counts_dev : R.d_counts,
                       st, true);
}

// Replay the graph for (n_events, to_host), or run directly and capture one
// for the next run with that shape.
static cudaError_t run_compute(Runner &R, uint32_t n_events, bool to_host, uint32_t fill_flags, cudaStream_t st)
{
    if (R.E.prof.on || !R.graphs_ok)
        return enqueue_compute(R, n_events, to_host, fill_flags, st);
    for (auto &g : R.graphs)
        if (g.n_events == n_events && g.to_host == to_host && g.fill_flags == fill_flags)
            return cudaGraphLaunch(g.exec, st);
    cudaError_t e = enqueue_compute(R, n_events, to_host, fill_flags, st);
    if (e != cudaSuccess)
        return e;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const cudaError_t ec = enqueue_compute(R, n_events, to_host, fill_flags, st);
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
        R.graphs_ok = false;
        return cudaSuccess;
    }
    if (R.graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(R.graphs.front().exec);
        R.graphs.erase(R.graphs.begin());
    }
    R.graphs.push_back({n_events, to_host, fill_flags, exec});
    return cudaSuccess;
}

cudaError_t runner_enqueue(Runner &R, uint32_t n_events, uint32_t n_hits, bool host_in, bool to_host,
                           cudaStream_t st, uint32_t fill_flags)
{
    Engine &E = R.E;
    const size_t mh = E.max_hits, bytes = (size_t)n_hits * 4;
    cudaError_t e;
    if (host_in) {
        if (n_hits && ((e = cudaMemcpyAsync(R.d_xyz, R.h_xyz, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                       (e = cudaMemcpyAsync(R.d_xyz + mh, R.h_xyz + mh, bytes, cudaMemcpyHostToDevice, st)) !=
                           cudaSuccess ||
                       (e = cudaMemcpyAsync(R.d_xyz + 2 * mh, R.h_xyz + 2 * mh, bytes, cudaMemcpyHostToDevice, st)) !=
                           cudaSuccess))
            return e;
        if ((e = cudaMemcpyAsync(R.d_off, R.h_off, ((size_t)n_events + 1) * 4, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
            return e;
    }
    if ((e = run_compute(R, n_events, to_host, fill_flags, st)) != cudaSuccess)
        return e;
    E.last_hit_off = R.d_off;         // what a later autotune re-times (also after a replay)
    E.last_n_hits0 = (uint32_t)mh;
    E.last_n_events = n_events;
    E.last_accumulate = false;
    if (to_host)
        return cudaMemcpyAsync(R.h_counts + E.max_events, engine_status(E), 4, cudaMemcpyDeviceToHost, st);
    return cudaSuccess;
}

ht_status runner_status(Runner &R, uint32_t status, cudaStream_t st, std::string *why)
{
    if (!status)
        return HT_OK;
    cudaError_t e = cudaMemsetAsync(R.E.d_ctr, 0, engine_ctr_words(R.E) * 4, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    R.E.ctr_dirty = false;
    R.E.fused_valid = false;
    if (e != cudaSuccess) {
        *why = std::string("counter reset failed: ") + cudaGetErrorString(e);
        return HT_E_CUDA;
    }
    if (status & htk::ST_WAIT_TIMEOUT) {
        *why = "a bounded device-side wait gave up (scan pipeline)";
        return HT_E_TIMEOUT;
    }
    if (status & htk::ST_SCRATCH_OVERFLOW) {
        *why = "peak scratch overflow";
        return HT_E_NOMEM;
    }
    *why = "kernel reported an invalid argument";
    return HT_E_CUDA;
}

} // namespace hte

namespace {

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

ht_status status_of(ht_batch *b, uint32_t status, cudaStream_t st)
{
    std::string why;
    ht_status s = hte::runner_status(b->R, status, st, &why);
    if (s == HT_E_CUDA)
        b->poisoned = true;
    return s == HT_OK ? HT_OK : hte::report(s, why);
}

} // namespace

extern "C" {

ht_status ht_batch_create(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                          uint32_t max_events, uint32_t max_hits, uint32_t capacity, ht_batch **out)
{
    if (!out)
        return hte::report(HT_E_INVAL, "out is NULL");
    *out = nullptr;
    ht_batch *b = new (std::nothrow) ht_batch();
    if (!b)
        return hte::report(HT_E_NOMEM, "host allocation failed");
    std::string why;
    ht_status s = hte::runner_create(b->R, binning, ranges, threshold, max_events, max_hits, capacity, &why);
    if (s != HT_OK) {
        delete b;
        return hte::report(s, why);
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess) {
        cudaGetLastError();
        ht_batch_destroy(b);
        return hte::report(HT_E_NOMEM, std::string("stream / event creation failed: ") + cudaGetErrorString(e));
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
    hte::runner_destroy(b->R);
    if (b->done)
        cudaEventDestroy(b->done);
    if (b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
    return HT_OK;
}

// Host memory the GPU can copy from directly (cudaHostAlloc'd or registered).
static bool page_locked(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

ht_status ht_batch_run(ht_batch *b, const float *x, const float *y, const float *z, const uint32_t *hit_off,
                       uint32_t n_events, uint32_t n_hits, ht_peak *out, uint32_t *counts, uint32_t flags,
                       void *stream)
{
    hte::TraceRange tr("ht_batch_run");
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    hte::Runner &R = b->R;
    hte::Engine &E = R.E;
    if (flags & ~(uint32_t)(HT_MEM_DEVICE | HT_PEAKS_ONLY | HT_FILL_NAIVE))
        return hte::report(HT_E_INVAL, "unknown flag (batches take HT_MEM_DEVICE, HT_PEAKS_ONLY and HT_FILL_NAIVE)");
    if ((flags & HT_PEAKS_ONLY) && (flags & HT_FILL_NAIVE))
        return hte::report(HT_E_INVAL, "HT_PEAKS_ONLY does not combine with HT_FILL_NAIVE");
    const bool po = (flags & HT_PEAKS_ONLY) != 0;
    const uint32_t fill_flags = flags & (uint32_t)(HT_PEAKS_ONLY | HT_FILL_NAIVE);
    if (po) {
        std::string why;
        s = hte::engine_ensure_edges(E, &why);
        if (s != HT_OK) {
            if (s == HT_E_CUDA)
                b->poisoned = true;
            return hte::report(s, why);
        }
    }
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
    const size_t mh = E.max_hits, bytes = (size_t)n_hits * 4, off_bytes = ((size_t)n_events + 1) * 4;

    if (dev) {
        // device inputs into the fixed staging, results out of the device buffers
        if (n_hits) {
            BK(cudaMemcpyAsync(R.d_xyz, x, bytes, cudaMemcpyDeviceToDevice, st));
            BK(cudaMemcpyAsync(R.d_xyz + mh, y, bytes, cudaMemcpyDeviceToDevice, st));
            BK(cudaMemcpyAsync(R.d_xyz + 2 * mh, z, bytes, cudaMemcpyDeviceToDevice, st));
        }
        BK(cudaMemcpyAsync(R.d_off, hit_off, off_bytes, cudaMemcpyDeviceToDevice, st));
        BK(hte::runner_enqueue(R, n_events, n_hits, false, false, st, fill_flags));
        BK(cudaMemcpyAsync(counts, R.d_counts, (size_t)n_events * 4, cudaMemcpyDeviceToDevice, st));
        BK(cudaMemcpyAsync(out, R.d_out, (size_t)R.capacity * sizeof(htk::Peak), cudaMemcpyDeviceToDevice, st));
        BK(cudaEventRecord(b->done, st));
        b->done_pending = true;
        return HT_OK;
    }
    // host inputs through the pinned staging (page-locked inputs straight to
    // the device: the call returns only once the run is done, so the caller
    // may reuse them on return either way); the order kernel writes the
    // peaks and counts into mapped pinned memory
    if (b->done_pending)
        BK(cudaEventSynchronize(b->done));
    b->done_pending = false;
    std::memcpy(R.h_off, hit_off, off_bytes);
    if (n_hits && page_locked(x) && page_locked(y) && page_locked(z)) {
        BK(cudaMemcpyAsync(R.d_xyz, x, bytes, cudaMemcpyHostToDevice, st));
        BK(cudaMemcpyAsync(R.d_xyz + mh, y, bytes, cudaMemcpyHostToDevice, st));
        BK(cudaMemcpyAsync(R.d_xyz + 2 * mh, z, bytes, cudaMemcpyHostToDevice, st));
        BK(cudaMemcpyAsync(R.d_off, R.h_off, off_bytes, cudaMemcpyHostToDevice, st));
        BK(hte::runner_enqueue(R, n_events, n_hits, false, true, st, fill_flags));
    } else {
        if (n_hits) {
            std::memcpy(R.h_xyz, x, bytes);
            std::memcpy(R.h_xyz + mh, y, bytes);
            std::memcpy(R.h_xyz + 2 * mh, z, bytes);
        }
        BK(hte::runner_enqueue(R, n_events, n_hits, true, true, st, fill_flags));
    }
    BK(cudaStreamSynchronize(st));
    if ((s = status_of(b, R.h_counts[E.max_events], st)) != HT_OK)
        return s;
    uint64_t total = 0;
    for (uint32_t e = 0; e < n_events; ++e)
        total += R.h_counts[e];
    const uint32_t k = (uint32_t)(total < R.capacity ? total : R.capacity);
    std::memcpy(out, R.h_out, (size_t)k * sizeof(htk::Peak));
    std::memcpy(counts, R.h_counts, (size_t)n_events * 4);
    return total > R.capacity ? HT_TRUNCATED : HT_OK;
}

ht_status ht_batch_sync(ht_batch *b, void *stream)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    cudaStream_t st = stream ? (cudaStream_t)stream : b->stream;
    if (b->done_pending)
        BK(cudaStreamWaitEvent(st, b->done, 0));
    hte::Runner &R = b->R;
    BK(cudaMemcpyAsync(R.h_counts + R.E.max_events, hte::engine_status(R.E), 4, cudaMemcpyDeviceToHost, st));
    BK(cudaStreamSynchronize(st));
    b->done_pending = false;
    return status_of(b, R.h_counts[R.E.max_events], st);
}

ht_status ht_batch_copy_matrix(ht_batch *b, uint32_t event, uint32_t *dst, uint64_t n_cells)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    const hte::Engine &E = b->R.E;
    if (!dst || n_cells != E.n_cells || event >= E.max_events)
        return hte::report(HT_E_INVAL, "dst, n_cells (one event's matrix) or event out of range");
    if (b->done_pending)
        BK(cudaEventSynchronize(b->done));
    BK(cudaStreamSynchronize(b->stream));
    BK(cudaMemcpy(dst, E.d_M + (size_t)event * E.n_cells, n_cells * 4, cudaMemcpyDeviceToHost));
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
    hte::runner_drop_graphs(b->R);
    std::string why;
    s = hte::engine_set_tuning(b->R.E, *t, &b->poisoned, &why);
    return s == HT_OK ? HT_OK : hte::report(s, why);
}

ht_status ht_batch_get_tuning(ht_batch *b, ht_tuning *t)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    if (!t)
        return hte::report(HT_E_INVAL, "tuning is NULL");
    hte::engine_get_tuning(b->R.E, t);
    return HT_OK;
}

ht_status ht_batch_autotune(ht_batch *b, uint32_t reps, ht_tuning *chosen, double *us_per_event)
{
    hte::TraceRange tr("ht_batch_autotune");
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    if (b->done_pending)
        BK(cudaEventSynchronize(b->done));
    hte::runner_drop_graphs(b->R);
    std::string why;
    s = hte::engine_autotune(b->R.E, reps, b->stream, us_per_event, &why);
    if (s == HT_E_CUDA)
        b->poisoned = true;
    if (s != HT_OK)
        return hte::report(s, why);
    if (chosen)
        hte::engine_get_tuning(b->R.E, chosen);
    return HT_OK;
}

ht_status ht_batch_profile(ht_batch *b, int enable)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    BK(hte::prof_enable(b->R.E, enable != 0));
    return HT_OK;
}

ht_status ht_batch_profile_read(ht_batch *b, ht_kernel_time *out, uint32_t cap, uint32_t *n)
{
    ht_status s = check_batch(b);
    if (s != HT_OK)
        return s;
    if (!n || (cap && !out))
        return hte::report(HT_E_INVAL, "NULL argument");
    BK(hte::prof_read(b->R.E, out, cap, n));
    return HT_OK;
}

} // extern "C"
