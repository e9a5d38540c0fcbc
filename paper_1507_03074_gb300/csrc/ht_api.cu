// C ABI: single-event context (ht_create / ht_fill / ht_find_maxima ...).
//
// Sec. 3 allocates M_H once and re-initialises it for every event; here the
// context keeps M_H, the sorted-hit workspace and the peak scratch resident
// on the device, and pinned host staging for host-side hits and results.
#include "ht_engine.h"
#include "ht_geom.h"
#include "ht_trace.h"

#include <cstdio>
#include <cstring>
#include <string>

namespace {

thread_local std::string g_last_error = "no error";

ht_status set_err(ht_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

} // namespace


struct ht_ctx {
    hte::Engine E;
    cudaStream_t stream = nullptr;
    float *d_in = nullptr;        // 3 * max_hits device staging
    float *h_in = nullptr;        // 3 * max_hits pinned staging
    uint32_t *h_small = nullptr;  // mapped pinned: [0] count (written by the order kernel), [1] status
    uint32_t *h_small_dev = nullptr;  // its device address
    uint32_t *d_small = nullptr;  // device: [2] the 4-D scan's 2-D count
    htk::Peak *h_peaks = nullptr;     // mapped pinned peaks of host-mode ht_find_maxima
    htk::Peak *h_peaks_dev = nullptr; // their device address
    uint32_t peaks_cap = 0;
    cudaEvent_t ev_in = nullptr;
    bool ev_in_pending = false;
    uint32_t acc_hits = 0;
    bool last_peaks_only = false;  // the last fill left M_H as it was
    htk::Peak *d_p2 = nullptr;     // the 2-D peak list of 4-D scans (E.scan.entries_cap entries)
    uint8_t *d_keep = nullptr;     // and its keep flags
    uint32_t p2_cap = 0;
    bool poisoned = false;
};

namespace hte {
// Shared with the batch, server and sector objects.
ht_status report(ht_status s, const std::string &msg) { return set_err(s, msg); }
Engine &ctx_engine(ht_ctx *c) { return c->E; }
} // namespace hte

static ht_status cuda_fail(ht_ctx *c, cudaError_t e, const char *what)
{
    if (c)
        c->poisoned = true;
    char buf[320];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return set_err(HT_E_CUDA, buf);
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return cuda_fail(ctx, e_, #call);                                                      \
    } while (0)

static ht_status check_ctx(ht_ctx *ctx)
{
    if (!ctx)
        return set_err(HT_E_INVAL, "context is NULL");
    if (ctx->poisoned)
        return set_err(HT_E_STATE, "context failed earlier (HT_E_CUDA); destroy it");
    return HT_OK;
}

// Read and clear the device status word; map its bits to a status.
static ht_status read_status(ht_ctx *ctx, cudaStream_t st)
{
    uint32_t *d_status = hte::engine_status(ctx->E);
    CK(cudaMemcpyAsync(ctx->h_small + 1, d_status, 4, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const uint32_t s = ctx->h_small[1];
    if (!s)
        return HT_OK;
    // reset the status and every counter the kernels may have left behind
    CK(cudaMemsetAsync(ctx->E.d_ctr, 0, hte::engine_ctr_words(ctx->E) * 4, st));
    ctx->E.ctr_dirty = false;
    ctx->E.fused_valid = false;
    CK(cudaStreamSynchronize(st));
    if (s & htk::ST_WAIT_TIMEOUT)
        return set_err(HT_E_TIMEOUT, "a bounded device-side wait gave up (scan pipeline)");
    if (s & htk::ST_SCRATCH_OVERFLOW)
        return set_err(HT_E_NOMEM, "peak scratch overflow");
    return set_err(HT_E_CUDA, "kernel reported an invalid argument");
}

extern "C" {

const char *ht_last_error(void) { return g_last_error.c_str(); }

ht_status ht_create(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                    uint32_t max_hits, ht_ctx **out)
{
    if (!out)
        return set_err(HT_E_INVAL, "out is NULL");
    *out = nullptr;
    if (max_hits < 1)
        return set_err(HT_E_INVAL, "max_hits must be >= 1");
    ht_ctx *ctx = new (std::nothrow) ht_ctx();
    if (!ctx)
        return set_err(HT_E_NOMEM, "host allocation failed");
    std::string why;
    ht_status s = hte::engine_create(ctx->E, binning, ranges, threshold, 1, max_hits, nullptr, &why);
    if (s != HT_OK) {
        delete ctx;
        return set_err(s, why);
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMalloc(&ctx->d_in, (size_t)max_hits * 12 + 64)) != cudaSuccess ||
        (e = cudaMalloc(&ctx->d_small, 16)) != cudaSuccess ||
        (e = cudaMallocHost(&ctx->h_in, (size_t)max_hits * 12 + 64)) != cudaSuccess ||
        (e = cudaHostAlloc(&ctx->h_small, 16, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer((void **)&ctx->h_small_dev, ctx->h_small, 0)) != cudaSuccess) {
        cudaGetLastError();
        ht_destroy(ctx);
        return set_err(HT_E_NOMEM, std::string("allocation failed: ") + cudaGetErrorString(e));
    }
    *out = ctx;
    return HT_OK;
}

ht_status ht_destroy(ht_ctx *ctx)
{
    if (!ctx)
        return HT_OK;
    if (ctx->stream)
        cudaStreamSynchronize(ctx->stream);
    hte::engine_destroy(ctx->E);
    cudaFree(ctx->d_in);
    cudaFree(ctx->d_small);
    cudaFreeHost(ctx->h_peaks);
    cudaFree(ctx->d_p2);
    cudaFree(ctx->d_keep);
    cudaFreeHost(ctx->h_in);
    cudaFreeHost(ctx->h_small);
    if (ctx->ev_in)
        cudaEventDestroy(ctx->ev_in);
    if (ctx->stream)
        cudaStreamDestroy(ctx->stream);
    delete ctx;
    return HT_OK;
}

ht_status ht_fill(ht_ctx *ctx, const float *x, const float *y, const float *z, uint32_t n_hits,
                  uint32_t flags, void *stream)
{
    hte::TraceRange tr("ht_fill");
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    if (flags & ~(uint32_t)(HT_MEM_DEVICE | HT_ACCUMULATE | HT_FILL_NAIVE | HT_PEAKS_ONLY))
        return set_err(HT_E_INVAL, "unknown flag");
    if ((flags & HT_PEAKS_ONLY) && (flags & (HT_ACCUMULATE | HT_FILL_NAIVE)))
        return set_err(HT_E_INVAL, "HT_PEAKS_ONLY does not combine with HT_ACCUMULATE or HT_FILL_NAIVE");
    if (flags & HT_PEAKS_ONLY) {
        std::string why;
        s = hte::engine_ensure_edges(ctx->E, &why);
        if (s != HT_OK) {
            if (s == HT_E_CUDA)
                ctx->poisoned = true;
            return set_err(s, why);
        }
    }
    if (n_hits && (!x || !y || !z))
        return set_err(HT_E_INVAL, "hit arrays must not be NULL");
    const bool accumulate = (flags & HT_ACCUMULATE) != 0;
    const uint64_t acc = (accumulate ? (uint64_t)ctx->acc_hits : 0ull) + n_hits;
    if (acc > ctx->E.max_hits)
        return set_err(HT_E_INVAL, "more hits than max_hits (accumulated fills count together)");
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;

    const float *px = x, *py = y, *pz = z;
    if (!(flags & HT_MEM_DEVICE) && n_hits) {
        if (ctx->ev_in_pending)
            CK(cudaEventSynchronize(ctx->ev_in));       // staging free again
        const size_t bytes = (size_t)n_hits * 4;
        std::memcpy(ctx->h_in, x, bytes);
        std::memcpy(ctx->h_in + n_hits, y, bytes);
        std::memcpy(ctx->h_in + 2 * (size_t)n_hits, z, bytes);
        CK(cudaMemcpyAsync(ctx->d_in, ctx->h_in, 3 * bytes, cudaMemcpyHostToDevice, st));
        CK(cudaEventRecord(ctx->ev_in, st));
        ctx->ev_in_pending = true;
        px = ctx->d_in;
        py = ctx->d_in + n_hits;
        pz = ctx->d_in + 2 * (size_t)n_hits;
    }
    CK(hte::engine_fill(ctx->E, px, py, pz, nullptr, n_hits, 1, n_hits, flags & ~(uint32_t)HT_MEM_DEVICE, st));
    ctx->acc_hits = (uint32_t)acc;
    ctx->last_peaks_only = (flags & HT_PEAKS_ONLY) != 0;
    return HT_OK;
}

ht_status ht_find_maxima(ht_ctx *ctx, ht_peak *out, uint32_t capacity, uint32_t *n_found,
                         uint32_t flags, void *stream)
{
    hte::TraceRange tr("ht_find_maxima");
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    if (flags & ~(uint32_t)(HT_MEM_DEVICE | HT_MAXIMA_4D))
        return set_err(HT_E_INVAL, "unknown flag");
    if (!n_found || (capacity && !out))
        return set_err(HT_E_INVAL, "out (capacity > 0) and n_found must not be NULL");
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    const bool four = (flags & HT_MAXIMA_4D) != 0;
    if (four) {
        if (ctx->last_peaks_only)
            return set_err(HT_E_INVAL, "HT_MAXIMA_4D reads M_H, which a peaks-only fill does not write");
        if (ctx->p2_cap < ctx->E.scan.entries_cap) {
            CK(cudaStreamSynchronize(st));
            cudaFree(ctx->d_p2);
            cudaFree(ctx->d_keep);
            ctx->d_p2 = nullptr;
            ctx->d_keep = nullptr;
            ctx->p2_cap = 0;
            CK(cudaMalloc(&ctx->d_p2, (size_t)ctx->E.scan.entries_cap * sizeof(htk::Peak)));
            CK(cudaMalloc(&ctx->d_keep, (size_t)ctx->E.scan.entries_cap));
            ctx->p2_cap = ctx->E.scan.entries_cap;
        }
    }
    // the 2-D list's total goes to d_small[2] (h_small[0] receives the result's)
    auto scan = [&](htk::Peak *dst, uint32_t cap, uint32_t *cnt) {
        return four ? hte::engine_scan4d(ctx->E, ctx->d_p2, ctx->d_keep, ctx->p2_cap, ctx->d_small + 2, dst, cap, cnt,
                                         st)
                    : hte::engine_scan(ctx->E, 1, dst, cap, cnt, st);
    };
    if (flags & HT_MEM_DEVICE) {
        CK(scan(reinterpret_cast<htk::Peak *>(out), capacity, n_found));
        return HT_OK;
    }
    if (capacity > ctx->peaks_cap) {
        CK(cudaStreamSynchronize(st));
        cudaFreeHost(ctx->h_peaks);
        ctx->h_peaks = ctx->h_peaks_dev = nullptr;
        ctx->peaks_cap = 0;
        CK(cudaHostAlloc(&ctx->h_peaks, (size_t)capacity * sizeof(htk::Peak), cudaHostAllocMapped));
        CK(cudaHostGetDevicePointer((void **)&ctx->h_peaks_dev, ctx->h_peaks, 0));
        ctx->peaks_cap = capacity;
    }
    // the order kernel writes the peaks and their count into mapped pinned
    // memory: one wait, then a host copy
    CK(scan(ctx->h_peaks_dev, capacity, ctx->h_small_dev));
    s = read_status(ctx, st);   // synchronises the stream
    if (s != HT_OK)
        return s;
    const uint32_t n = ctx->h_small[0];
    const uint32_t k = n < capacity ? n : capacity;
    if (k)
        std::memcpy(out, ctx->h_peaks, (size_t)k * sizeof(ht_peak));
    *n_found = n;
    return n > capacity ? HT_TRUNCATED : HT_OK;
}

ht_status ht_sync(ht_ctx *ctx, void *stream)
{
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    return read_status(ctx, st);
}

ht_status ht_measure_atomics(uint64_t footprint_bytes, uint32_t updates_per_thread, double *updates_per_s)
{
    if (!updates_per_s || footprint_bytes < 4096 || footprint_bytes > (1ull << 34) ||
        (footprint_bytes & (footprint_bytes - 1)) || updates_per_thread < 1 || updates_per_thread > 4096)
        return set_err(HT_E_INVAL, "footprint_bytes: a power of two in 4 KiB .. 16 GiB; updates_per_thread 1 .. 4096");
    int dev = 0, sms = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return set_err(HT_E_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
    uint32_t *buf = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    const uint32_t grid = (uint32_t)sms * 8u;
    const uint32_t mask = (uint32_t)(footprint_bytes / 4 - 1);
    float ms = 0.f;
    if ((e = cudaMalloc(&buf, footprint_bytes)) == cudaSuccess &&
        (e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) == cudaSuccess &&
        (e = cudaEventCreate(&a)) == cudaSuccess && (e = cudaEventCreate(&b)) == cudaSuccess &&
        (e = cudaMemsetAsync(buf, 0, footprint_bytes, st)) == cudaSuccess &&
        (e = htk::launch_atomic_rate(buf, mask, updates_per_thread, 1u, grid, st)) == cudaSuccess &&   // warm-up
        (e = cudaEventRecord(a, st)) == cudaSuccess &&
        (e = htk::launch_atomic_rate(buf, mask, updates_per_thread, 2u, grid, st)) == cudaSuccess &&
        (e = cudaEventRecord(b, st)) == cudaSuccess && (e = cudaEventSynchronize(b)) == cudaSuccess)
        e = cudaEventElapsedTime(&ms, a, b);
    if (st)
        cudaStreamSynchronize(st);
    cudaFree(buf);
    if (a)
        cudaEventDestroy(a);
    if (b)
        cudaEventDestroy(b);
    if (st)
        cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(e == cudaErrorMemoryAllocation ? HT_E_NOMEM : HT_E_CUDA,
                       std::string("atomic rate measurement: ") + cudaGetErrorString(e));
    }
    *updates_per_s = (double)grid * 256.0 * updates_per_thread / (ms * 1e-3);
    return HT_OK;
}

ht_status ht_check_wait_timeout(ht_ctx *ctx, uint32_t limit_ms)
{
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    if (limit_ms < 1 || limit_ms > 1000)
        return set_err(HT_E_INVAL, "limit_ms must be 1 .. 1000");
    CK(htk::launch_wait_probe(hte::engine_status(ctx->E), limit_ms, ctx->stream));
    return read_status(ctx, ctx->stream);   // HT_E_TIMEOUT, counters reset
}

ht_status ht_last_admitted(ht_ctx *ctx, uint64_t *records)
{
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    if (!records)
        return set_err(HT_E_INVAL, "records must not be NULL");
    if (!ctx->E.last_n_events) {
        *records = 0;
        return HT_OK;
    }
    // the unit lists' total length: the last offset of the last fill's units
    const uint64_t units = (uint64_t)ctx->E.last_n_events * ctx->E.geom.n_slices;
    const size_t max_units = (size_t)ctx->E.max_events * ctx->E.geom.n_slices;
    const uint32_t *d_off = ctx->E.d_slice + 2 * max_units;
    CK(cudaDeviceSynchronize());   // the fill may have run on any stream
    CK(cudaMemcpy(ctx->h_small + 2, d_off + units, 4, cudaMemcpyDeviceToHost));
    *records = ctx->h_small[2];
    return HT_OK;
}

ht_status ht_copy_matrix(ht_ctx *ctx, uint32_t *dst, uint64_t n_cells, uint32_t flags, void *stream)
{
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    if (!dst || n_cells != ctx->E.n_cells)
        return set_err(HT_E_INVAL, "dst must hold exactly n_theta*n_phi*n_a*n_b cells");
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    const cudaMemcpyKind kind = (flags & HT_MEM_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(dst, ctx->E.d_M, n_cells * 4, kind, st));
    if (!(flags & HT_MEM_DEVICE))
        CK(cudaStreamSynchronize(st));
    return HT_OK;
}

ht_status ht_get_edges(ht_ctx *ctx, float *theta_edges, float *phi_edges)
{
    if (!ctx || !theta_edges || !phi_edges)
        return set_err(HT_E_INVAL, "NULL argument");
    std::memcpy(theta_edges, ctx->E.et.data(), ctx->E.et.size() * 4);
    std::memcpy(phi_edges, ctx->E.ep.data(), ctx->E.ep.size() * 4);
    return HT_OK;
}

ht_status ht_set_matrix(ht_ctx *ctx, const uint32_t *src, uint64_t n_cells, uint32_t flags, void *stream)
{
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    if (!src || n_cells != ctx->E.n_cells)
        return set_err(HT_E_INVAL, "src must hold exactly n_theta*n_phi*n_a*n_b cells");
    std::string why;
    if ((s = hte::engine_ensure_any_matrix(ctx->E, &why)) != HT_OK)
        return set_err(s, why);
    ctx->last_peaks_only = false;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    const cudaMemcpyKind kind = (flags & HT_MEM_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(ctx->E.d_M, src, n_cells * 4, kind, st));
    if (!(flags & HT_MEM_DEVICE))
        CK(cudaStreamSynchronize(st));
    return HT_OK;
}

uint64_t ht_launch_count(const ht_ctx *ctx) { return ctx ? ctx->E.launches : 0; }

ht_status ht_set_tuning(ht_ctx *ctx, const ht_tuning *t)
{
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    if (!t)
        return set_err(HT_E_INVAL, "tuning is NULL");
    CK(cudaStreamSynchronize(ctx->stream));
    std::string why;
    s = hte::engine_set_tuning(ctx->E, *t, &ctx->poisoned, &why);
    return s == HT_OK ? HT_OK : set_err(s, why);
}

ht_status ht_get_tuning(ht_ctx *ctx, ht_tuning *t)
{
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    if (!t)
        return set_err(HT_E_INVAL, "tuning is NULL");
    hte::engine_get_tuning(ctx->E, t);
    return HT_OK;
}

ht_status ht_autotune(ht_ctx *ctx, uint32_t reps, ht_tuning *chosen, double *us_per_event)
{
    hte::TraceRange tr("ht_autotune");
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    std::string why;
    s = hte::engine_autotune(ctx->E, reps, ctx->stream, us_per_event, &why);
    if (s == HT_E_CUDA)
        ctx->poisoned = true;
    if (s != HT_OK)
        return set_err(s, why);
    if (chosen)
        return ht_get_tuning(ctx, chosen);
    return HT_OK;
}

ht_status ht_profile(ht_ctx *ctx, int enable)
{
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    CK(hte::prof_enable(ctx->E, enable != 0));
    return HT_OK;
}

ht_status ht_profile_read(ht_ctx *ctx, ht_kernel_time *out, uint32_t cap, uint32_t *n)
{
    ht_status s = check_ctx(ctx);
    if (s != HT_OK)
        return s;
    if (!n || (cap && !out))
        return set_err(HT_E_INVAL, "NULL argument");
    CK(hte::prof_read(ctx->E, out, cap, n));
    return HT_OK;
}

ht_status ht_validate(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold)
{
    std::string why;
    if (!htg::validate(binning, ranges, threshold, &why))
        return set_err(HT_E_INVAL, why);
    return HT_OK;
}

ht_status ht_compute_b_thresholds(const ht_binning *binning, const ht_ranges *ranges, float *beta)
{
    std::string why;
    if (!beta)
        return set_err(HT_E_INVAL, "beta must not be NULL");
    if (!htg::validate(binning, ranges, 1, &why))
        return set_err(HT_E_INVAL, why);
    htg::b_thresholds(ranges->b_min, htg::delta(ranges->b_min, ranges->b_max, binning->n_b), binning->n_b, beta);
    return HT_OK;
}

ht_status ht_compute_edges(const ht_binning *binning, const ht_ranges *ranges, float *theta_edges,
                           float *phi_edges)
{
    std::string why;
    if (!theta_edges || !phi_edges)
        return set_err(HT_E_INVAL, "edge arrays must not be NULL");
    if (!htg::validate(binning, ranges, 1, &why))
        return set_err(HT_E_INVAL, why);
    htg::theta_edges(ranges->theta_min, ranges->theta_max, binning->n_theta, theta_edges);
    htg::phi_edges(ranges->phi_min, ranges->phi_max, binning->n_phi, phi_edges);
    return HT_OK;
}

} // extern "C"
