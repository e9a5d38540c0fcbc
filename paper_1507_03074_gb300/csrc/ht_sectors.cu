// C ABI: phi sectors (ht_sectors_*).
//
// Sec. 4 splits the transverse plane into four phi sectors, read out
// independently, runs one Hough transform per sector with a lighter matrix
// M_H(A, B, theta) and merges the results.  On one GPU the sectors are
// contexts on their own streams: a fill or a maxima scan forks from the
// caller's stream into every sector and joins back, so the sectors' kernels
// overlap on the device, and a merge kernel puts the sectors' peak lists
// into the unsplit matrix's numbering and order.  Each sector context takes
// its slice of the unsplit phi edge table, so it bins every hit exactly as
// the unsplit context does: its matrix is those phi bins of the unsplit
// M_H, and (the maxima rule compares (A, B) neighbours within a slice) its
// peaks are the unsplit peaks of those bins.
#include "ht_engine.h"
#include "ht_geom.h"
#include "ht_trace.h"

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace hte {
ht_status report(ht_status s, const std::string &msg);   // ht_api.cu
Engine &ctx_engine(ht_ctx *c);                            // ht_api.cu
} // namespace hte

struct ht_sectors {
    uint32_t S = 0, m = 0;            // sectors, phi bins per sector
    uint32_t max_hits = 0;
    std::vector<ht_ctx *> ctx;
    std::vector<cudaStream_t> st;
    std::vector<cudaEvent_t> done;    // per sector: its part of the last fork
    cudaEvent_t fork = nullptr;
    cudaStream_t stream = nullptr;    // the object's own stream
    float *d_in = nullptr, *h_in = nullptr;   // hit staging (x | y | z)
    cudaEvent_t ev_in = nullptr;
    bool ev_in_pending = false;
    htk::Peak *d_sec = nullptr;       // S lists of sec_cap peaks
    uint32_t sec_cap = 0;
    uint32_t *d_cnt = nullptr;        // S counts + merged total
    htk::Peak *h_out = nullptr;       // mapped pinned: merged peaks of host-memory calls
    htk::Peak *h_out_dev = nullptr;   // its device address
    uint32_t out_cap = 0;
    uint32_t *h_small = nullptr;      // mapped pinned: merged total of host-memory calls
    uint32_t *h_small_dev = nullptr;  // its device address
    bool poisoned = false;
};

namespace {

ht_status sec_fail(ht_sectors *s, cudaError_t e, const char *what)
{
    if (s)
        s->poisoned = true;
    char buf[320];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return hte::report(HT_E_CUDA, buf);
}

#define SCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return sec_fail(sec, e_, #call);                                                       \
    } while (0)

ht_status check_sec(ht_sectors *sec)
{
    if (!sec)
        return hte::report(HT_E_INVAL, "sectors object is NULL");
    if (sec->poisoned)
        return hte::report(HT_E_STATE, "sectors object failed earlier (HT_E_CUDA); destroy it");
    return HT_OK;
}

// Number of entries of the sorted list p[0, n) with itheta < t (less) or
// itheta <= t (!less).
__device__ uint32_t theta_bound(const htk::Peak *p, uint32_t n, uint32_t t, bool less)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        const uint32_t v = p[mid].itheta;
        if (less ? v < t : v <= t)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Merge of the sectors' peak lists.  Sector k's list (at sec + k cap)
// holds its first min(cnt[k], cap) peaks in its own linear order, (itheta,
// iphi - k m, ia, ib); the unsplit order is (itheta, k, iphi - k m, ia, ib).
// A peak's place is the number of entries that precede it: its rank q in its
// own list plus, in every other sector k2, the entries with a smaller theta
// bin, or the same one when k2 < k.  Places below `limit` (<= cap) are
// written.  When sector k2's list was cut at cap and all of it precedes the
// peak, the place is >= cap: the written places are exactly the unsplit
// list's first `limit` entries.  *n_found receives the total.
__global__ void k_merge_sectors(const htk::Peak *sec, const uint32_t *cnt, uint32_t S, uint32_t cap,
                                uint32_t limit, uint32_t m, htk::Peak *out, uint32_t *n_found)
{
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (tid == 0) {
        uint64_t total = 0;
        for (uint32_t k = 0; k < S; ++k)
            total += cnt[k];
        *n_found = total > 0xffffffffull ? 0xffffffffu : (uint32_t)total;
    }
    for (uint32_t k = 0; k < S; ++k) {
        const uint32_t valid = min(cnt[k], cap);
        for (uint32_t q = tid; q < valid; q += stride) {
            htk::Peak p = sec[(size_t)k * cap + q];
            uint64_t pos = q;
            for (uint32_t k2 = 0; k2 < S; ++k2)
                if (k2 != k)
                    pos += theta_bound(sec + (size_t)k2 * cap, min(cnt[k2], cap), p.itheta, k2 > k);
            if (pos < limit) {
                p.iphi += k * m;
                out[pos] = p;
            }
        }
    }
}

// Fork the sectors' streams from st (every sector stream waits for st's
// work so far).
ht_status fork_from(ht_sectors *sec, cudaStream_t st)
{
    SCK(cudaEventRecord(sec->fork, st));
    for (uint32_t k = 0; k < sec->S; ++k)
        SCK(cudaStreamWaitEvent(sec->st[k], sec->fork, 0));
    return HT_OK;
}

// Join: st waits for every sector stream's work so far.
ht_status join_into(ht_sectors *sec, cudaStream_t st)
{
    for (uint32_t k = 0; k < sec->S; ++k) {
        SCK(cudaEventRecord(sec->done[k], sec->st[k]));
        SCK(cudaStreamWaitEvent(st, sec->done[k], 0));
    }
    return HT_OK;
}

} // namespace

extern "C" {

ht_status ht_sectors_destroy(ht_sectors *sec)
{
    if (!sec)
        return HT_OK;
    if (sec->stream)
        cudaStreamSynchronize(sec->stream);
    for (cudaStream_t s : sec->st)
        if (s)
            cudaStreamSynchronize(s);
    for (ht_ctx *c : sec->ctx)
        ht_destroy(c);
    for (cudaStream_t s : sec->st)
        if (s)
            cudaStreamDestroy(s);
    for (cudaEvent_t e : sec->done)
        if (e)
            cudaEventDestroy(e);
    if (sec->fork)
        cudaEventDestroy(sec->fork);
    if (sec->ev_in)
        cudaEventDestroy(sec->ev_in);
    if (sec->stream)
        cudaStreamDestroy(sec->stream);
    cudaFree(sec->d_in);
    cudaFree(sec->d_sec);
    cudaFree(sec->d_cnt);
    cudaFreeHost(sec->h_out);
    cudaFreeHost(sec->h_in);
    cudaFreeHost(sec->h_small);
    delete sec;
    return HT_OK;
}

ht_status ht_sectors_create(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                            uint32_t n_sectors, uint32_t max_hits, ht_sectors **out)
{
    if (!out)
        return hte::report(HT_E_INVAL, "out is NULL");
    *out = nullptr;
    std::string why;
    if (!htg::validate(binning, ranges, threshold, &why))
        return hte::report(HT_E_INVAL, why);
    if (n_sectors < 1 || binning->n_phi % n_sectors)
        return hte::report(HT_E_INVAL, "n_sectors must be >= 1 and divide n_phi");
    if (binning->win_phi && n_sectors > 1)
        return hte::report(HT_E_INVAL, "phi sectors need win_phi == 0 (a window would reach the next sector)");
    if (max_hits < 1)
        return hte::report(HT_E_INVAL, "max_hits must be >= 1");
    ht_sectors *sec = new (std::nothrow) ht_sectors();
    if (!sec)
        return hte::report(HT_E_NOMEM, "host allocation failed");
    sec->S = n_sectors;
    sec->m = binning->n_phi / n_sectors;
    sec->max_hits = max_hits;
    // the unsplit phi edge table; sector k takes entries k m .. (k + 1) m
    std::vector<float> ep(binning->n_phi + 1);
    htg::phi_edges(ranges->phi_min, ranges->phi_max, binning->n_phi, ep.data());
    const double lo = htg::snap_quarter(ranges->phi_min), hi = htg::snap_quarter(ranges->phi_max);
    ht_binning sb = *binning;
    sb.n_phi = sec->m;
    for (uint32_t k = 0; k < n_sectors; ++k) {
        ht_ranges sr = *ranges;
        sr.phi_min = (float)(lo + (hi - lo) * k / n_sectors);
        sr.phi_max = (float)(lo + (hi - lo) * (k + 1) / n_sectors);
        if (!(sr.phi_min < sr.phi_max)) {
            ht_sectors_destroy(sec);
            return hte::report(HT_E_INVAL, "sector phi ranges collapse in float; use fewer sectors");
        }
        ht_ctx *c = nullptr;
        ht_status s = ht_create(&sb, &sr, threshold, max_hits, &c);
        if (s != HT_OK) {
            const std::string msg = std::string("sector context: ") + ht_last_error();
            ht_sectors_destroy(sec);
            return hte::report(s, msg);
        }
        sec->ctx.push_back(c);
        cudaError_t e = hte::engine_set_phi_edges(hte::ctx_engine(c), ep.data() + (size_t)k * sec->m);
        cudaStream_t sk = nullptr;
        cudaEvent_t dk = nullptr;
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&sk, cudaStreamNonBlocking);
        sec->st.push_back(sk);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&dk, cudaEventDisableTiming);
        sec->done.push_back(dk);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ht_sectors_destroy(sec);
            return hte::report(HT_E_CUDA, std::string("sector setup: ") + cudaGetErrorString(e));
        }
    }
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&sec->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&sec->fork, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&sec->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMalloc(&sec->d_in, (size_t)max_hits * 12 + 64)) != cudaSuccess ||
        (e = cudaMalloc(&sec->d_cnt, (size_t)(n_sectors + 1) * 4)) != cudaSuccess ||
        (e = cudaMallocHost(&sec->h_in, (size_t)max_hits * 12 + 64)) != cudaSuccess ||
        (e = cudaHostAlloc(&sec->h_small, 16, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer((void **)&sec->h_small_dev, sec->h_small, 0)) != cudaSuccess) {
        cudaGetLastError();
        ht_sectors_destroy(sec);
        return hte::report(HT_E_NOMEM, std::string("allocation failed: ") + cudaGetErrorString(e));
    }
    *out = sec;
    return HT_OK;
}

ht_status ht_sectors_fill(ht_sectors *sec, const float *x, const float *y, const float *z, uint32_t n_hits,
                          uint32_t flags, void *stream)
{
    hte::TraceRange tr("ht_sectors_fill");
    ht_status s = check_sec(sec);
    if (s != HT_OK)
        return s;
    if (flags & ~(uint32_t)(HT_MEM_DEVICE | HT_ACCUMULATE | HT_FILL_NAIVE | HT_PEAKS_ONLY))
        return hte::report(HT_E_INVAL, "unknown flag");
    if (n_hits && (!x || !y || !z))
        return hte::report(HT_E_INVAL, "hit arrays must not be NULL");
    if (n_hits > sec->max_hits)
        return hte::report(HT_E_INVAL, "more hits than max_hits");
    cudaStream_t st = stream ? (cudaStream_t)stream : sec->stream;
    const float *px = x, *py = y, *pz = z;
    if (!(flags & HT_MEM_DEVICE) && n_hits) {
        if (sec->ev_in_pending)
            SCK(cudaEventSynchronize(sec->ev_in));   // the pinned staging is free again
        const size_t bytes = (size_t)n_hits * 4;
        std::memcpy(sec->h_in, x, bytes);
        std::memcpy(sec->h_in + n_hits, y, bytes);
        std::memcpy(sec->h_in + 2 * (size_t)n_hits, z, bytes);
        SCK(cudaMemcpyAsync(sec->d_in, sec->h_in, 3 * bytes, cudaMemcpyHostToDevice, st));
        SCK(cudaEventRecord(sec->ev_in, st));
        sec->ev_in_pending = true;
        px = sec->d_in;
        py = sec->d_in + n_hits;
        pz = sec->d_in + 2 * (size_t)n_hits;
    }
    s = fork_from(sec, st);
    if (s != HT_OK)
        return s;
    for (uint32_t k = 0; k < sec->S; ++k) {
        s = ht_fill(sec->ctx[k], px, py, pz, n_hits, flags | HT_MEM_DEVICE, sec->st[k]);
        if (s != HT_OK) {
            if (s == HT_E_CUDA || s == HT_E_STATE)
                sec->poisoned = true;
            join_into(sec, st);
            return s;   // the context's message stands
        }
    }
    return join_into(sec, st);
}

ht_status ht_sectors_find_maxima(ht_sectors *sec, ht_peak *out, uint32_t capacity, uint32_t *n_found,
                                 uint32_t flags, void *stream)
{
    hte::TraceRange tr("ht_sectors_find_maxima");
    ht_status s = check_sec(sec);
    if (s != HT_OK)
        return s;
    if (flags & ~(uint32_t)HT_MEM_DEVICE)
        return hte::report(HT_E_INVAL, "unknown flag");
    if (!n_found || (capacity && !out))
        return hte::report(HT_E_INVAL, "out (capacity > 0) and n_found must not be NULL");
    cudaStream_t st = stream ? (cudaStream_t)stream : sec->stream;
    const bool dev = (flags & HT_MEM_DEVICE) != 0;
    const uint32_t cap = capacity ? capacity : 1;
    if (cap > sec->sec_cap) {
        SCK(cudaDeviceSynchronize());   // buffers may be in use on any sector stream
        cudaFree(sec->d_sec);
        sec->d_sec = nullptr;
        sec->sec_cap = 0;
        SCK(cudaMalloc(&sec->d_sec, (size_t)sec->S * cap * sizeof(htk::Peak)));
        sec->sec_cap = cap;
    }
    if (!dev && cap > sec->out_cap) {
        SCK(cudaStreamSynchronize(st));
        cudaFreeHost(sec->h_out);
        sec->h_out = sec->h_out_dev = nullptr;
        sec->out_cap = 0;
        SCK(cudaHostAlloc(&sec->h_out, (size_t)cap * sizeof(htk::Peak), cudaHostAllocMapped));
        SCK(cudaHostGetDevicePointer((void **)&sec->h_out_dev, sec->h_out, 0));
        sec->out_cap = cap;
    }
    s = fork_from(sec, st);
    if (s != HT_OK)
        return s;
    for (uint32_t k = 0; k < sec->S; ++k) {
        s = ht_find_maxima(sec->ctx[k], reinterpret_cast<ht_peak *>(sec->d_sec + (size_t)k * cap), cap,
                           sec->d_cnt + k, HT_MEM_DEVICE, sec->st[k]);
        if (s != HT_OK) {
            if (s == HT_E_CUDA || s == HT_E_STATE)
                sec->poisoned = true;
            join_into(sec, st);
            return s;
        }
    }
    s = join_into(sec, st);
    if (s != HT_OK)
        return s;
    // host-memory calls: the merge writes peaks and total into mapped pinned memory
    htk::Peak *dst = dev ? reinterpret_cast<htk::Peak *>(out) : sec->h_out_dev;
    uint32_t *cnt = dev ? n_found : sec->h_small_dev;
    int nsm = 0, dv = 0;
    SCK(cudaGetDevice(&dv));
    SCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dv));
    k_merge_sectors<<<(unsigned)nsm, 256, 0, st>>>(sec->d_sec, sec->d_cnt, sec->S, cap, capacity, sec->m, dst, cnt);
    SCK(cudaGetLastError());
    if (dev)
        return HT_OK;
    SCK(cudaStreamSynchronize(st));
    for (uint32_t k = 0; k < sec->S; ++k) {
        s = ht_sync(sec->ctx[k], sec->st[k]);   // device-side failures of the sector's kernels
        if (s != HT_OK)
            return s;
    }
    const uint32_t n = sec->h_small[0];
    const uint32_t kk = n < capacity ? n : capacity;
    if (kk)
        std::memcpy(out, sec->h_out, (size_t)kk * sizeof(ht_peak));
    *n_found = n;
    return n > capacity ? HT_TRUNCATED : HT_OK;
}

ht_status ht_sectors_copy_matrix(ht_sectors *sec, uint32_t sector, uint32_t *dst, uint64_t n_cells)
{
    ht_status s = check_sec(sec);
    if (s != HT_OK)
        return s;
    if (sector >= sec->S)
        return hte::report(HT_E_INVAL, "sector out of range");
    SCK(cudaStreamSynchronize(sec->stream));
    SCK(cudaStreamSynchronize(sec->st[sector]));
    return ht_copy_matrix(sec->ctx[sector], dst, n_cells, HT_MEM_HOST, sec->st[sector]);
}

} // extern "C"
