// ht_find_maxima_noalloc: Step 2 (threshold + local-maxima scan) on a vote
// matrix the caller holds in device memory, with no device allocation.
//
// Who needs it: callers whose device memory belongs to someone else and that
// may not call cudaMalloc / cudaFree themselves -- a plugin running inside a
// framework whose caching allocator or fixed-budget pool owns every byte of
// the GPU (a raw cudaMalloc there can fail against the pool's reservation, or
// take memory the pool has promised elsewhere), or a trigger loop that cannot
// afford the device-wide synchronisation cudaFree implies.  Such callers
// cannot create an ht_ctx (it allocates M_H and its scratch), so this entry
// point takes the matrix and the output buffers from the caller and keeps its
// own scratch (peak entries, chunk descriptors, counters) in one file-scope
// __device__ array that every GPU loading the library holds until exit.
//
// The kernels are the standalone scan and the order kernel of ht_kernels.cu,
// given pointers into that array.
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "ht_geom.h"
#include "ht_internal.h"

namespace hte {
ht_status report(ht_status s, const std::string &msg);   // ht_api.cu
}

namespace {

// Limits of the static scratch.
constexpr uint32_t kMaxEvents = 4096;      // events per call
constexpr uint32_t kMaxGrid = 1024;        // scan CTAs
constexpr uint32_t kMaxSeq = 128;          // chunk descriptors per CTA
constexpr uint32_t kMaxEntries = 1u << 18; // peak entries over all events of a call
constexpr uint32_t kPeakBuf = 1024;        // K: entries buffered per scan CTA
constexpr uint32_t kThreads = 256;         // scan block size

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
// layout: counter block | cta_nseq | cta_total | desc | entries
constexpr size_t kOffCtr = 0;
constexpr size_t kOffNseq = align256(kOffCtr + (size_t)(htk::CTR_EVENTS + kMaxEvents) * 4);
constexpr size_t kOffTotal = align256(kOffNseq + (size_t)kMaxGrid * 4);
constexpr size_t kOffDesc = align256(kOffTotal + (size_t)kMaxGrid * 4);
constexpr size_t kOffEntries = align256(kOffDesc + (size_t)kMaxGrid * kMaxSeq * 8);
constexpr size_t kScratchBytes = align256(kOffEntries + (size_t)kMaxEntries * 16);
static_assert(kScratchBytes == 5267712, "the static scratch is stated as 5,267,712 bytes");

// The scratch.  In host code this name is only a handle for
// cudaGetSymbolAddress, never a device address.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Chunks a CTA owning `rows` rows may need (every chunk but the last holds
// at least K - per_round entries; a row holds at most ceil(n_b / 2) peaks).
uint32_t chunks_for(uint64_t rows, uint32_t nb, uint32_t K, uint32_t per_round)
{
    const uint64_t peaks = rows * ((nb + 1) / 2);
    const uint64_t c = peaks / (K - per_round) + 2;
    return (uint32_t)(c < kMaxSeq ? c : kMaxSeq);
}

ht_status cuda_err(cudaError_t e, const char *what)
{
    char buf[320];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    return hte::report(HT_E_CUDA, buf);
}

} // namespace

extern "C" ht_status ht_find_maxima_noalloc(const ht_binning *binning, const ht_ranges *ranges,
                                            uint32_t threshold, const uint32_t *M, uint32_t n_events,
                                            ht_peak *out, uint32_t capacity, uint32_t *counts, void *stream)
{
    std::string why;
    if (!binning || !ranges)
        return hte::report(HT_E_INVAL, "binning and ranges must not be NULL");
    if (!htg::validate(binning, ranges, threshold, &why))
        return hte::report(HT_E_INVAL, why);
    if (n_events < 1 || n_events > kMaxEvents)
        return hte::report(HT_E_INVAL, "ht_find_maxima_noalloc: need 1 <= n_events <= 4096 (static scratch limit)");
    if (!M || !counts || (capacity && !out))
        return hte::report(HT_E_INVAL, "M, counts and out (capacity > 0) must not be NULL");
    if ((uint64_t)n_events * capacity > 0xffffffffull)
        return hte::report(HT_E_INVAL, "n_events * capacity must be < 2^32");
    const cudaStream_t st = (cudaStream_t)stream;

    // --- set-up: the device address of the scratch, once per device --------
    int dev = 0, num_sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_err(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return hte::report(HT_E_INVAL, "ht_find_maxima_noalloc supports device ordinals below 64");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return cuda_err(e, "cudaGetSymbolAddress(static scratch)");
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    if ((e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_err(e, "cudaDeviceGetAttribute");

    // --- geometry (the scan reads sizes, threshold and the A / B ranges) ------
    htk::Geom g{};
    g.nt = binning->n_theta;
    g.np = binning->n_phi;
    g.na = binning->n_a;
    g.nb = binning->n_b;
    g.wt = binning->win_theta;
    g.wp = binning->win_phi;
    g.n_slices = g.nt * g.np;
    g.threshold = threshold;
    g.a_min = ranges->a_min;
    g.b_min = ranges->b_min;
    g.da = htg::delta(ranges->a_min, ranges->a_max, g.na);
    g.db = htg::delta(ranges->b_min, ranges->b_max, g.nb);
    g.nbf = (float)g.nb;
    g.inv_db = (float)(1.0 / (double)g.db);

    unsigned char *base = static_cast<unsigned char *>(scratch);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(base + kOffCtr);
    htk::Work w{};
    w.n_events = n_events;
    w.M = const_cast<uint32_t *>(M);   // read only
    w.n_cells = (uint64_t)g.n_slices * g.na * g.nb;
    w.status = ctr + htk::CTR_STATUS;
    w.ctr = ctr;

    // --- scan shape: register streaming (n_b % 4 == 0) or direct loads --------
    const int kind = (g.nb & 3u) == 0 ? htk::SCAN_LDG : htk::SCAN_DIRECT;
    const uint64_t G = (uint64_t)g.n_slices * g.na * n_events;
    htk::ScanArgs a{};
    a.K = kPeakBuf;
    a.S = 0;
    a.slot_words = 0;
    a.R = kind == htk::SCAN_LDG ? std::max<uint32_t>(1, htk::kLdgUPT * kThreads / (g.nb / 4)) : 16;
    // hot-chunk bitmap of the streaming scan, sized for the longest run of
    // rows a CTA can get (grid >= min(SMs, rows))
    const uint64_t grid_min = std::min<uint64_t>((uint64_t)num_sms, G);
    const uint64_t rows_max = (G + grid_min - 1) / grid_min + 1;
    a.hot_words = kind == htk::SCAN_LDG ? (uint32_t)((rows_max + a.R - 1) / a.R / 32 + 2) : 0u;
    if (htk::scan_smem_bytes(a) > 227 * 1024)
        return hte::report(HT_E_INVAL, "ht_find_maxima_noalloc: matrix too large for the scan's shared memory");
    int occ = 0;
    if ((e = htk::scan_occupancy(kind, htk::scan_smem_bytes(a), &occ)) != cudaSuccess)
        return cuda_err(e, "scan occupancy query");
    if (occ < 1)
        return hte::report(HT_E_CUDA, "ht_find_maxima_noalloc: the scan kernel cannot be resident");
    a.grid = (uint32_t)std::min<uint64_t>(std::min<uint64_t>((uint64_t)num_sms * occ, kMaxGrid), G);
    const uint64_t rows1 = (G + a.grid - 1) / a.grid + 1;   // longest run of rows of one CTA
    a.seq_max = chunks_for(rows1, g.nb, a.K, 2 * kThreads);
    a.entries_cap = kMaxEntries;
    a.entries = reinterpret_cast<uint4 *>(base + kOffEntries);
    a.g_count = ctr + htk::CTR_ENTRIES;
    a.desc = reinterpret_cast<uint2 *>(base + kOffDesc);
    a.cta_nseq = reinterpret_cast<uint32_t *>(base + kOffNseq);
    a.cta_total = reinterpret_cast<uint32_t *>(base + kOffTotal);
    a.ev_count = ctr + htk::CTR_EVENTS;

    htk::OrderArgs o{};
    o.out = reinterpret_cast<htk::Peak *>(out);
    o.capacity = capacity;
    o.counts = counts;
    o.ev_count = a.ev_count;
    o.ticket = ctr + htk::CTR_OTICKET;
    o.g_count = a.g_count;

    // --- run: clear the counters (the array keeps the last call's contents),
    // scan, order, then read the status word ---------------------------------
    if ((e = cudaMemsetAsync(ctr, 0, (size_t)(htk::CTR_EVENTS + n_events) * 4, st)) != cudaSuccess)
        return cuda_err(e, "clear the static counters");
    if ((e = htk::launch_scan(g, w, a, kind, st)) != cudaSuccess)
        return cuda_err(e, "scan launch");
    if ((e = htk::launch_order(g, w, a, o, st)) != cudaSuccess)
        return cuda_err(e, "order launch");
    uint32_t status = 0;
    if ((e = cudaMemcpyAsync(&status, w.status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_err(e, "read the status word");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_err(e, "ht_find_maxima_noalloc");
    if (status & htk::ST_SCRATCH_OVERFLOW)
        return hte::report(HT_E_NOMEM, "ht_find_maxima_noalloc: more peaks than the static scratch holds "
                                       "(262144 entries per call, 128 chunks per scan CTA)");
    if (status)
        return hte::report(HT_E_CUDA, "ht_find_maxima_noalloc: a kernel reported a failure");
    return HT_OK;
}
