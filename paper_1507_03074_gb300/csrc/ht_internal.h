// Internal host/device interface between the C ABI (ht_api.cu) and the
// kernels (ht_kernels.cu).  Not installed; not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "ht_device.cuh"

namespace htk {

// Privatised fill: A-strip of W rows per work item (u16 counters; W/2 rows
// per pass when a slice holds >= 65536 hits and needs u32 counters).
struct FillCfg {
    uint32_t W;           // rows per item (power of two, divides threads)
    uint32_t strips;      // ceil(n_a / W)
    uint32_t pitch16;     // tile words per row in u16 mode (multiple of 32)
    uint32_t pitch32;     // tile words per row in u32 mode (multiple of 32)
    uint32_t HC;          // hits staged in shared memory per chunk (>= 2 * threads)
    uint32_t tile_words;  // W * pitch16
    uint32_t threads;     // block size
    uint32_t accumulate;  // add the tile to M_H instead of storing it
    uint32_t beta_words;  // shared-memory copy of the B-bin thresholds (n_b + 1, rounded to 4)
    uint32_t dyn;         // 1: the last dyn_items() items are handed out at run time (see below)
    uint32_t bulk;        // fused fill: 1 = passes leave through u32 staging and bulk copies (k_fill_bulk)
    uint32_t vote_weight; // cost of one vote against one cell written, in the static split (cta_items)
    uint32_t vote_agg;    // bulk-copy-tile fill: warp-aggregated vote increments (match.any + one add)
};

// Shared-memory words of the fused fill's two u32 staging buffers (half a
// u16 pass, W / 2 rows of n_b cells, each), or 0 without bulk copies.
__host__ __device__ constexpr uint32_t staging_words(const FillCfg &c, uint32_t nb) { return c.bulk ? c.W * nb : 0u; }

// The fills split the first items - dyn_items(items, grid) work items over
// their CTAs by estimated cost, and hand the rest out one at a time to the
// CTAs that finish first (an atomic counter), which absorbs the spread of
// the static split.  In the fused fill every handed-out item gets its own
// list of candidate chunks, numbered grid + its rank, so the lists stay in
// linear order.
__host__ __device__ constexpr uint64_t dyn_items(uint64_t items, uint32_t grid)
{
    return items / 8 < 2ull * grid ? items / 8 : 2ull * grid;
}

// Scan (and its chunk bookkeeping).  Shared with k_order.
struct ScanArgs {
    uint32_t grid;        // persistent CTAs (each owns a contiguous run of rows)
    uint32_t R;           // own rows per stage (bulk) / per chunk (streaming, direct)
    uint32_t S;           // stages in the shared-memory ring (<= 8)
    uint32_t K;           // peak entries buffered in shared memory (>= 2*256)
    uint32_t slot_words;  // (R + 2) * n_b
    uint32_t hot_words;   // streaming: words of the per-CTA hot-chunk bitmap
    uint32_t seq_max;     // chunk descriptors per CTA
    uint32_t entries_cap; // global entry scratch capacity
    uint4 *entries;       // {lin within event, event, votes, 0}
    uint32_t *g_count;    // entries used (reset by k_order)
    uint2 *desc;          // [grid][seq_max] {base, n}
    uint32_t *cta_nseq;   // [grid] interior chunks
    uint32_t *cta_total;  // [grid] entries
    uint32_t *ev_count;   // [n_events] peaks per event (reset by k_order)
};

struct OrderArgs {
    Peak *out;            // [n_events][capacity]
    uint32_t capacity;
    uint32_t *counts;     // [n_events] total peaks per event
    uint32_t *ev_count;
    uint32_t *ticket;     // last-CTA detection (reset by k_order)
    uint32_t *g_count;    // entries used (reset by the last CTA)
    uint32_t compact;     // 1: one list out[rank] over all events, else out[e][capacity]
};

cudaError_t launch_bin(const Geom &g, const Work &w, uint32_t grid, cudaStream_t st);
cudaError_t launch_scatter(const Geom &g, const Work &w, uint32_t grid, cudaStream_t st);
// k_bin + k_scatter as one cluster of cs <= kBinClusterMax CTAs of
// kBinClusterThreads threads, each holding at most kBinClusterHPT hits: for
// launches of at most kBinClusterMax * kBinClusterThreads * kBinClusterHPT hits
// whose three words per unit and hit offsets fit kBinClusterSmem bytes.
constexpr uint32_t kBinClusterMax = 8, kBinClusterThreads = 1024, kBinClusterHPT = 2;
constexpr size_t kBinClusterSmem = 40 * 1024;
size_t bin_cluster_smem_bytes(const Geom &g, uint32_t n_events);
cudaError_t launch_bin_cluster(const Geom &g, const Work &w, uint32_t cs, cudaStream_t st);
// Whether this device runs a cluster of kBinClusterMax such CTAs.
bool bin_cluster_supported(size_t smem);
size_t fill_smem_bytes(const FillCfg &c);
cudaError_t launch_fill_priv(const Geom &g, const Work &w, const FillCfg &c, uint32_t grid,
                             cudaStream_t st);
size_t fill_scan_smem_bytes(const FillCfg &c, const ScanArgs &a, uint32_t nb);
cudaError_t launch_fill_scan(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                             cudaStream_t st);
cudaError_t fill_scan_occupancy(const FillCfg &c, const ScanArgs &a, uint32_t nb, int *blocks_per_sm);
// Warp-specialised fused fill: kWsThreads threads, two tiles (c.threads is
// the vote group's size, kWsThreads / 2).
constexpr uint32_t kWsThreads = 1024;
size_t fill_ws_smem_bytes(const FillCfg &c, const ScanArgs &a);
cudaError_t launch_fill_ws(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                           cudaStream_t st);
cudaError_t fill_ws_occupancy(const FillCfg &c, const ScanArgs &a, int *blocks_per_sm);
// Fused fill whose passes leave as bulk copies of two alternating u32 tiles
// of W x n_b cells each (c.tile_words = W * n_b; n_b a multiple of 4).
size_t fill_tma_smem_bytes(const FillCfg &c, const ScanArgs &a);
cudaError_t launch_fill_tma(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                            cudaStream_t st);
cudaError_t fill_tma_occupancy(const FillCfg &c, const ScanArgs &a, int *blocks_per_sm);
// After a fused fill (same grid): test its candidate entries, keep the peaks
// (peaks_only: after k_fill_peaks, finishing the edge-flagged tests).
cudaError_t launch_peaks(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                         bool peaks_only, cudaStream_t st);
// The fused fill without writing M_H (same shapes and grid as k_fill_scan).
cudaError_t launch_fill_peaks(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                              cudaStream_t st);
cudaError_t launch_clear(uint32_t *M, uint64_t words, uint32_t grid, cudaStream_t st);
cudaError_t launch_fill_naive(const Geom &g, const Work &w, uint32_t num_sms, cudaStream_t st);
size_t scan_smem_bytes(const ScanArgs &a);

// Layout of the counter block: [0] status, [1] entries used, [2] order
// ticket, [3] binning ticket (reset by k_bin's last block), [4] next
// handed-out fill item and [5] fill CTAs done with them (both reset by the
// last such CTA), [6 ..) peaks per event.  k_bin zeroes words 1, 2 and
// [6, 6 + n_events) before every fill.
enum : uint32_t {
    CTR_STATUS = 0, CTR_ENTRIES = 1, CTR_OTICKET = 2, CTR_BTICKET = 3, CTR_DYN = 4, CTR_DYN_DONE = 5,
    CTR_P4TICKET = 6, CTR_EVENTS = 7
};

// Cost model of the balanced split of (event, slice, strip) work items over
// the fill CTAs: a strip of r rows in a slice of h hits costs
// r * (n_b + v * h) (writing a cell ~ 1, one vote ~ v = FillCfg::vote_weight).
// The fills that write M_H take kVoteWeight; the peaks-only fill, whose
// cells cost only their clearing, weighs votes more (kPeaksVoteWeight; 6,
// 12 and 24 were measured on paper-scale events, 24 balancing its CTAs best).
constexpr uint32_t kVoteWeight = 6;
constexpr uint32_t kPeaksVoteWeight = 24;

// Scan variants: bulk-copy (TMA) ring, register streaming, direct (any n_b).
// The streaming variant keeps kLdgUPT 16-byte loads per thread in flight.
constexpr uint32_t kLdgUPT = 8;
// Candidate cells (>= threshold) a streaming-scan CTA lists before testing them.
constexpr uint32_t kCand = 1024;
// Candidate cells a fused-fill CTA lists per pass; a pass with more emits
// its rows' cells >= T read back from M_H.
constexpr uint32_t kFusedCand = 256;
// Entries the fused fill emits per group round: at most this many per
// round, so every chunk but the last holds at least K - fused_round(threads, K).
__host__ __device__ constexpr uint32_t fused_round(uint32_t threads, uint32_t K) { return threads < K / 2 ? threads : K / 2; }
enum ScanKind { SCAN_DIRECT = 0, SCAN_BULK = 1, SCAN_LDG = 2 };
cudaError_t launch_scan(const Geom &g, const Work &w, const ScanArgs &a, int kind, cudaStream_t st);
cudaError_t launch_order(const Geom &g, const Work &w, const ScanArgs &a, const OrderArgs &o,
                         cudaStream_t st);
// L2 atomic increments at pseudo-random words of buf (mask + 1 words,
// per_thread per thread, 256 threads per CTA).
cudaError_t launch_atomic_rate(uint32_t *buf, uint32_t mask, uint32_t per_thread, uint32_t seed, uint32_t grid,
                               cudaStream_t st);
// One bounded wait that nothing ends (k_wait_probe): flags ST_WAIT_TIMEOUT
// after limit_ms (at most about a second).
cudaError_t launch_wait_probe(uint32_t *status, uint32_t limit_ms, cudaStream_t st);
// The 4-D filter of a 2-D peak list (k_peaks4d): keep holds cap_in flags;
// ticket is a zero counter word (reset by the kernel).
cudaError_t launch_peaks4d(const Geom &g, const uint32_t *M, const Peak *in, const uint32_t *n_in, uint32_t cap_in,
                           uint8_t *keep, Peak *out, uint32_t cap_out, uint32_t *n_out, uint32_t *ticket,
                           uint32_t *status, uint32_t grid, cudaStream_t st);
cudaError_t scan_occupancy(int kind, size_t smem, int *blocks_per_sm);
cudaError_t fill_occupancy(const FillCfg &c, int *blocks_per_sm);

} // namespace htk
