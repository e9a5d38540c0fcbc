// Engine: the resident device workspace for up to max_events events of one
// binning, and the enqueue functions of the two steps.  Internal; the C ABI
// objects (context, batch, server) are built on it.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "ht.h"   // include/ht.h (the build adds include/ to the search path)
#include "ht_internal.h"

namespace hte {

// Launch-shape knobs (the C ABI's ht_tuning); 0 means automatic.  Results
// do not depend on them.
struct Tuning {
    uint32_t fill_W = 0;              // A rows per shared-memory tile (power of two)
    uint32_t fill_threads = 0;        // 256, 512 or 1024
    uint32_t fill_HC = 0;             // hits staged per chunk (>= 2 * threads)
    uint32_t fill_blocks_per_sm = 0;  // cap below the occupancy limit
    uint32_t scan_kind = 0;           // 0 auto, 1 bulk-copy ring, 2 register streaming, 3 direct
    uint32_t scan_stage_bytes = 0;    // bulk-copy stage size
    uint32_t scan_slots = 0;          // bulk-copy ring depth (2..8)
    uint32_t scan_blocks_per_sm = 0;  // cap below the occupancy limit
    uint32_t fused = 0;               // 0 auto, 1 fused (one thread group), 2 off, 3 fused warp-specialised,
                                      // 4 fused with bulk-copy staging, 5 fused with bulk-copy u32 tiles
    uint32_t vote_agg = 0;            // warp-aggregated vote increments (bulk-copy-tile fill)
    uint32_t bin_cluster = 0;         // 0 auto, 1 k_bin_cluster when it fits, 2 k_bin + k_scatter
};

// Optional per-kernel timing with CUDA events recorded on the launching
// stream around every launch (enabled by ht_profile).
enum KernelKind {
    K_BIN, K_SCATTER, K_FILL_PRIV, K_FILL_SCAN, K_FILL_WS, K_FILL_PEAKS, K_PEAKS, K_CLEAR, K_FILL_NAIVE, K_SCAN,
    K_ORDER, K_PEAKS4D, K_FILL_TMA, K_BIN_CLUSTER, K_NKINDS
};
extern const char *const kKernelNames[K_NKINDS];

struct Prof {
    bool on = false;
    struct Rec { int kind; cudaEvent_t a, b; };
    std::vector<Rec> pending;
    std::vector<cudaEvent_t> pool;
    double ms[K_NKINDS] = {};
    uint64_t n[K_NKINDS] = {};
};

struct Engine {
    ht_binning b{};
    ht_ranges r{};
    uint32_t threshold = 1;
    uint32_t max_events = 1;
    uint32_t max_hits = 0;       // total hits over all events of one launch
    uint32_t max_admit = 1;
    uint64_t n_cells = 0;        // per event
    int device = 0;
    int num_sms = 0;
    std::vector<float> et, ep, bth;   // edge tables, B-bin thresholds

    htk::Geom geom{};
    htk::FillCfg fill{};
    bool fill_priv_ok = false;   // the tile fits in shared memory
    uint32_t fill_grid = 0;
    bool fused_ok = false;       // the fused fill + maxima kernel fits
    htk::FillCfg fused_fill{};   // its tile / staging shape
    uint32_t fused_grid = 0;
    uint32_t fused_K = 0;
    bool ws_ok = false;          // the warp-specialised fused kernel fits
    htk::FillCfg ws_fill{};      // its shape (threads = one group)
    uint32_t ws_grid = 0;
    bool use_ws = false;         // fills run the warp-specialised kernel
    bool tma_ok = false;         // the bulk-copy-tile fused kernel fits
    htk::FillCfg tma_fill{};     // its shape (two u32 tiles of W x n_b)
    uint32_t tma_grid = 0;
    uint32_t tma_K = 0;          // its peak buffer
    bool use_tma = false;        // fills run the bulk-copy-tile kernel
    htk::ScanArgs scan{};
    int scan_kind = 0;            // htk::ScanKind in use
    uint32_t scan_grid_max = 0;
    uint32_t grid_cap = 0;        // CTAs the bookkeeping arrays are sized for
    size_t book_bytes = 0;        // allocated bookkeeping
    uint32_t clear_grid = 0;
    Tuning tune;

    // state of the last fill: peaks already found by the fused kernel
    bool fused_valid = false;
    uint32_t fused_grid_used = 0;
    uint32_t fused_events = 0;
    bool ctr_dirty = false;      // counters hold an unconsumed fused fill's peaks
    int bin_cluster = -1;        // k_bin_cluster usable here (-1: not checked yet)
    bool tma_capped = false;     // fill_blocks_per_sm holds the bulk-copy-tile fill below its occupancy
    bool fused_capped = false;   // ... and the fused fills (the peaks-only fill among them)
    uint32_t split_mode = htk::kSplitEarly;   // Work::split_mode of the fill after the last binning
    uint32_t split_grid = 0, split_strips = 0, split_vw = 0;
    uint64_t split_n_static = 0;
    uint64_t *d_split = nullptr;              // [split_cap] k_bin_cluster's split for the fill
    uint32_t split_cap = 0;
    const uint32_t *last_hit_off = nullptr;   // what the last fill binned
    uint32_t last_n_hits0 = 0, last_n_events = 0;
    bool last_accumulate = false;

    float *d_edges = nullptr;
    uint32_t *d_M = nullptr;
    float4 *d_hits4 = nullptr;
    uint32_t *d_codes = nullptr;
    uint32_t *d_edge = nullptr;   // peaks-only fills: edge rows of every pass (allocated on first use)
    uint32_t edge_pass = 0;       // passes per unit the edge buffer holds
    uint32_t *d_slice = nullptr;  // unit counts | scatter cursors | offsets (3 * units + 1)
    float4 *d_list = nullptr;     // hit records unit by unit
    uint32_t list_cap = 0;
    uint4 *d_entries = nullptr;
    void *d_book = nullptr;       // desc | cta arrays
    uint32_t *d_ctr = nullptr;    // counter block (htk::CTR_*)
    size_t device_bytes = 0;
    uint64_t launches = 0;
    Prof prof;
};

// Profiling: enable (resets totals) / disable; read folds every completed
// record into the totals (synchronises on the last recorded event).
cudaError_t prof_enable(Engine &E, bool on);
cudaError_t prof_collect(Engine &E);

// Create / destroy.  Returns HT_OK, HT_E_INVAL or HT_E_NOMEM / HT_E_CUDA with *why.
ht_status engine_create(Engine &E, const ht_binning *b, const ht_ranges *r, uint32_t threshold,
                        uint32_t max_events, uint32_t max_hits, const Tuning *tune, std::string *why);
void engine_destroy(Engine &E);

// Re-derive launch shapes after changing E.tune (the autotuner does this).
ht_status engine_configure(Engine &E, std::string *why);

// Step 1 for n_events events whose hits (device pointers) are concatenated;
// d_hit_off (device, n_events + 1) or nullptr for one event of n_hits0 hits.
// n_total (host) is the total hit count; it sizes the binning grid.  Unless
// HT_ACCUMULATE or HT_FILL_NAIVE is set (or the tuning turns it off), the
// fused kernel also finds the peaks, which engine_scan then only orders.
cudaError_t engine_fill(Engine &E, const float *x, const float *y, const float *z,
                        const uint32_t *d_hit_off, uint32_t n_hits0, uint32_t n_events,
                        uint32_t n_total, uint32_t flags, cudaStream_t st);

// The voting part of engine_fill alone, on the hits engine_fill last binned
// (the autotuner re-runs it under each candidate tuning).
cudaError_t engine_vote(Engine &E, const uint32_t *d_hit_off, uint32_t n_hits0, uint32_t n_events, uint32_t flags,
                        cudaStream_t st);

// Time candidate tunings on the hits of the last fill (vote + maxima, reps
// times each) and keep the fastest; M_H and the peak state end as after a
// fill with the chosen tuning.  *best_us receives its time per event.
ht_status engine_autotune(Engine &E, uint32_t reps, cudaStream_t st, double *best_us, std::string *why);

// Step 2: peaks of every event into out[e * capacity ...], totals into counts[e].
// compact: one list ordered by (event, linear index) in out[0 .. capacity)
// instead of capacity entries per event.
cudaError_t engine_scan(Engine &E, uint32_t n_events, htk::Peak *out, uint32_t capacity,
                        uint32_t *counts, cudaStream_t st, bool compact = false);

// Grow the peak-entry scratch to the bound that holds for any matrix (no two
// peaks are neighbours): needed once M_H is written by something else than
// engine_fill (ht_set_matrix).
ht_status engine_ensure_any_matrix(Engine &E, std::string *why);

// ABI tuning <-> engine: apply (re-deriving the shapes; on failure the old
// tuning is restored, and *poisoned is set if even that fails) / report the
// shapes in use.
ht_status engine_set_tuning(Engine &E, const ht_tuning &t, bool *poisoned, std::string *why);
void engine_get_tuning(const Engine &E, ht_tuning *t);

// Per-kernel totals into the ABI's records (waits for recorded events).
cudaError_t prof_read(Engine &E, ht_kernel_time *out, uint32_t cap, uint32_t *n);

// Allocate the edge-row buffer of peaks-only fills (once; synchronises the
// device the first time).
ht_status engine_ensure_edges(Engine &E, std::string *why);

// Replace the phi edge table (n_phi + 1 pseudo-angles, host memory) on the
// host and on the device (synchronous copy).  A sector context takes its
// slice of the full circle's table, so that it bins hits exactly as the
// unsplit matrix does.
cudaError_t engine_set_phi_edges(Engine &E, const float *ep);

// Step 2 with the 4-D neighbourhood for one event: the 2-D peaks into
// p2 (p2_cap entries, total in *p2_count), then those that also beat their
// neighbours in the adjacent (theta, phi) slices, in order, into out
// (capacity entries, total in *counts).  p2_cap must be >= the engine's
// entry bound (E.scan.entries_cap); keep holds p2_cap flags.
cudaError_t engine_scan4d(Engine &E, htk::Peak *p2, uint8_t *keep, uint32_t p2_cap, uint32_t *p2_count,
                          htk::Peak *out, uint32_t capacity, uint32_t *counts, cudaStream_t st);

// Device status word (bits of htk::ST_*).
inline uint32_t *engine_status(Engine &E) { return E.d_ctr + htk::CTR_STATUS; }

// Counter words of the block (status + counters + per-event counts).
inline uint32_t engine_ctr_words(const Engine &E) { return htk::CTR_EVENTS + E.max_events; }

} // namespace hte
