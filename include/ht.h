/*
 * ht.h -- C ABI of the GB300 Hough-Transform track finder (libht_gb300.so).
 *
 * The method (arXiv 1507.03074, Sec. 2): every hit (x, y, z) votes, for every
 * admitted (theta, phi) bin and every A bin, for the B of the circle
 * x^2 + y^2 - 2Ax - 2By = 0 through the hit and the interaction point; the
 * cell M_H(theta, phi, A, B) is incremented by one.  Cells holding at least
 * `threshold` votes that are local maxima of their (A, B) neighbourhood are the
 * track candidates ("peaks").  Sec. 3 gives the GPU split into a fill step and
 * a maxima step and the transfer of the maxima back to the host.
 *
 * Conventions for every call:
 *   - Status codes: HT_OK (0) or a positive informational code on success,
 *     a negative HT_E_* code on failure.  No call aborts or throws; the
 *     message of the last failure on the calling thread is ht_last_error().
 *   - After HT_E_CUDA a context is poisoned: every later call on it returns
 *     HT_E_STATE (destroy it and create a new one).
 *   - Streams are cudaStream_t passed as void*; NULL means the object's own
 *     (non-blocking) stream.  Calls taking device pointers only enqueue work
 *     on that stream and return; the caller keeps the pointers valid until
 *     the stream has run the work.
 *   - Layout of the vote matrix M_H: uint32 M[theta][phi][A][B], B fastest;
 *     linear index ((itheta*n_phi + iphi)*n_a + ia)*n_b + ib.
 *   - The arithmetic of the vote is fixed (FP32, IEEE round-to-nearest, no
 *     fused multiply-add, in this order) so that results are bit-exact:
 *       dA = (a_max - a_min) / n_a,  dB = (b_max - b_min) / n_b
 *       A_i = a_min + ((float)i + 0.5f) * dA
 *       r2 = x*x + y*y,  d = 2*y
 *       B = (r2 - (2*A_i)*x) / d,  t = (B - b_min) / dB
 *       vote in bin floor(t) iff 0 <= t < n_b (out-of-range and NaN drop).
 *   - Slice admission: the hit's polar angle (from +z) and azimuth select
 *     its (theta, phi) bin, found by comparing FP32 pseudo-angles (built from
 *     + - / sqrt only) with edge tables (see ht_get_edges); +-win_theta and
 *     +-win_phi neighbouring bins are admitted too (phi wraps only when the
 *     phi range is the full circle).  Hits with x = y = 0 are dropped.
 *   - Peak rule: votes >= threshold, and > every one of the 8 (A,B)
 *     neighbours (same slice) with a smaller linear index, and >= every
 *     neighbour with a larger one.  Peaks come in ascending linear index.
 */
#ifndef HT_H
#define HT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ht_ctx ht_ctx;
typedef struct ht_batch ht_batch;
typedef struct ht_server ht_server;
typedef struct ht_sectors ht_sectors;

/* Sizes of M_H (Sec. 2: the four Hough dimensions, binned 4 x 16 x 1024 x
 * 1024 for (theta, phi, A, B)) and the slice admission half-windows.
 * Limits: 1 <= n_theta, n_phi <= 1024; n_theta*n_phi <= 8192;
 * 1 <= n_a, n_b <= 65535; n_theta*n_phi*n_a*n_b < 2^32. */
typedef struct {
    uint32_t n_theta, n_phi, n_a, n_b;
    uint32_t win_theta, win_phi;
} ht_binning;

/* Ranges: theta in [0, pi] (rad, from +z), phi in [-pi, pi] (rad), A and B
 * (mm, the circle centre).  Float endpoints within float rounding of a
 * multiple of pi/4 are taken as that exact multiple.  min < max for all. */
typedef struct {
    float theta_min, theta_max, phi_min, phi_max;
    float a_min, a_max, b_min, b_max;
} ht_ranges;

/* One peak (32 bytes).  a_c, b_c are the cell centres
 * a_min + (ia + 0.5) dA and b_min + (ib + 0.5) dB in FP32. */
typedef struct {
    uint32_t itheta, iphi, ia, ib, votes;
    float a_c, b_c;
    uint32_t event;          /* event index within a batch; 0 otherwise */
} ht_peak;

typedef enum {
    HT_OK = 0,
    HT_PENDING = 1,          /* ht_poll: result not ready before the timeout */
    HT_TRUNCATED = 2,        /* more peaks than capacity; first ones returned */
    HT_E_INVAL = -1,         /* bad argument (NULL, size, range, flag) */
    HT_E_NOMEM = -2,         /* device or pinned allocation failed */
    HT_E_CUDA = -3,          /* a CUDA call or a kernel failed; object poisoned */
    HT_E_BUSY = -4,          /* no admission possible within the memory budget */
    HT_E_TIMEOUT = -5,       /* a bounded device-side wait gave up */
    HT_E_STATE = -6          /* object poisoned by an earlier HT_E_CUDA */
} ht_status;

/* Flags. */
enum {
    HT_MEM_HOST = 0,         /* pointers are host memory (default) */
    HT_MEM_DEVICE = 1,       /* pointers are device memory; call is async */
    HT_ACCUMULATE = 2,       /* ht_fill: add to M_H instead of overwriting it */
    HT_FILL_NAIVE = 4,       /* ht_fill: clear + one global atomic per vote */
    HT_PEAKS_ONLY = 8,       /* ht_fill: find the peaks without writing M_H to device memory */
    HT_MAXIMA_4D = 16        /* ht_find_maxima: the 80-neighbour rule in (theta, phi, A, B) */
};

/* Thread-local text of the last failure (never NULL). */
const char *ht_last_error(void);

/* ------------------------------------------------------------------------ */
/* Single-event context (Sec. 3: one fill kernel, one maxima kernel).        */
/* ------------------------------------------------------------------------ */

/* Create a context on the current CUDA device.  It owns the resident M_H,
 * the sorted-hit workspace for up to max_hits hits per fill (accumulated
 * fills count together), the peak scratch, pinned staging and a stream.
 * threshold >= 1.  Errors: HT_E_INVAL, HT_E_NOMEM, HT_E_CUDA. */
ht_status ht_create(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                    uint32_t max_hits, ht_ctx **out);

/* Wait for the context's work and free everything it owns.  NULL is a no-op. */
ht_status ht_destroy(ht_ctx *ctx);

/* Step 1 (Sec. 2): fill M_H from n_hits hits given as three float arrays
 * (mm).  Unless HT_ACCUMULATE is set M_H is overwritten (cleared in place).
 * HT_MEM_HOST: the hits are copied to pinned staging before the call returns
 * (the caller may reuse its arrays at once).  HT_MEM_DEVICE: device arrays,
 * kept valid by the caller until the stream has run the work.
 * HT_FILL_NAIVE selects the reference-design fill (explicit clear, then one
 * global atomicAdd per vote).  HT_PEAKS_ONLY keeps every vote tile in shared
 * memory: the next ht_find_maxima returns the same peaks, but M_H is left as
 * it was (ht_copy_matrix does not show this fill); not with HT_ACCUMULATE or
 * HT_FILL_NAIVE; the first such fill allocates a small edge-row buffer and
 * waits for the device.  n_hits may be 0 (M_H becomes all zero).
 * Errors: HT_E_INVAL (NULL pointer with n_hits > 0, n_hits > max_hits, or
 * accumulated hits beyond max_hits), HT_E_CUDA, HT_E_STATE. */
ht_status ht_fill(ht_ctx *ctx, const float *x, const float *y, const float *z, uint32_t n_hits,
                  uint32_t flags, void *stream);

/* Step 2 (Sec. 2, Sec. 3): threshold + local-maxima scan of M_H.  A cell
 * with v >= threshold is a peak iff it is > each neighbour with a smaller
 * linear index and >= each one with a larger index; the neighbours are its
 * 8 cells in the (A, B) plane of its (theta, phi) slice, or with
 * HT_MAXIMA_4D the up to 80 cells whose four indices each differ by at
 * most one (phi does not wrap; not after an HT_PEAKS_ONLY fill, whose M_H
 * is not in device memory; the first such call allocates a list buffer and
 * waits for the device).
 * HT_MEM_HOST: blocks until done; writes min(total, capacity) peaks to out
 * and the total to *n_found; returns HT_TRUNCATED if total > capacity.
 * HT_MEM_DEVICE: out (capacity entries) and n_found are device pointers; the
 * call only enqueues; *n_found receives the total (may exceed capacity).
 * Errors: HT_E_INVAL, HT_E_NOMEM, HT_E_CUDA, HT_E_TIMEOUT, HT_E_STATE. */
ht_status ht_find_maxima(ht_ctx *ctx, ht_peak *out, uint32_t capacity, uint32_t *n_found,
                         uint32_t flags, void *stream);

/* Step 2 without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that may not call cudaMalloc / cudaFree --
 * code whose device memory is owned by a framework's caching allocator or a
 * fixed-budget pool (a raw allocation there can fail against, or take from,
 * the pool's reservation), or loops that cannot afford the device-wide
 * synchronisation of cudaFree.  Such callers cannot create an ht_ctx, which
 * allocates M_H and its scratch.
 *
 * M: device, n_events vote matrices of the binning back to back (event e at
 * M + e * n_cells, layout as above); read only.  out: device, n_events *
 * capacity peaks (event e's at out + e * capacity, ascending linear index,
 * the first `capacity` of the event, each with its event number); counts:
 * device, n_events totals (a total above capacity means out holds only the
 * first capacity).  The caller owns all three.  Same peak rule as
 * ht_find_maxima.  stream: cudaStream_t as void*, NULL = the default stream;
 * the call runs its kernels there and returns once they have finished.
 *
 * Scratch: one static device array of 5,267,712 bytes in the library, which
 * every GPU that loads the library holds until the process exits.  Limits:
 * 1 <= n_events <= 4096 (else HT_E_INVAL); at most 262,144 peaks per call in
 * total and 128 chunks of the scan per CTA (else HT_E_NOMEM after the run,
 * with out and counts incomplete).  Every call shares the array and clears
 * its counters first; calls that overlap on the GPU (from several host
 * threads, or on several streams) race on it and must be serialised by the
 * caller.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current).  No cudaMalloc, cudaFree
 * or other allocating call is made.  Errors: HT_E_INVAL (NULL pointer, bad binning, n_events or
 * capacity), HT_E_NOMEM (scratch limit), HT_E_CUDA. */
ht_status ht_find_maxima_noalloc(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                                 const uint32_t *M, uint32_t n_events, ht_peak *out, uint32_t capacity,
                                 uint32_t *counts, void *stream);

/* Measurement helper (no counterpart in the paper): the rate of L2 atomic
 * increments (reductions, result unused) at pseudo-random 4-byte words of a
 * device buffer of footprint_bytes (a power of two, 4 KiB .. 16 GiB),
 * updates_per_thread (1 .. 4096) per thread of 8 CTAs x 256 threads per SM,
 * timed with CUDA events after one warm-up launch on the current device.
 * The roofline the naive fill's votes are compared with.  *updates_per_s
 * receives the rate.  Blocks; allocates and frees the buffer.  Errors:
 * HT_E_INVAL, HT_E_NOMEM, HT_E_CUDA. */
ht_status ht_measure_atomics(uint64_t footprint_bytes, uint32_t updates_per_thread, double *updates_per_s);

/* Admitted (hit, slice) records of the last fill (its unit lists' total
 * length; times n_a: the (hit, slice, A) candidate evaluations).  Waits for
 * the device; 0 before any fill.  Errors: HT_E_INVAL, HT_E_CUDA,
 * HT_E_STATE. */
ht_status ht_last_admitted(ht_ctx *ctx, uint64_t *records);

/* Exercise the failure path of the kernels' bounded waits: one device
 * thread waits on a barrier that nothing completes, gives up after
 * limit_ms (1 .. 1000) and flags the timeout as a real wait would.  Waits
 * for the context's stream; returns HT_E_TIMEOUT (the expected outcome; the
 * context stays usable and its counters are reset), or HT_E_INVAL /
 * HT_E_CUDA / HT_E_STATE. */
ht_status ht_check_wait_timeout(ht_ctx *ctx, uint32_t limit_ms);

/* Wait for the context's stream (or `stream`) and report any device-side
 * failure flagged by its kernels (HT_E_TIMEOUT). */
ht_status ht_sync(ht_ctx *ctx, void *stream);

/* Copy M_H (n_cells must equal the matrix size) to host (HT_MEM_HOST,
 * blocking) or device (HT_MEM_DEVICE, async) memory.  For tests. */
ht_status ht_copy_matrix(ht_ctx *ctx, uint32_t *dst, uint64_t n_cells, uint32_t flags,
                         void *stream);

/* The FP32 pseudo-angle edge tables the context bins hits with (host
 * arrays of n_theta+1 and n_phi+1 floats).  For tests. */
ht_status ht_get_edges(ht_ctx *ctx, float *theta_edges, float *phi_edges);

/* Overwrite M_H with n_cells counters from host (HT_MEM_HOST, blocking) or
 * device (HT_MEM_DEVICE, async) memory, e.g. to run ht_find_maxima on a
 * hand-built matrix.  For tests. */
ht_status ht_set_matrix(ht_ctx *ctx, const uint32_t *src, uint64_t n_cells, uint32_t flags,
                        void *stream);

/* Kernel launches the context has issued since creation (for accounting). */
uint64_t ht_launch_count(const ht_ctx *ctx);

/* Per-kernel device time.  ht_profile(ctx, 1) resets the totals and, from
 * then on, records a pair of CUDA events on the launching stream around
 * every kernel launch of the context; ht_profile(ctx, 0) stops recording.
 * ht_profile_read waits for the recorded events and writes up to cap
 * entries (one per kernel kind: k_prep, k_fill_priv, k_clear, k_fill_naive,
 * k_scan, k_order) with their launch count and summed duration. */
typedef struct {
    char name[32];
    uint64_t launches;
    double total_ms;
} ht_kernel_time;

ht_status ht_profile(ht_ctx *ctx, int enable);
ht_status ht_profile_read(ht_ctx *ctx, ht_kernel_time *out, uint32_t cap, uint32_t *n);

/* Launch shapes.  Every field 0 means automatic; results (M_H and peaks)
 * are identical for every accepted tuning, only the speed changes.
 *   fill_rows          A rows per shared-memory vote tile (power of two)
 *   fill_threads       256, 512 or 1024 threads per fill CTA
 *   fill_hits_staged   hits staged in shared memory per selection chunk
 *   fill_blocks_per_sm cap on resident fill CTAs per SM
 *   scan_kind          HT_SCAN_BULK (1-D bulk-copy ring), HT_SCAN_STREAM
 *                      (register streaming), HT_SCAN_DIRECT (scalar)
 *   scan_stage_bytes   bulk-copy stage size; scan_slots: ring depth (2..8)
 *   scan_blocks_per_sm cap on resident scan CTAs per SM
 *   fill_fused_scan    1: ht_fill also lists the cells >= threshold of each
 *                      vote tile as it writes it (M_H is still written in
 *                      full) and tests only those, so ht_find_maxima only
 *                      orders the peaks; 3: the same with two tiles per SM,
 *                      one voted into while the other is written
 *                      (warp-specialised, 1024 threads); 4: as 1, but each
 *                      tile leaves through two u32 staging buffers in shared
 *                      memory and bulk async copies (cp.async.bulk), so the
 *                      stores drain while the next votes run (1024 threads
 *                      by default; n_b a multiple of 4); 5: as 1 with u32
 *                      tiles in M_H's own layout (fill_rows rows, two in
 *                      rotation), each pass leaving as one bulk async copy
 *                      that no thread converts or stores, the votes listing
 *                      the cells that reach the threshold (n_b a multiple of
 *                      4); 2: never (a full scan in ht_find_maxima); 0: 5
 *                      when n_b is a multiple of 4, else 1, when it fits
 *                      (the fused modes only for non-accumulating, non-naive
 *                      fills)
 *   fill_vote_agg      1: the bulk-copy-tile fill (fill_fused_scan 5)
 *                      aggregates the vote increments of a warp -- lanes
 *                      voting for the same cell find each other and one of
 *                      them adds their number; 0: one shared-memory atomic
 *                      per vote
 *   bin_cluster        1: a fill of at most 16384 hits whose (event, slice)
 *                      units fit the cluster's 40 KB of counts (3 words per
 *                      unit and 1 per event: up to 53 events of 64 slices)
 *                      bins them and builds the unit lists in one launch of
 *                      a thread-block cluster (up to 8 CTAs of 1024 threads
 *                      reading each other's counts), which also splits the
 *                      work of the fill after it (bulk-copy-tile or
 *                      peaks-only) ahead of it -- shorter latency of one
 *                      event; larger fills take two launches anyway; 2: two
 *                      launches (binning, lists) of small CTAs that fit
 *                      beside other events' kernels -- more events per
 *                      second when several contexts' events overlap; 0: 1
 *                      for the bulk-copy-tile and the peaks-only fill
 *                      unless fill_blocks_per_sm holds that fill below the
 *                      CTAs per SM that fit (the SMs are then shared with
 *                      other events), else 2
 * ht_set_tuning waits for the device, re-derives the shapes and returns
 * HT_E_INVAL for an impossible value; ht_get_tuning reports the shapes in
 * effect (0 fields filled in). */
enum { HT_SCAN_AUTO = 0, HT_SCAN_BULK = 1, HT_SCAN_STREAM = 2, HT_SCAN_DIRECT = 3 };
typedef struct {
    uint32_t fill_rows, fill_threads, fill_hits_staged, fill_blocks_per_sm;
    uint32_t scan_kind, scan_stage_bytes, scan_slots, scan_blocks_per_sm;
    uint32_t fill_fused_scan;
    uint32_t fill_vote_agg;
    uint32_t bin_cluster;
} ht_tuning;

ht_status ht_set_tuning(ht_ctx *ctx, const ht_tuning *tuning);
ht_status ht_get_tuning(ht_ctx *ctx, ht_tuning *tuning);

/* Autotuner: re-runs the hits of the last (non-accumulating) ht_fill under
 * candidate launch shapes -- fused or two-kernel fill, tile rows, threads,
 * scan variant -- reps times each, and keeps the fastest.  M_H and the
 * result of a following ht_find_maxima are those of the last fill.  chosen
 * (may be NULL) receives the shapes in effect, us_per_event (may be NULL)
 * the device time per event of fill + maxima.  Blocks.  Errors: HT_E_INVAL
 * (no fill yet, or the last fill accumulated), HT_E_CUDA, HT_E_NOMEM. */
ht_status ht_autotune(ht_ctx *ctx, uint32_t reps, ht_tuning *chosen, double *us_per_event);

/* ------------------------------------------------------------------------ */
/* Batches: many independent events in one fill + maxima launch sequence.   */
/* ------------------------------------------------------------------------ */
/* The paper processes its events one after another (Sec. 4); the
 * arithmetic of each event here is unchanged (an event's M_H and peaks are
 * identical alone and in any batch).  A batch holds max_events resident
 * vote matrices (event e at e * n_cells), device staging for max_hits hits
 * in total and room for `capacity` peaks over the whole batch.  Each run
 * enqueues the hit copies, then the kernels of steps 1 and 2 for all events
 * at once: a CUDA graph captured for that event count on the first run with
 * it (later runs with the same count replay it), then the result copies. */
ht_status ht_batch_create(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                          uint32_t max_events, uint32_t max_hits, uint32_t capacity, ht_batch **out);
ht_status ht_batch_destroy(ht_batch *batch);

/* Steps 1 + 2 for n_events (1..max_events) events whose hits are
 * concatenated: event e owns hits [hit_off[e], hit_off[e+1]) of x, y, z,
 * with hit_off[0] = 0 and hit_off[n_events] = n_hits <= max_hits.
 * Peaks come in one list ordered by (event, linear index), each with its
 * event number: event e's at out + sum of counts[e' < e] as long as the
 * total fits `capacity` (the batch's); counts[e] is event e's total.
 * HT_MEM_HOST: every array is host memory (the caller may reuse them on
 * return: hits in page-locked memory are copied to the device directly,
 * others through the batch's pinned staging); blocks; writes min(total,
 * capacity) peaks and returns HT_TRUNCATED when the total exceeds capacity.
 * HT_MEM_DEVICE: every array (hit_off included) is device memory; the call
 * only enqueues on `stream` (NULL = the batch's own stream); the caller
 * checks counts for truncation; ht_batch_sync reports device-side failures.
 * HT_PEAKS_ONLY: the same peaks without writing the matrices (as ht_fill;
 * the first such run allocates the edge rows and waits for the device;
 * ht_batch_copy_matrix does not show such a run).
 * HT_FILL_NAIVE: the paper's fill for every event (as ht_fill: clear, then
 * one global atomic per vote; the same matrices and peaks); not with
 * HT_PEAKS_ONLY.
 * Errors: HT_E_INVAL, HT_E_CUDA (batch poisoned), HT_E_NOMEM (peak scratch),
 * HT_E_TIMEOUT, HT_E_STATE. */
ht_status ht_batch_run(ht_batch *batch, const float *x, const float *y, const float *z, const uint32_t *hit_off,
                       uint32_t n_events, uint32_t n_hits, ht_peak *out, uint32_t *counts, uint32_t flags,
                       void *stream);
ht_status ht_batch_sync(ht_batch *batch, void *stream);

/* Copy event e's M_H from the last run (n_cells cells) to host memory
 * (blocking).  For tests. */
ht_status ht_batch_copy_matrix(ht_batch *batch, uint32_t event, uint32_t *dst, uint64_t n_cells);

/* Launch shapes of the batch (see ht_tuning); drops the captured graphs. */
ht_status ht_batch_set_tuning(ht_batch *batch, const ht_tuning *tuning);
ht_status ht_batch_get_tuning(ht_batch *batch, ht_tuning *tuning);

/* ht_autotune for a batch: times candidate shapes on the hits of the last
 * run (its events), keeps the fastest and drops the captured graphs; the
 * result of the last run stays valid.  us_per_event is the device time of
 * fill + maxima per event.  Blocks. */
ht_status ht_batch_autotune(ht_batch *batch, uint32_t reps, ht_tuning *chosen, double *us_per_event);

/* Per-kernel device times of the batch's runs that are not replayed from a
 * graph (see ht_profile; with profiling on, runs do not use graphs). */
ht_status ht_batch_profile(ht_batch *batch, int enable);
ht_status ht_batch_profile_read(ht_batch *batch, ht_kernel_time *out, uint32_t cap, uint32_t *n);

/* ------------------------------------------------------------------------ */
/* Serving: a request loop with continuous batching.                         */
/* ------------------------------------------------------------------------ */
/* Not in the paper (its events are processed one after another, Sec. 4);
 * the arithmetic of every event is unchanged: a request's peaks are those
 * ht_find_maxima returns for the event alone.  ht_submit copies the hits and
 * returns at once.  A worker thread keeps "lanes": for one (binning,
 * ranges, threshold) a lane holds the resident vote matrices of a
 * micro-batch of events, staging and its own stream.  Whenever a lane is
 * free the worker takes the waiting requests of its binning (oldest first,
 * up to max_batch events and the lane's hit room) and runs them as one
 * batch; lanes of several binnings and several lanes of one binning run at
 * the same time.  A lane is created when a request needs one and its device
 * memory fits hbm_budget_bytes (idle lanes of other binnings are freed to
 * make room); otherwise the request waits for a lane.  M_H stays resident
 * in a lane and is overwritten in place by every fill. */
typedef struct {
    uint64_t hbm_budget_bytes;   /* device memory for all lanes; 0 = 80% of the free memory at creation */
    uint32_t n_streams;          /* lanes per binning (micro-batches in flight); 0 = 4 */
    uint32_t max_batch;          /* events per micro-batch; 0 = 16 */
    uint32_t max_hits_per_event; /* 0 = 65536 */
    uint32_t queue_depth;        /* waiting requests before ht_submit answers HT_E_BUSY; 0 = 65536 */
    uint32_t flags;              /* 0, or HT_PEAKS_ONLY: every micro-batch runs peaks-only fills (the
                                    same peaks; the lanes' matrices are not written) */
    uint32_t fill_blocks_per_sm; /* fill CTAs per SM in every lane, 0 = the engine's choice (2 on
                                    GB300); 1 lets the fills of micro-batches in flight on
                                    several lanes share every SM; at most 32 */
} ht_server_cfg;

/* Create on the current CUDA device (cfg NULL = all defaults). */
ht_status ht_server_create(const ht_server_cfg *cfg, ht_server **out);
/* Finishes the requests on the GPU, drops the waiting ones, frees all lanes. */
ht_status ht_server_destroy(ht_server *server);

/* Queue one event (host arrays, copied before return).  *ticket names it
 * for ht_poll.  Errors: HT_E_INVAL (binning, n_hits > max_hits_per_event,
 * NULL), HT_E_BUSY (queue_depth requests already waiting), HT_E_STATE. */
ht_status ht_submit(ht_server *server, const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                    const float *x, const float *y, const float *z, uint32_t n_hits, uint64_t *ticket);

/* Wait up to timeout_us for the request's result; HT_PENDING if it is not
 * ready by then (the ticket stays valid).  On completion writes
 * min(total, capacity) peaks (event field 0) to out and the total to
 * *n_found, forgets the ticket and returns HT_OK, HT_TRUNCATED (total >
 * capacity, or more peaks than its micro-batch could hold), or the
 * request's error (HT_E_NOMEM: its matrix never fits the budget).
 * HT_E_INVAL for an unknown ticket. */
ht_status ht_poll(ht_server *server, uint64_t ticket, ht_peak *out, uint32_t capacity, uint32_t *n_found,
                  uint32_t timeout_us);

/* Counters; latency = submit to result ready (host steady clock) over the
 * requests completed since the last reset (reset != 0 restarts them). */
typedef struct {
    uint64_t submitted, completed, waiting, in_flight;
    uint64_t micro_batches;      /* dispatched micro-batches */
    double mean_batch;           /* events per micro-batch */
    uint32_t lanes;
    uint64_t lane_bytes;         /* device memory held by the lanes */
    double p50_us, p99_us, mean_us, max_us;
} ht_server_stats;
ht_status ht_server_get_stats(ht_server *server, ht_server_stats *stats, int reset);

/* ------------------------------------------------------------------------ */
/* Host-only helpers (no device needed).                                     */
/* ------------------------------------------------------------------------ */

/* HT_OK if (binning, ranges, threshold) is accepted by ht_create, else
 * HT_E_INVAL with the reason in ht_last_error(). */
ht_status ht_validate(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold);

/* The FP32 pseudo-angle edge tables of a binning (what ht_get_edges of a
 * context with these arguments returns): n_theta+1 and n_phi+1 floats.
 * Edge k is the pseudo-angle of the k-th uniform angle edge, evaluated in
 * double and rounded once; multiples of pi/4 are exact. */
ht_status ht_compute_edges(const ht_binning *binning, const ht_ranges *ranges, float *theta_edges,
                           float *phi_edges);

/* The B-bin thresholds the kernels use (n_b + 1 floats): beta[k] is the
 * smallest float B whose bin floor(fl(fl(B - b_min) / dB)) is >= k, so a vote
 * is in range iff beta[0] <= B < beta[n_b] and its bin is the number of
 * beta[1..n_b-1] that are <= B -- identical to the division rule for every
 * float B. */
ht_status ht_compute_b_thresholds(const ht_binning *binning, const ht_ranges *ranges, float *beta);

/* ------------------------------------------------------------------------ */
/* Phi sectors (Sec. 4).                                                     */
/* ------------------------------------------------------------------------ */

/* Sec. 4 splits the transverse plane into phi sectors that are read out
 * independently, runs one Hough transform with its own M_H(A, B, theta) per
 * sector and merges the results.  Here the n_sectors sectors are contexts on
 * the current device, each on its own stream: sector k owns phi bins
 * [k m, (k + 1) m) of the binning (m = n_phi / n_sectors), with exactly the
 * unsplit binning's edges for them, so its matrix equals those phi bins of
 * the unsplit M_H and the merged peaks equal the unsplit peaks.
 * Requirements: n_phi % n_sectors == 0 and win_phi == 0 (a phi window would
 * need the neighbouring sector's hits); otherwise as ht_create.  max_hits
 * bounds one fill.  Errors: HT_E_INVAL, HT_E_NOMEM, HT_E_CUDA. */
ht_status ht_sectors_create(const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                            uint32_t n_sectors, uint32_t max_hits, ht_sectors **out);

/* Wait for the sectors' work and free everything.  NULL is a no-op. */
ht_status ht_sectors_destroy(ht_sectors *sec);

/* Step 1 for every sector: the hits (flags and memory as ht_fill; every
 * sector receives all n_hits hits and keeps those in its phi range, as a
 * sector's own read-out would deliver them) are voted by the n_sectors
 * contexts concurrently, forked from and joined back into `stream` (NULL =
 * the object's stream).  HT_MEM_HOST copies the hits once to pinned staging
 * and one device copy before returning.  Flags: HT_MEM_DEVICE,
 * HT_ACCUMULATE, HT_FILL_NAIVE, HT_PEAKS_ONLY.  Errors as ht_fill. */
ht_status ht_sectors_fill(ht_sectors *sec, const float *x, const float *y, const float *z, uint32_t n_hits,
                          uint32_t flags, void *stream);

/* Step 2 for every sector, concurrently, then the merge: the sectors' peaks
 * in the unsplit binning's numbering (iphi + k m) and ascending linear
 * index of the unsplit M_H.  Memory, capacity and truncation as
 * ht_find_maxima (HT_MEM_DEVICE: out and n_found on the device, enqueued
 * only).  Errors as ht_find_maxima. */
ht_status ht_sectors_find_maxima(ht_sectors *sec, ht_peak *out, uint32_t capacity, uint32_t *n_found,
                                 uint32_t flags, void *stream);

/* Copy sector k's matrix (n_theta x m x n_a x n_b cells) to host memory;
 * waits for the object's work.  Errors: HT_E_INVAL, HT_E_CUDA. */
ht_status ht_sectors_copy_matrix(ht_sectors *sec, uint32_t sector, uint32_t *dst, uint64_t n_cells);

/* ------------------------------------------------------------------------ */
/* Track read-out (host, FP64; no device needed).                            */
/* ------------------------------------------------------------------------ */

/* The track parameters of one peak (Sec. 2, Fig. 1).  (a, b) is the centre
 * of the peak's (A, B) cell, a_min + (ia + 0.5) (a_max - a_min) / n_a and
 * likewise for b, evaluated in double from the FP32 ranges; rho =
 * sqrt(a^2 + b^2) is the circle radius and varphi = atan2(b, a) the azimuth
 * of the circle centre (the paper's tan^-1(B/A), read over all four
 * quadrants); pt = 0.3 * b_field * rho / 1000 is the transverse momentum
 * (GeV) of a unit charge in a solenoid of b_field tesla (rho in mm).  theta
 * is the centre of the peak's polar-angle bin, theta_min + (itheta + 0.5)
 * (theta_max - theta_min) / n_theta, and eta = -ln tan(theta / 2); phi_c
 * the centre of its azimuth bin. */
typedef struct {
    double a, b;             /* mm */
    double rho;              /* mm */
    double varphi;           /* rad, in [-pi, pi] */
    double pt;               /* GeV */
    double theta, eta, phi_c;
    uint32_t votes, event;   /* copied from the peak */
} ht_track;

/* Read out n peaks (host memory) into out[0 .. n) (host memory, caller-
 * owned).  HT_E_INVAL (nothing written) for a NULL pointer with n > 0, an
 * invalid binning or ranges, b_field_t not finite and > 0, or a peak whose
 * cell lies outside the binning. */
ht_status ht_track_params(const ht_binning *binning, const ht_ranges *ranges, const ht_peak *peaks, uint32_t n,
                          double b_field_t, ht_track *out);

#ifdef __cplusplus
}
#endif

#endif /* HT_H */
