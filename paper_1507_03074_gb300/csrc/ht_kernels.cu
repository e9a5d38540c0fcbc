// Hough-Transform kernels for sm_103a (GB300).
//
//   k_bin         one thread per hit (all events of a launch): the bin code
//                 of the hit's own (theta, phi) slice, found from FP32
//                 pseudo-angles and the edge tables (Sec. 2: the angles
//                 select the slice a hit votes in), and the per-hit terms
//                 x, x^2 + y^2, 2y of the vote.
//   k_scatter     the admitted hits into per-(event, slice) unit lists.
//   k_bin_cluster k_bin + k_scatter in one thread-block cluster for launches
//                 of few hits (distributed shared memory for the counts),
//                 which also writes the work split of the fill after it.
//   k_fill_tma    Step 1 fused with the candidates of step 2 (default): the
//                 votes of a pass of W A-rows go into a u32 shared-memory
//                 tile laid out as M_H's rows, the tile leaves as one bulk
//                 copy, and a vote taking a cell to T lists it.  k_peaks then
//                 tests the listed cells against their neighbours.
//   k_fill_priv   Step 1 (Sec. 2), privatised.  Work item = (event, slice,
//                 strip of W A-rows); each CTA takes a contiguous range of
//                 items.  It selects the event's hits admitted to the slice
//                 (ballot compaction into shared memory, cached while the
//                 CTA stays on that slice), votes them into a shared-memory
//                 u16 (or u32) tile with shared-memory atomics, and writes
//                 the tile to HBM once with 16-byte stores that also zero it.
//                 Every cell is written, so M_H needs no separate clear.
//   k_clear,      Step 1 as the paper's CUDA design (Sec. 3): an explicit
//   k_fill_naive  clear, then a 1-D grid over hits, a thread block over A,
//                 and one global atomicAdd per vote.
//   k_scan_tma    Step 2 (Sec. 2, Sec. 3): threshold + local maxima.  Each
//                 persistent CTA streams a contiguous run of M_H rows through
//                 a ring of shared-memory stages filled by 1-D bulk copies
//                 (TMA, mbarrier-completed).  A stage with no cell >= T (the
//                 common case) costs one 16-byte load per thread and row and
//                 one block vote; only stages holding candidates check the 8
//                 (A,B) neighbours and compact peaks, in order, into per-CTA
//                 chunks.  k_scan_direct is the same without staging, for
//                 n_b not a multiple of 4.
//   k_order       places every list's chunks at their global rank: ascending
//                 linear index per event, expanded to 32-byte peak records.
#include "ht_device.cuh"
#include "ht_internal.h"

#include <cooperative_groups.h>

#include <atomic>
#include <utility>

namespace htk {

// ---------------------------------------------------------------------------
// Block-wide helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += n;
    }
    return v;
}

// Thread groups that share the block-level helpers below: the whole block
// (barrier 0), or a warp-aligned range of FIRST .. FIRST + N - 1 threads
// synchronising on named barrier ID (the warp-specialised fill runs two
// such groups side by side, each with its own barrier).
struct BlockGroup {
    static __device__ __forceinline__ uint32_t rank() { return threadIdx.x; }
    static __device__ __forceinline__ uint32_t size() { return blockDim.x; }
    static __device__ __forceinline__ void sync() { __syncthreads(); }
    static __device__ __forceinline__ int sync_or(int p) { return __syncthreads_or(p); }
};

template <uint32_t ID, uint32_t FIRST, uint32_t N>
struct WarpGroup {
    static_assert(FIRST % 32 == 0 && N % 32 == 0 && ID >= 1 && ID < 16, "warp-aligned group, named barrier 1..15");
    static __device__ __forceinline__ uint32_t rank() { return threadIdx.x - FIRST; }
    static __device__ __forceinline__ uint32_t size() { return N; }
    static __device__ __forceinline__ void sync() { asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(N) : "memory"); }
    static __device__ __forceinline__ int sync_or(int p)
    {
        uint32_t r;
        asm volatile("{\n\t.reg .pred pi, po;\n\t"
                     "setp.ne.u32 pi, %1, 0;\n\t"
                     "bar.red.or.pred po, %2, %3, pi;\n\t"
                     "selp.u32 %0, 1, 0, po;\n\t}"
                     : "=r"(r)
                     : "r"((uint32_t)p), "n"(ID), "n"(N)
                     : "memory");
        return (int)r;
    }
};

// Programmatic dependent launch: every kernel here is launched so that it may
// start while the previous kernel of its stream finishes; it runs only
// set-up that touches no global data of earlier kernels before this wait
// (a no-op when the launch had no such dependency).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel of the stream launch once every CTA of this one has
// passed this point (its grid_dep_wait still waits for this kernel to end).
// Only k_scatter uses it, after its own wait: what k_bin wrote is then
// complete when the fill after k_scatter starts, so the fill may read the
// unit offsets before its own wait.
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Exclusive scan of n values in shared memory (in place); returns the total.
// All threads of the block must call it.  wsum: >= 33 words of scratch.
__device__ uint32_t block_exclusive_scan(uint32_t *a, uint32_t n, uint32_t *wsum)
{
    const uint32_t tid = threadIdx.x, bd = blockDim.x;
    const uint32_t per = (n + bd - 1) / bd;
    const uint32_t b0 = min(tid * per, n), b1 = min(b0 + per, n);
    uint32_t s = 0;
    for (uint32_t i = b0; i < b1; ++i)
        s += a[i];
    const uint32_t incl = warp_incl_scan(s);
    const uint32_t warp = tid >> 5, lane = tid & 31u, nw = (bd + 31) >> 5;
    if (lane == 31u)
        wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < nw ? wsum[lane] : 0u;
        const uint32_t vi = warp_incl_scan(v);
        wsum[lane] = vi - v;
        if (lane == 31u)
            wsum[32] = vi;
    }
    __syncthreads();
    uint32_t run = wsum[warp] + incl - s;
    for (uint32_t i = b0; i < b1; ++i) {
        const uint32_t v = a[i];
        a[i] = run;
        run += v;
    }
    const uint32_t total = wsum[32];
    __syncthreads();
    return total;
}

// ---------------------------------------------------------------------------
// k_bin: one thread per hit.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bin(Geom g, Work w)
{
    __shared__ float et[1025], ep[1025];
    __shared__ uint32_t s_last, s_wsum[40];
    extern __shared__ uint32_t s_off[];   // n_events + 1 hit offsets (batches)
    const uint32_t tid = threadIdx.x, bd = blockDim.x;
    for (uint32_t i = tid; i <= g.nt; i += bd)
        et[i] = g.et[i];
    for (uint32_t i = tid; i <= g.np; i += bd)
        ep[i] = g.ep[i];
    grid_dep_wait();   // counters and hits of earlier kernels
    if (blockIdx.x == 0) {   // fresh counters for the fill and scan that follow
        if (tid == 0)
            w.ctr[CTR_ENTRIES] = w.ctr[CTR_OTICKET] = 0u;
        for (uint32_t i = tid; i < w.n_events; i += bd)
            w.ctr[CTR_EVENTS + i] = 0u;
    }
    if (w.hit_off)
        for (uint32_t i = tid; i <= w.n_events; i += bd)
            s_off[i] = w.hit_off[i];
    __syncthreads();
    const uint32_t n = w.hit_off ? min(s_off[w.n_events], w.n_hits0) : w.n_hits0;
    for (uint32_t h = blockIdx.x * bd + tid; h < n; h += gridDim.x * bd) {
        const float x = w.x[h], y = w.y[h];
        float r2;
        const uint32_t code = bin_code(g, et, ep, x, y, w.z[h], r2);
        uint32_t e = 0;
        if (w.hit_off) {   // the last event whose first hit is <= h
            uint32_t lo = 0, hi = w.n_events - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= h)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            e = lo;
        }
        w.hits4[h] = make_float4(x, r2, __fmul_rn(2.0f, y), __uint_as_float(e));
        w.codes[h] = code;
        for_each_slice(g, code, [&](uint32_t s) { atomicAdd(&w.slice_cnt[e * g.n_slices + s], 1u); });
    }
    // the last block to finish turns the counts into unit offsets
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&w.ctr[CTR_BTICKET], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    const uint32_t U = w.n_events * g.n_slices;
    constexpr uint32_t PER = 8;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < U; base += PER * bd) {
        uint32_t v[PER], sum = 0;
#pragma unroll
        for (uint32_t q = 0; q < PER; ++q) {
            const uint32_t u = base + tid * PER + q;
            v[q] = u < U ? __ldcg(&w.slice_cnt[u]) : 0u;
            sum += v[q];
        }
        const uint32_t incl = warp_incl_scan(sum);
        const uint32_t warp = tid >> 5, lane = tid & 31u, nw = (bd + 31) >> 5;
        if (lane == 31u)
            s_wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t t = lane < nw ? s_wsum[lane] : 0u;
            const uint32_t ti = warp_incl_scan(t);
            s_wsum[lane] = ti - t;
            if (lane == 31u)
                s_wsum[32] = ti;
        }
        __syncthreads();
        uint32_t run = carry + s_wsum[warp] + incl - sum;
#pragma unroll
        for (uint32_t q = 0; q < PER; ++q) {
            const uint32_t u = base + tid * PER + q;
            if (u < U) {
                w.slice_off[u] = run;
                w.slice_fill[u] = 0u;
            }
            run += v[q];
        }
        carry += s_wsum[32];
        __syncthreads();
    }
    if (tid == 0) {
        w.slice_off[U] = carry;
        w.ctr[CTR_BTICKET] = 0u;
    }
}

// Hits into their units' lists (after k_bin), then clear the unit counts
// for the next binning.
__global__ void __launch_bounds__(256) k_scatter(Geom g, Work w)
{
    grid_dep_wait();
    grid_dep_launch();   // k_bin is complete: the fill may start its set-up
    const uint32_t n = w.hit_off ? min(__ldg(&w.hit_off[w.n_events]), w.n_hits0) : w.n_hits0;
    const uint32_t stride = gridDim.x * blockDim.x, t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t h = t0; h < n; h += stride) {
        const uint32_t code = w.codes[h];
        if (code == kDropped)
            continue;
        const float4 hv = w.hits4[h];
        const uint32_t e = __float_as_uint(hv.w);
        for_each_slice(g, code, [&](uint32_t s) {
            const uint32_t u = e * g.n_slices + s;
            const uint32_t idx = w.slice_off[u] + atomicAdd(&w.slice_fill[u], 1u);
            if (idx < w.list_cap)
                w.list[idx] = hv;
        });
    }
    const uint32_t U = w.n_events * g.n_slices;
    for (uint32_t u = t0; u < U; u += stride)
        w.slice_cnt[u] = 0u;
}

// The static split of the fill that follows (the split cta_items computes,
// for the shape Work::split_* names), from unit offsets off[0..U) in shared
// memory and their total: split[c] = the first static item of fill CTA c.
// Work item cost as in cta_items: g.na * (g.nb * u + vote weight * off[u])
// up to unit u, strictly increasing in u; a CTA boundary at cost T falls in
// the unit u with cost(u) <= T < cost(u + 1), at the strip it reaches.
// Int: the arithmetic type, uint32_t when every cost (and G * G) is below
// 2^31, which spares the 64-bit divisions.
template <typename Int>
__device__ __forceinline__ void split_for_fill_t(const Geom &g, const Work &w, const uint32_t *off, uint32_t total,
                                                 uint64_t tot64)
{
    const uint32_t U = w.n_events * g.n_slices, G = w.split_grid, S = w.split_strips;
    const uint64_t ns = w.split_n_static;
    auto cost = [&](uint32_t u) {
        return (Int)((uint64_t)g.na * ((uint64_t)g.nb * u + (uint64_t)w.split_vw * (u < U ? off[u] : total)));
    };
    const Int tot = (Int)tot64, c_end = cost(U), q = tot / G, r = tot % G;
    for (uint32_t c = threadIdx.x; c <= G; c += blockDim.x) {
        uint64_t item = ns;
        if (c == 0) {
            item = 0;
        } else if (c < G) {
            const Int T = q * c + (r * c) / G;
            if (T < c_end) {
                uint32_t lo = 0, hi = U - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (cost(mid) <= T)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                const Int a = cost(lo), b = cost(lo + 1);
                const Int per = (b - a + S - 1) / S;
                const Int k = (T - a) / per;
                item = min((uint64_t)lo * S + min((uint64_t)k, (uint64_t)S - 1), ns);
            }
        }
        w.split[c] = item;
    }
}

__device__ void split_for_fill(const Geom &g, const Work &w, const uint32_t *off, uint32_t total)
{
    const uint32_t U = w.n_events * g.n_slices, G = w.split_grid, S = w.split_strips;
    const uint64_t ns = w.split_n_static;
    auto cost = [&](uint32_t u) {
        return (uint64_t)g.na * ((uint64_t)g.nb * u + (uint64_t)w.split_vw * (u < U ? off[u] : total));
    };
    const bool small = cost(U) < (1ull << 31) && ns < (1ull << 31) && (uint64_t)G * (G + 1) < (1ull << 31) &&
                       S < (1u << 30);
    // the cost of the first ns items
    uint64_t tot;
    if (small) {
        const uint32_t n32 = (uint32_t)ns, us = n32 / S, ks = n32 % S;
        uint32_t t = (uint32_t)cost(us);
        if (ks)
            t += ks * (((uint32_t)cost(us + 1) - t + S - 1) / S);
        tot = t;
    } else {
        const uint32_t us = (uint32_t)(ns / S), ks = (uint32_t)(ns % S);
        tot = cost(us);
        if (ks)
            tot += ks * ((cost(us + 1) - tot + S - 1) / S);
    }
    if (small)
        split_for_fill_t<uint32_t>(g, w, off, total, tot);
    else
        split_for_fill_t<uint64_t>(g, w, off, total, tot);
}

// k_bin and k_scatter in one launch for launches of few hits: one cluster of
// up to kBinClusterMax CTAs.  Each CTA counts its hits per unit in its own
// shared memory; after one cluster barrier every CTA reads all the CTAs'
// counts (distributed shared memory) and derives by itself the unit totals,
// its own place inside every unit (the counts of the CTAs ranked below it)
// and, by an exclusive scan of the totals, the unit offsets.  It then lists
// its hits with local cursors.  No CTA writes another's shared memory, and
// the only other cluster barrier (split into arrive and wait) keeps every
// CTA's counts alive until all have read them.  Each thread keeps its (at
// most kBinClusterHPT) hits in registers between counting and listing.
// Dynamic shared memory: U counts, U + 1 totals / offsets, U places and
// n_events + 1 hit offsets, where U = n_events * n_slices.
__global__ void __launch_bounds__(1024, 1) k_bin_cluster(Geom g, Work w)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ float et[1025], ep[1025];
    __shared__ uint32_t s_wsum[40];
    extern __shared__ uint32_t s_cnt[];
    const uint32_t tid = threadIdx.x, bd = blockDim.x;
    const uint32_t rank = cl.block_rank(), cs = cl.num_blocks();
    const uint32_t U = w.n_events * g.n_slices;
    uint32_t *s_tot = s_cnt + U, *s_pl = s_tot + U + 1, *s_off = s_pl + U;
    for (uint32_t i = tid; i <= g.nt; i += bd)
        et[i] = g.et[i];
    for (uint32_t i = tid; i <= g.np; i += bd)
        ep[i] = g.ep[i];
    for (uint32_t u = tid; u < U; u += bd)
        s_cnt[u] = 0u;
    grid_dep_wait();     // counters and hits of earlier kernels
    grid_dep_launch();   // the fill's set-up overlaps; it waits for this grid's end
    if (rank == 0) {   // fresh counters for the fill and scan that follow
        if (tid == 0)
            w.ctr[CTR_ENTRIES] = w.ctr[CTR_OTICKET] = 0u;
        for (uint32_t i = tid; i < w.n_events; i += bd)
            w.ctr[CTR_EVENTS + i] = 0u;
    }
    if (w.hit_off)
        for (uint32_t i = tid; i <= w.n_events; i += bd)
            s_off[i] = w.hit_off[i];
    __syncthreads();
    const uint32_t n = w.hit_off ? min(s_off[w.n_events], w.n_hits0) : w.n_hits0;
    uint32_t code[kBinClusterHPT], ev[kBinClusterHPT];
    float4 hv[kBinClusterHPT];
#pragma unroll
    for (uint32_t q = 0; q < kBinClusterHPT; ++q) {
        const uint32_t h = (q * cs + rank) * bd + tid;
        code[q] = kDropped;
        ev[q] = 0u;
        hv[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (h < n) {
            const float x = __ldg(&w.x[h]), y = __ldg(&w.y[h]);
            float r2;
            code[q] = bin_code(g, et, ep, x, y, __ldg(&w.z[h]), r2);
            if (w.hit_off) {   // the last event whose first hit is <= h
                uint32_t lo = 0, hi = w.n_events - 1;
                while (lo < hi) {
                    const uint32_t mid = (lo + hi + 1) >> 1;
                    if (s_off[mid] <= h)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                ev[q] = lo;
            }
            hv[q] = make_float4(x, r2, __fmul_rn(2.0f, y), __uint_as_float(ev[q]));
            const uint32_t e = ev[q];
            for_each_slice(g, code[q], [&](uint32_t s) { atomicAdd(&s_cnt[e * g.n_slices + s], 1u); });
        }
    }
    cl.sync();   // every CTA's counts are complete (and every CTA of the cluster runs)
    const uint32_t *r_cnt[kBinClusterMax];
#pragma unroll
    for (uint32_t r = 0; r < kBinClusterMax; ++r)
        r_cnt[r] = cl.map_shared_rank(s_cnt, r < cs ? r : 0u);
    for (uint32_t u = tid; u < U; u += bd) {
        uint32_t c[kBinClusterMax];
#pragma unroll
        for (uint32_t r = 0; r < kBinClusterMax; ++r)
            c[r] = r < cs ? r_cnt[r][u] : 0u;
        uint32_t tot = 0, below = 0;
#pragma unroll
        for (uint32_t r = 0; r < kBinClusterMax; ++r) {
            below += r < rank ? c[r] : 0u;
            tot += c[r];
        }
        s_tot[u] = tot;
        s_pl[u] = below;
    }
    // done with the other CTAs' counts: arrive now, wait before exiting, so
    // that every CTA's shared memory outlives every read of it
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    __syncthreads();
    const uint32_t total = block_exclusive_scan(s_tot, U, s_wsum);   // totals -> unit offsets
    if (tid == 0)
        s_tot[U] = total;
    for (uint32_t u = tid; u < U; u += bd) {
        s_pl[u] += s_tot[u];   // this CTA's first list index in unit u
        if (rank == 0)
            w.slice_off[u] = s_tot[u];
    }
    if (rank == 0 && tid == 0)
        w.slice_off[U] = total;
    __syncthreads();
#pragma unroll
    for (uint32_t q = 0; q < kBinClusterHPT; ++q) {
        const uint32_t e = ev[q];
        for_each_slice(g, code[q], [&](uint32_t s) {
            const uint32_t idx = atomicAdd(&s_pl[e * g.n_slices + s], 1u);
            if (idx < w.list_cap)
                w.list[idx] = hv[q];
        });
    }
    if (rank == 0 && w.split_mode == kSplitGiven)
        split_for_fill(g, w, s_tot, total);
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// k_fill_priv
// ---------------------------------------------------------------------------
// Row swizzle inside 32-word blocks of the shared tile: spreads the banks
// of a warp whose lanes (consecutive A rows) vote into the same B column.
__device__ __forceinline__ uint32_t row_hash(uint32_t r)
{
    return (r * 0x9E3779B9u) >> 27;  // 5 bits
}

// Cells >= T of one pass: hot[] marks their rows (bit r of word r / 32),
// cand[] lists them as r * n_b + j (up to cap; *n counts them all), candv[]
// holds their votes where the lister knows them.
struct FlushList {
    uint32_t *hot;
    uint32_t *cand;     // r * n_b + j
    uint32_t *candv;    // the cell's votes
    uint32_t *n;
    uint32_t cap;
};

// Votes of tile cell (r, j) (u16 or u32 counters, row swizzle as vote_rows).
__device__ __forceinline__ uint32_t tile_cell(const uint32_t *tile, uint32_t pitch, bool u16, uint32_t r, uint32_t j)
{
    if (u16)
        return (tile[r * pitch + ((j >> 1) ^ (row_hash(r) & 0x1Eu))] >> ((j & 1u) << 4)) & 0xffffu;
    return tile[r * pitch + (j ^ (row_hash(r) & 0x1Cu))];
}

// A cell of row r that just reached T: mark the row, list the cell.
__device__ __forceinline__ void note_candidate(const FlushList &L, uint32_t r, uint32_t key)
{
    atomicOr(&L.hot[r >> 5], 1u << (r & 31u));
    const uint32_t p = atomicAdd(L.n, 1u);
    if (p < L.cap)
        L.cand[p] = key;
}

// Votes of hits hs[hl], hs[hl + hstride], .. < nc into tile row r (A bin i).
// With LIST, a vote that lifts its cell from T - 1 to T lists the cell
// (note_candidate): votes are +1 increments and T >= 1 (the context
// rejects T = 0), so every cell >= T is listed exactly once.
template <bool U16, bool LIST = false>
__device__ __forceinline__ void vote_rows(const Geom &g, uint32_t *tile, const float4 *hs, const float *beta,
                                          uint32_t nc, uint32_t r, uint32_t i, uint32_t hl, uint32_t hstride,
                                          uint32_t pitch, const FlushList &L = FlushList{})
{
    const float twoA = __fmul_rn(2.0f, a_centre(g, i));
    const uint32_t rowbase = r * pitch;
    const uint32_t sw = U16 ? (row_hash(r) & 0x1Eu) : (row_hash(r) & 0x1Cu);
    const float b_lo = beta[0], b_hi = beta[g.nb];   // the in-range test of every vote
    const uint32_t tm1 = g.threshold - 1u;
#pragma unroll 4
    for (uint32_t h = hl; h < nc; h += hstride) {
        const float4 hv = hs[h];
        const int j = vote_bin_tab(g, beta, b_lo, b_hi, twoA, hv.x, hv.y, hv.z);
        if (j >= 0) {
            if (U16) {
                const uint32_t word = rowbase + ((uint32_t(j) >> 1) ^ sw);
                const uint32_t sh = (uint32_t(j) & 1u) << 4;
                if (LIST) {
                    if (((atomicAdd(&tile[word], 1u << sh) >> sh) & 0xffffu) == tm1)
                        note_candidate(L, r, r * g.nb + uint32_t(j));
                } else {
                    atomicAdd(&tile[word], 1u << sh);
                }
            } else {
                if (LIST) {
                    if (atomicAdd(&tile[rowbase + (uint32_t(j) ^ sw)], 1u) == tm1)
                        note_candidate(L, r, r * g.nb + uint32_t(j));
                } else {
                    atomicAdd(&tile[rowbase + (uint32_t(j) ^ sw)], 1u);
                }
            }
        }
    }
}

template <bool LIST>
__device__ __forceinline__ void list_cells(const Geom &g, const FlushList &L, uint32_t r, uint32_t j0,
                                           const uint32_t *v, uint32_t n)
{
    if (!LIST)
        return;
    uint32_t mx = 0;
    for (uint32_t m = 0; m < n; ++m)
        mx = max(mx, v[m]);
    if (mx < g.threshold)
        return;
    atomicOr(&L.hot[r >> 5], 1u << (r & 31u));
    for (uint32_t m = 0; m < n; ++m)
        if (v[m] >= g.threshold) {
            const uint32_t p = atomicAdd(L.n, 1u);
            if (p < L.cap) {
                L.cand[p] = r * g.nb + j0 + m;
                L.candv[p] = v[m];
            }
        }
}

// Write tile rows r0 .. r0 + rows - 1 of one pass to dst (M_H, or with
// !GDST a shared-memory staging buffer, from its first row on) and clear
// them; with LIST, list the cells >= T (as pass rows r0 + r); with
// accumulate, add to M_H.
// The tile keeps row r's logical word w at physical word w ^ sw(r) (sw even
// in u16 mode, a multiple of 4 in u32 mode).  When n_b is a multiple of 4
// each step moves 4 cells: consecutive threads write consecutive 16-byte
// pieces of the row, so every store instruction of a warp covers 512
// contiguous bytes.
template <bool U16, bool LIST, bool ACC, class G = BlockGroup, bool GDST = true>
__device__ __forceinline__ void flush_tile(const Geom &g, uint32_t *tile, uint32_t *dst, uint32_t rows,
                                           uint32_t pitch, const FlushList &L, uint32_t r0 = 0)
{
    const uint32_t tid = G::rank(), bd = G::size(), nb = g.nb;
    // one 16-byte unit (4 cells) of row r0 + r, column group c4: read + clear
    // the tile words, write (or add to) the output at o, list the cells >= T
    auto unit = [&](uint32_t rl, uint32_t c4, uint4 *o) {
        const uint32_t r = r0 + rl;
        uint32_t v[4];
        if (U16) {
            uint2 *p = reinterpret_cast<uint2 *>(&tile[r * pitch + ((2u * c4) ^ (row_hash(r) & 0x1Eu))]);
            const uint2 pr = *p;
            *p = make_uint2(0u, 0u);
            v[0] = pr.x & 0xffffu; v[1] = pr.x >> 16; v[2] = pr.y & 0xffffu; v[3] = pr.y >> 16;
        } else {
            uint4 *p = reinterpret_cast<uint4 *>(&tile[r * pitch + ((4u * c4) ^ (row_hash(r) & 0x1Cu))]);
            const uint4 pr = *p;
            *p = make_uint4(0u, 0u, 0u, 0u);
            v[0] = pr.x; v[1] = pr.y; v[2] = pr.z; v[3] = pr.w;
        }
        if (ACC) {
            const uint4 old = *o;
            v[0] += old.x; v[1] += old.y; v[2] += old.z; v[3] += old.w;
        }
        // to M_H a streaming store (evict-first): M_H is written once per fill and
        // read back only at the candidates, so its lines should not displace
        // other data in L2; a staging buffer in shared memory takes a plain store
        if (GDST)
            __stcs(o, make_uint4(v[0], v[1], v[2], v[3]));
        else
            *o = make_uint4(v[0], v[1], v[2], v[3]);
        list_cells<LIST>(g, L, r, 4u * c4, v, 4);
    };
    if ((nb & 3u) == 0) {
        const uint32_t q = nb >> 2;  // 16-byte units per row
        if (bd % q == 0) {
            // the group covers whole rows: each thread keeps its column group
            // and steps down bd / q rows at a time
            const uint32_t rstep = bd / q, c4 = tid % q;
            uint4 *o = reinterpret_cast<uint4 *>(dst) + tid;
            for (uint32_t r = tid / q; r < rows; r += rstep, o += bd)
                unit(r, c4, o);
        } else {
            const uint32_t qs = (q & (q - 1)) ? 32u : (uint32_t)(__ffs(q) - 1);
            const uint32_t units = rows * q;
            for (uint32_t u = tid; u < units; u += bd) {
                const uint32_t r = qs < 32u ? u >> qs : u / q;
                unit(r, u - r * q, reinterpret_cast<uint4 *>(dst) + u);
            }
        }
    } else {
        const uint32_t units = rows * nb;
        for (uint32_t u = tid; u < units; u += bd) {
            const uint32_t rl = u / nb, j = u - rl * nb, r = r0 + rl;
            uint32_t v;
            if (U16) {
                const uint32_t word = r * pitch + ((j >> 1) ^ (row_hash(r) & 0x1Eu));
                v = (tile[word] >> ((j & 1u) << 4)) & 0xffffu;
            } else {
                const uint32_t word = r * pitch + (j ^ (row_hash(r) & 0x1Cu));
                v = tile[word];
            }
            v = ACC ? dst[u] + v : v;
            dst[u] = v;
            list_cells<LIST>(g, L, r, j, &v, 1);
        }
        G::sync();
        // clear the rows after every thread has read its cells
        for (uint32_t k = tid; k < rows * pitch; k += bd)
            tile[r0 * pitch + k] = 0u;
    }
}

// Copy up to cap hit records of a unit's list, from list index pos on (pos
// < end), into hs; advances pos.  All threads of the group call it.
template <class G = BlockGroup>
__device__ __forceinline__ uint32_t stage_hits(const Work &w, float4 *hs, uint32_t cap, uint32_t &pos, uint32_t end)
{
    G::sync();   // the previous readers of hs are done
    const uint32_t n = min(cap, end - pos);
    constexpr uint32_t U = 4;
    for (uint32_t k0 = 0; k0 < n; k0 += U * G::size()) {
        float4 v[U];
#pragma unroll
        for (uint32_t q = 0; q < U; ++q) {
            const uint32_t k = k0 + q * G::size() + G::rank();
            if (k < n)
                v[q] = __ldg(&w.list[pos + k]);
        }
#pragma unroll
        for (uint32_t q = 0; q < U; ++q) {
            const uint32_t k = k0 + q * G::size() + G::rank();
            if (k < n)
                hs[k] = v[q];
        }
    }
    pos += n;
    G::sync();
    return n;
}

// The votes of one strip pass: tile rows 0 .. pr - 1 are A bins i - r ..,
// from the hits of list entries l0 .. l1 of unit es.  Hits are staged HC at
// a time; when a unit's hits fit they stay staged for its later passes
// (cached_es / cached_n).  SYNC: a cached pass starts with a group barrier
// (the previous pass's readers of the tile are done); without it the caller
// orders the tile by other means.  All threads of the group call it.
template <class G, bool SYNC, bool LIST>
__device__ __forceinline__ void vote_pass(const Geom &g, const Work &w, uint32_t *tile, float4 *hs, const float *beta,
                                          uint32_t HC, uint64_t es, uint32_t l0, uint32_t l1, uint64_t &cached_es,
                                          uint32_t &cached_n, bool u16, uint32_t r, uint32_t pr, uint32_t i,
                                          uint32_t hl, uint32_t hstride, uint32_t pitch, const FlushList &L)
{
    if (cached_es == es) {
        if (SYNC)
            G::sync();
        if (r < pr) {
            if (u16)
                vote_rows<true, LIST>(g, tile, hs, beta, cached_n, r, i, hl, hstride, pitch, L);
            else
                vote_rows<false, LIST>(g, tile, hs, beta, cached_n, r, i, hl, hstride, pitch, L);
        }
        return;
    }
    cached_es = ~0ull;   // hs is about to be overwritten
    uint32_t pos = l0;
    bool first = true;
    while (first || pos < l1) {
        const uint32_t nsel = stage_hits<G>(w, hs, HC, pos, l1);
        if (first && pos >= l1) {
            cached_es = es;   // the whole list fits: keep it
            cached_n = nsel;
        }
        first = false;
        if (r < pr) {
            if (u16)
                vote_rows<true, LIST>(g, tile, hs, beta, nsel, r, i, hl, hstride, pitch, L);
            else
                vote_rows<false, LIST>(g, tile, hs, beta, nsel, r, i, hl, hstride, pitch, L);
        }
    }
}

// The work items [it0, it1) of CTA `cta` of `grid`: the (event, slice,
// strip) items in order, cut where the estimated cost -- v = c.vote_weight
// per (hit, row) vote plus one per cell written -- reaches cta / grid of the
// total.  A unit u = (event, slice) costs n_a (n_b + v hits(u)), so the cost
// before unit u is n_a (n_b u + v slice_off[u]); a cut inside a unit falls
// on a strip boundary.  Every thread of the group calls
// it and gets the same result; s_res: 2 shared words.
template <class G = BlockGroup>
__device__ __forceinline__ void cta_items(const Geom &g, const Work &w, const FillCfg &c, uint32_t cta,
                                          uint32_t grid, uint64_t n_static, uint64_t &it0, uint64_t &it1,
                                          unsigned long long *s_res)
{
    const uint32_t U = w.n_events * g.n_slices;
    auto cost = [&](uint32_t u) {
        return (uint64_t)g.na * ((uint64_t)g.nb * u + (uint64_t)c.vote_weight * __ldcg(&w.slice_off[u]));
    };
    // the cost of the first n_static items
    const uint32_t us = (uint32_t)(n_static / c.strips), ks = (uint32_t)(n_static % c.strips);
    uint64_t total = cost(us);
    if (ks)
        total += ks * ((cost(us + 1) - total + c.strips - 1) / c.strips);
    const uint64_t items = n_static;
    const uint64_t T0 = (total / grid) * cta + ((total % grid) * cta) / grid;
    const uint64_t T1 = (total / grid) * (cta + 1) + ((total % grid) * (cta + 1)) / grid;
    if (G::rank() == 0)
        s_res[0] = s_res[1] = items;
    G::sync();
    for (uint32_t u = G::rank(); u < U; u += G::size()) {
        const uint64_t a = cost(u), b = cost(u + 1);
        const uint64_t per = (b - a + c.strips - 1) / c.strips;   // one strip, rounded up
        const uint64_t last = c.strips - 1;
        if (a <= T0 && T0 < b) {
            const uint64_t k = (T0 - a) / per;
            s_res[0] = (uint64_t)u * c.strips + (k < last ? k : last);
        }
        if (a <= T1 && T1 < b) {
            const uint64_t k = (T1 - a) / per;
            s_res[1] = (uint64_t)u * c.strips + (k < last ? k : last);
        }
    }
    G::sync();
    it0 = min((uint64_t)s_res[0], items);
    it1 = cta + 1 == grid ? items : min((uint64_t)s_res[1], items);
    G::sync();   // s_res may be reused
}

// Hand out the next run-time item (see dyn_items): returns its rank, or
// n_dyn once none is left -- after which the last CTA to find none resets
// both counters for the next fill.  All threads of the block call it.
__device__ __forceinline__ uint32_t next_dyn_item(const Work &w, uint32_t n_dyn, uint32_t *s_word)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t d = n_dyn;
        if (n_dyn)
            d = atomicAdd(&w.ctr[CTR_DYN], 1u);
        if (d >= n_dyn) {
            d = n_dyn;
            __threadfence();
            if (atomicAdd(&w.ctr[CTR_DYN_DONE], 1u) == gridDim.x - 1) {
                w.ctr[CTR_DYN] = 0u;
                w.ctr[CTR_DYN_DONE] = 0u;
            }
        }
        *s_word = d;
    }
    __syncthreads();
    return *s_word;
}

// The run-time items with the claim of the next one in flight: thread 0
// claims an item (dyn_claim) while the block still works on the one before,
// and dyn_take publishes the claim to the block, ending the hand-out as
// next_dyn_item does (rank n_dyn: none left).  Each CTA claims until it
// gets none, once per rank, so the counters reset as with next_dyn_item.
__device__ __forceinline__ uint32_t dyn_claim(const Work &w, uint32_t n_dyn)
{
    return atomicAdd(&w.ctr[CTR_DYN], 1u);   // thread 0 only; n_dyn > 0
}

__device__ __forceinline__ uint32_t dyn_take(const Work &w, uint32_t n_dyn, uint32_t claim, uint32_t *s_word)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t d = claim;
        if (d >= n_dyn) {
            d = n_dyn;
            __threadfence();
            if (atomicAdd(&w.ctr[CTR_DYN_DONE], 1u) == gridDim.x - 1) {
                w.ctr[CTR_DYN] = 0u;
                w.ctr[CTR_DYN_DONE] = 0u;
            }
        }
        *s_word = d;
    }
    __syncthreads();
    return *s_word;
}

// Walks the (event, slice, strip) work items it0, it0 + 1, ... of a CTA with
// one 64-bit decomposition at the start and carries afterwards (a 64-bit
// division per item and thread costs more than a strip's flush setup).
struct ItemCursor {
    uint32_t k, s, e;   // strip, slice, event
    uint64_t es;        // e * n_slices + s
    __device__ __forceinline__ ItemCursor(const Geom &g, const FillCfg &c, uint64_t item)
    {
        k = (uint32_t)(item % c.strips);
        es = item / c.strips;
        s = (uint32_t)(es % g.n_slices);
        e = (uint32_t)(es / g.n_slices);
    }
    __device__ __forceinline__ void next(const Geom &g, const FillCfg &c)
    {
        if (++k == c.strips) {
            k = 0;
            ++es;
            if (++s == g.n_slices) {
                s = 0;
                ++e;
            }
        }
    }
};

__global__ void __launch_bounds__(1024) k_fill_priv(Geom g, Work w, FillCfg c)
{
    extern __shared__ uint4 sm4[];
    uint32_t *tile = reinterpret_cast<uint32_t *>(sm4);
    float4 *hs = reinterpret_cast<float4 *>(tile + c.tile_words);
    float *beta = reinterpret_cast<float *>(hs + c.HC);

    const uint32_t tid = threadIdx.x, bd = blockDim.x;
    for (uint32_t k = tid; k < c.tile_words / 4; k += bd)
        sm4[k] = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t k = tid; k <= g.nb; k += bd)
        beta[k] = g.bth[k];
    grid_dep_wait();   // the unit lists of k_scatter

    __shared__ unsigned long long s_rng[2];
    __shared__ uint32_t s_dyn;
    const uint64_t items = (uint64_t)w.n_events * g.n_slices * c.strips;
    const uint64_t n_dyn = c.dyn ? dyn_items(items, gridDim.x) : 0, n_static = items - n_dyn;
    uint64_t it0, it1;
    cta_items(g, w, c, blockIdx.x, gridDim.x, n_static, it0, it1, s_rng);
    uint64_t cached_es = ~0ull;   // (event, slice) whose whole hit list is in hs
    uint32_t cached_n = 0;

    auto do_item = [&](const ItemCursor &cur) {
        const uint32_t k = cur.k;
        const uint64_t es = cur.es;
        const uint32_t s = cur.s;
        const uint32_t e = cur.e;
        const uint32_t l0 = __ldg(&w.slice_off[es]), l1 = __ldg(&w.slice_off[es + 1]);   // the unit's hits
        const uint32_t i0 = k * c.W;
        const uint32_t rows = min(c.W, g.na - i0);
        // u16 counters are exact while the slice holds < 65536 hits
        const bool u16 = (l1 - l0) < 65536u;
        const uint32_t rpass = u16 ? c.W : c.W / 2;
        const uint32_t pitch = u16 ? c.pitch16 : c.pitch32;
        uint32_t *Mrow = w.M + (size_t)e * w.n_cells + ((size_t)s * g.na + i0) * g.nb;
        const uint32_t r = tid % rpass, hl = tid / rpass, hstride = bd / rpass;

        for (uint32_t p0 = 0; p0 < rows; p0 += rpass) {
            const uint32_t pr = min(rpass, rows - p0);
            const uint32_t i = i0 + p0 + r;
            vote_pass<BlockGroup, true, false>(g, w, tile, hs, beta, c.HC, es, l0, l1, cached_es, cached_n, u16, r, pr,
                                               i, hl, hstride, pitch, FlushList{});
            __syncthreads();
            uint32_t *dst = Mrow + (size_t)p0 * g.nb;
            if (c.accumulate) {
                if (u16)
                    flush_tile<true, false, true>(g, tile, dst, pr, pitch, FlushList{});
                else
                    flush_tile<false, false, true>(g, tile, dst, pr, pitch, FlushList{});
            } else {
                if (u16)
                    flush_tile<true, false, false>(g, tile, dst, pr, pitch, FlushList{});
                else
                    flush_tile<false, false, false>(g, tile, dst, pr, pitch, FlushList{});
            }
        }
    };
    ItemCursor cur(g, c, it0);
    for (uint64_t item = it0; item < it1; ++item, cur.next(g, c))
        do_item(cur);
    if (c.dyn)
        for (uint32_t d; (d = next_dyn_item(w, (uint32_t)n_dyn, &s_dyn)) < n_dyn;)
            do_item(ItemCursor(g, c, n_static + d));
}

// ---------------------------------------------------------------------------
// Naive path (the paper's CUDA fill): clear + global atomics.
// ---------------------------------------------------------------------------
__global__ void k_clear(uint32_t *M, uint64_t words)
{
    grid_dep_wait();
    const uint64_t n4 = words >> 2;
    uint4 *M4 = reinterpret_cast<uint4 *>(M);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += stride)
        M4[k] = make_uint4(0u, 0u, 0u, 0u);
    for (uint64_t k = (n4 << 2) + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < words; k += stride)
        M[k] = 0u;
}

// The unit (event, slice) of hit record rec of the (event, slice) lists: the
// largest u' <= u with slice_off[u'] <= rec (slice_off[0] = 0), found by the
// warp 32 units at a time.  Every lane returns it; the whole warp calls it.
__device__ __forceinline__ uint32_t unit_below(const uint32_t *slice_off, uint32_t u, uint32_t rec)
{
    const uint32_t lane = threadIdx.x & 31u;
    for (;;) {
        const bool ok = lane <= u && __ldg(&slice_off[u - lane]) <= rec;
        const uint32_t m = __ballot_sync(0xffffffffu, ok);
        if (m)
            return u - (uint32_t)(__ffs(m) - 1);
        if (u < 32u)
            return 0u;
        u -= 32u;
    }
}

// The paper's fill (Sec. 3): a 1-D grid over hits, a thread block over A,
// one global atomicAdd per vote.  The hits come from k_scatter's (event,
// slice) lists, one (hit, slice) record per block at a time, and the grid
// (what the GPU holds at once) strides over the records from the last to
// the first: the blocks in flight work on neighbouring records, so their
// votes land in a few slices of M_H that stay in L2, and the first slices
// voted are the last ones the clear wrote.  The B bin comes from the
// threshold table in shared memory when it fits (48 KB), else from the
// division rule; both give the same bin for every B.
__global__ void __launch_bounds__(1024, 2) k_fill_naive(Geom g, Work w)
{
    extern __shared__ float s_beta[];   // n_b + 1 B-bin thresholds, or none
    const uint32_t tid = threadIdx.x, bd = blockDim.x;
    const bool tab = ((size_t)g.nb + 1) * 4 <= 48u * 1024u;
    if (tab)
        for (uint32_t k = tid; k <= g.nb; k += bd)
            s_beta[k] = g.bth[k];
    __syncthreads();
    grid_dep_wait();
    const float b_lo = tab ? s_beta[0] : 0.0f, b_hi = tab ? s_beta[g.nb] : 0.0f;
    const uint32_t U = w.n_events * g.n_slices;
    if (U == 0)
        return;
    const uint32_t n_rec = min(__ldg(&w.slice_off[U]), w.list_cap);
    const uint64_t slice_cells = (uint64_t)g.na * g.nb;
    uint32_t u = U - 1u;
    for (uint32_t k = blockIdx.x; k < n_rec; k += gridDim.x) {
        const uint32_t rec = n_rec - 1u - k;
        u = unit_below(w.slice_off, u, rec);
        const float4 hv = w.list[rec];
        const uint32_t e = u / g.n_slices, s = u - e * g.n_slices;
        uint32_t *Ms = w.M + (size_t)e * w.n_cells + (size_t)s * slice_cells;
        for (uint32_t i = tid; i < g.na; i += bd) {
            const float twoA = __fmul_rn(2.0f, a_centre(g, i));
            const int j = tab ? vote_bin_tab(g, s_beta, b_lo, b_hi, twoA, hv.x, hv.y, hv.z)
                              : vote_bin(g, twoA, hv.x, hv.y, hv.z);
            if (j >= 0)
                atomicAdd(&Ms[(size_t)i * g.nb + (uint32_t)j], 1u);
        }
    }
}

// ---------------------------------------------------------------------------
// Scan
// ---------------------------------------------------------------------------
// Peak test of the cell at column j of `row` (value v >= threshold).
// up / dn are the neighbouring rows of the same slice or nullptr.
__device__ __forceinline__ bool is_peak(const uint32_t *row, const uint32_t *up, const uint32_t *dn,
                                        uint32_t j, uint32_t nb, uint32_t v)
{
    const bool hl = j > 0, hr = j + 1 < nb;
    if (up) {
        if (hl && !(v > up[j - 1])) return false;
        if (!(v > up[j])) return false;
        if (hr && !(v > up[j + 1])) return false;
    }
    if (hl && !(v > row[j - 1])) return false;
    if (hr && !(v >= row[j + 1])) return false;
    if (dn) {
        if (hl && !(v >= dn[j - 1])) return false;
        if (!(v >= dn[j])) return false;
        if (hr && !(v >= dn[j + 1])) return false;
    }
    return true;
}

struct ScanSmem {
    uint32_t wsum[40];
    uint32_t round_total;
    uint32_t chunk_base;
    uint32_t abort;
    uint32_t pad;
};

// Where a CTA (or a handed-out fill item) registers its chunks: its row of
// a.desc, seq_max entries.
struct ChunkList {
    uint2 *desc;
    uint32_t cap;
};

__device__ __forceinline__ ChunkList interior_list(const ScanArgs &a, uint32_t cta)
{
    return ChunkList{a.desc + (size_t)cta * a.seq_max, a.seq_max};
}

// Flush the CTA's buffered peaks as one chunk of list L.
template <class G = BlockGroup>
__device__ __forceinline__ void flush_chunk(const ScanArgs &a, ScanSmem &ss, const uint4 *pbuf,
                                            uint32_t &buf_n, uint32_t &nseq, const ChunkList &L,
                                            uint32_t *status)
{
    if (buf_n == 0)
        return;
    if (G::rank() == 0) {
        ss.chunk_base = atomicAdd(a.g_count, buf_n);
        if (nseq < L.cap)
            L.desc[nseq] = make_uint2(ss.chunk_base, buf_n);
        if (nseq >= L.cap || ss.chunk_base + buf_n > a.entries_cap)
            atomicOr(status, (uint32_t)ST_SCRATCH_OVERFLOW);
    }
    G::sync();
    const uint32_t base = ss.chunk_base;
    for (uint32_t k = G::rank(); k < buf_n; k += G::size())
        if (base + k < a.entries_cap)
            a.entries[base + k] = pbuf[k];
    nseq += 1;
    buf_n = 0;
    G::sync();
}

// Ordered compaction of one round: each thread holds cnt peaks in pj/pv
// (columns of the row starting at row_lin0); appends them to pbuf in
// thread order and counts them for their event.
template <class G = BlockGroup, bool COUNT = true>
__device__ __forceinline__ void compact_round(ScanSmem &ss, uint4 *pbuf, uint32_t &buf_n, uint32_t cnt,
                                              const uint32_t *pj, const uint32_t *pv, uint32_t row_lin0,
                                              uint32_t event, uint32_t *ev_count)
{
    const uint32_t tid = G::rank(), warp = tid >> 5, lane = tid & 31u;
    const uint32_t nw = (G::size() + 31) >> 5;
    const uint32_t incl = warp_incl_scan(cnt);
    if (lane == 31u)
        ss.wsum[warp] = incl;
    G::sync();
    if (warp == 0) {
        const uint32_t v = lane < nw ? ss.wsum[lane] : 0u;
        const uint32_t vi = warp_incl_scan(v);
        ss.wsum[lane] = vi - v;
        if (lane == 31u) {
            ss.round_total = vi;
            if (COUNT)
                atomicAdd(&ev_count[event], vi);
        }
    }
    G::sync();
    const uint32_t pos = buf_n + ss.wsum[warp] + incl - cnt;
    for (uint32_t k = 0; k < cnt; ++k)
        pbuf[pos + k] = make_uint4(row_lin0 + pj[k], event, pv[k], 0u);
    buf_n += ss.round_total;
    G::sync();
}

// Ordered compaction of one entry per thread (has = 0 or 1): appends the
// entries to pbuf in thread order and counts them for their events.
template <class G = BlockGroup, bool COUNT = true>
__device__ __forceinline__ void compact_entry(ScanSmem &ss, uint4 *pbuf, uint32_t &buf_n, uint32_t has,
                                              const uint4 &ent, uint32_t *ev_count)
{
    const uint32_t tid = G::rank(), warp = tid >> 5, lane = tid & 31u;
    const uint32_t nw = (G::size() + 31) >> 5;
    const uint32_t incl = warp_incl_scan(has);
    if (lane == 31u)
        ss.wsum[warp] = incl;
    G::sync();
    if (warp == 0) {
        const uint32_t v = lane < nw ? ss.wsum[lane] : 0u;
        const uint32_t vi = warp_incl_scan(v);
        ss.wsum[lane] = vi - v;
        if (lane == 31u)
            ss.round_total = vi;
    }
    G::sync();
    if (has) {
        pbuf[buf_n + ss.wsum[warp] + incl - 1] = ent;
        if (COUNT)
            atomicAdd(&ev_count[ent.y], 1u);
    }
    buf_n += ss.round_total;
    G::sync();
}

// Detailed pass over global rows [ra, rb): candidates, neighbour tests and
// ordered compaction.  Rows [ra - 1, rb + 1) (clipped) are readable at
// base + (gr - b_first) * nb.  Each thread takes VEC consecutive cells.
template <int VEC>
__device__ void scan_rows_slow(const Geom &g, const Work &w, const ScanArgs &a, ScanSmem &ss, uint4 *pbuf,
                               uint32_t &buf_n, uint32_t &nseq, uint32_t &total, uint64_t ra, uint64_t rb,
                               const uint32_t *base, uint64_t b_first)
{
    const uint32_t tid = threadIdx.x, bd = blockDim.x, nb = g.nb, T = g.threshold;
    const uint64_t rows_ev = (uint64_t)g.n_slices * g.na;
    const uint32_t units = nb / VEC;
    const uint32_t rounds = (units + bd - 1) / bd;
    for (uint64_t gr = ra; gr < rb; ++gr) {
        const uint32_t i = (uint32_t)(gr % g.na);
        const uint32_t ev = (uint32_t)(gr / rows_ev);
        const uint32_t row_lin0 = (uint32_t)((gr - (uint64_t)ev * rows_ev) * nb);
        const uint32_t *row = base + (gr - b_first) * nb;
        const uint32_t *up = i > 0 ? row - nb : nullptr;
        const uint32_t *dn = i + 1 < g.na ? row + nb : nullptr;
        for (uint32_t rd = 0; rd < rounds; ++rd) {
            const uint32_t u = rd * bd + tid;
            uint32_t cnt = 0, pj[VEC], pv[VEC];
            if (u < units) {
#pragma unroll
                for (uint32_t c = 0; c < (uint32_t)VEC; ++c) {
                    const uint32_t j = VEC * u + c;
                    const uint32_t v = row[j];
                    if (v >= T && is_peak(row, up, dn, j, nb, v)) {
                        pj[cnt] = j;
                        pv[cnt] = v;
                        ++cnt;
                    }
                }
            }
            if (__syncthreads_or(cnt)) {
                // at most 2 peaks among 4 consecutive cells (no two peaks are neighbours)
                if (buf_n + (VEC > 1 ? 2u : 1u) * bd > a.K)
                    flush_chunk(a, ss, pbuf, buf_n, nseq, interior_list(a, blockIdx.x), w.status);
                compact_round(ss, pbuf, buf_n, cnt, pj, pv, row_lin0, ev, a.ev_count);
                total += ss.round_total;
            }
        }
    }
}

// TMA-staged scan (n_b % 4 == 0).
__global__ void __launch_bounds__(256) k_scan_tma(Geom g, Work w, ScanArgs a)
{
    grid_dep_wait();
    extern __shared__ uint4 sm4[];
    // layout: [0, 192) ScanSmem | [192, 256) 8 mbarriers | K peak entries | S stage slots
    ScanSmem &ss = *reinterpret_cast<ScanSmem *>(sm4);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm4 + 12);
    uint4 *pbuf = sm4 + 16;
    uint32_t *slots = reinterpret_cast<uint32_t *>(pbuf + a.K);

    const uint32_t tid = threadIdx.x, bd = blockDim.x;
    const uint32_t nb = g.nb, T = g.threshold;
    const uint64_t G = (uint64_t)g.n_slices * g.na * w.n_events;
    const uint64_t g0 = G * blockIdx.x / gridDim.x, g1 = G * (blockIdx.x + 1) / gridDim.x;
    const uint32_t R = a.R, S = a.S;
    const uint64_t n_stages = (g1 - g0 + R - 1) / R;
    uint32_t buf_n = 0, nseq = 0, total = 0;

    if (tid == 0) {
        ss.abort = 0;
        for (uint32_t q = 0; q < S; ++q)
            mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // stage k: own rows [g0 + kR, min(g0 + (k+1)R, g1)), loaded with one
    // halo row on each side (clipped to the matrix).
    auto issue = [&](uint64_t k) {
        const uint64_t ra = g0 + k * R, rb = min(ra + R, g1);
        const uint64_t ba = ra > 0 ? ra - 1 : 0, bb = min(rb + 1, G);
        const uint32_t q = (uint32_t)(k % S);
        const uint32_t bytes = (uint32_t)((bb - ba) * nb * 4u);
        mbar_arrive_expect_tx(&bars[q], bytes);
        bulk_load(slots + (size_t)q * a.slot_words, w.M + ba * nb, bytes, &bars[q]);
    };
    if (tid == 0)
        for (uint64_t k = 0; k < n_stages && k < S; ++k)
            issue(k);

    uint64_t k_abort = 0;
    for (uint64_t k = 0; k < n_stages; ++k) {
        const uint64_t ra = g0 + k * R, rb = min(ra + R, g1);
        const uint64_t ba = ra > 0 ? ra - 1 : 0;
        const uint32_t q = (uint32_t)(k % S);
        const uint32_t *slot = slots + (size_t)q * a.slot_words;
        if (!mbar_wait_bounded(&bars[q], (uint32_t)((k / S) & 1u)))
            atomicOr(&ss.abort, 1u);
        __syncthreads();
        if (ss.abort) {
            k_abort = k;
            break;
        }
        // fast path: any cell >= T among the stage's own rows?
        const uint4 *own = reinterpret_cast<const uint4 *>(slot + (ra - ba) * nb);
        const uint32_t n4 = (uint32_t)(rb - ra) * (nb >> 2);
        uint32_t hot = 0;
        for (uint32_t u = tid; u < n4; u += bd) {
            const uint4 v = own[u];
            hot |= (max(max(v.x, v.y), max(v.z, v.w)) >= T);
        }
        if (__syncthreads_or(hot))
            scan_rows_slow<4>(g, w, a, ss, pbuf, buf_n, nseq, total, ra, rb, slot, ba);
        __syncthreads();  // every thread is done with slot q
        if (tid == 0 && k + S < n_stages) {
            fence_proxy_async_smem();
            issue(k + S);
        }
    }
    if (ss.abort) {
        // let the copies still in flight (bounded wait) land before the CTA exits
        if (tid == 0) {
            atomicOr(w.status, (uint32_t)ST_WAIT_TIMEOUT);
            const uint64_t k_end = min(n_stages, k_abort + S);
            for (uint64_t kk = k_abort; kk < k_end; ++kk)
                (void)mbar_wait_bounded(&bars[kk % S], (uint32_t)((kk / S) & 1u));
        }
        __syncthreads();
    }
    flush_chunk(a, ss, pbuf, buf_n, nseq, interior_list(a, blockIdx.x), w.status);
    if (tid == 0) {
        a.cta_nseq[blockIdx.x] = min(nseq, a.seq_max);
        a.cta_total[blockIdx.x] = total;
    }
}

// Direct-load scan for any n_b (no staging).
__global__ void __launch_bounds__(256) k_scan_direct(Geom g, Work w, ScanArgs a)
{
    grid_dep_wait();
    extern __shared__ uint4 sm4[];
    ScanSmem &ss = *reinterpret_cast<ScanSmem *>(sm4);
    uint4 *pbuf = sm4 + 16;
    const uint32_t tid = threadIdx.x, bd = blockDim.x;
    const uint32_t nb = g.nb, T = g.threshold;
    const uint64_t G = (uint64_t)g.n_slices * g.na * w.n_events;
    const uint64_t g0 = G * blockIdx.x / gridDim.x, g1 = G * (blockIdx.x + 1) / gridDim.x;
    const uint32_t R = a.R;
    uint32_t buf_n = 0, nseq = 0, total = 0;
    for (uint64_t ra = g0; ra < g1; ra += R) {
        const uint64_t rb = min(ra + R, g1);
        const uint32_t *own = w.M + ra * nb;
        const uint64_t n = (rb - ra) * nb;
        uint32_t hot = 0;
        for (uint64_t u = tid; u < n; u += bd)
            hot |= own[u] >= T;
        if (__syncthreads_or(hot))
            scan_rows_slow<1>(g, w, a, ss, pbuf, buf_n, nseq, total, ra, rb, w.M, 0);
    }
    flush_chunk(a, ss, pbuf, buf_n, nseq, interior_list(a, blockIdx.x), w.status);
    if (tid == 0) {
        a.cta_nseq[blockIdx.x] = min(nseq, a.seq_max);
        a.cta_total[blockIdx.x] = total;
    }
}

// ---------------------------------------------------------------------------
// The fused fill: Step 1 plus the first half of Step 2.
//
// Like k_fill_priv, a CTA owns a contiguous range of (event, slice, strip)
// items, votes each strip pass into a shared-memory tile and writes it to
// M_H, clearing the tile as it goes.  While writing, it lists the cells of
// the pass that hold >= T votes and appends them, in linear order, to its
// chunks of candidate entries -- the cells a full scan would have to look
// at.  k_peaks then tests only those candidates against their neighbours,
// once the whole of M_H is written (no row waits for another CTA), and
// compacts each chunk in place to the peaks; k_order places the chunks.
// A pass listing more than kFusedCand cells emits its rows' cells >= T from
// M_H instead (read back through L2).
// ---------------------------------------------------------------------------

// Peak test with the neighbours read through L2; up / dn are null outside
// the slice.  All eight loads are issued before any comparison, so a test
// costs one memory latency.
__device__ __forceinline__ bool is_peak_l2(const uint32_t *row, const uint32_t *up, const uint32_t *dn, uint32_t j,
                                           uint32_t nb, uint32_t v)
{
    const bool hl = j > 0, hr = j + 1 < nb;
    const uint32_t ul = up && hl ? __ldcg(up + j - 1) : 0u, uc = up ? __ldcg(up + j) : 0u,
                   ur = up && hr ? __ldcg(up + j + 1) : 0u;
    const uint32_t rl = hl ? __ldcg(row + j - 1) : 0u, rr = hr ? __ldcg(row + j + 1) : 0u;
    const uint32_t dl = dn && hl ? __ldcg(dn + j - 1) : 0u, dc = dn ? __ldcg(dn + j) : 0u,
                   dr = dn && hr ? __ldcg(dn + j + 1) : 0u;
    // absent neighbours read as 0: v > 0 and v >= 0 hold for every v >= 1
    return v > ul && v > uc && v > ur && v > rl && v >= rr && v >= dl && v >= dc && v >= dr;
}

// Append the candidate cells of one pass (rows iA .. iA + pr - 1 of slice
// unit `slice_lin0`) to the CTA's candidate chunks, in linear order.  n_c
// cells were listed as r * n_b + j in cand / candv (up to kFusedCand); with
// more, the rows marked in hotm are read back: pass row r from rowsA + r rs
// when r < split, else from rowsB + (r - split) rs (rs = row_stride, or n_b
// when it is 0) -- M_H in global memory,
// or (SMEM) the shared staging buffers.  Entries are {lin within event,
// event, votes, 0}.  TV (the tile-store fill): the votes of a listed key are
// read from rowsA[key] (the pass's u32 tile, rows n_b apart) instead of
// candv.  All threads of the group call it.
template <class G, bool SMEM = false, bool TV = false>
__device__ __forceinline__ void emit_pass(const Geom &g, const Work &w, const ScanArgs &a, ScanSmem &ss, uint4 *pbuf,
                                          uint32_t &buf_n, uint32_t &nseq, uint32_t &total, const ChunkList &inner,
                                          const uint32_t *cand, const uint32_t *candv, uint32_t *srt, uint32_t *srtv,
                                          uint32_t n_c, uint64_t hotm, uint32_t pr, uint32_t iA, uint32_t slice_lin0,
                                          uint32_t e, const uint32_t *rowsA, const uint32_t *rowsB, uint32_t split,
                                          uint32_t row_stride = 0)
{
    const uint32_t tid = G::rank(), bd = G::size(), nb = g.nb;
    const size_t rs = row_stride ? row_stride : nb;   // words between consecutive rows of rowsA / rowsB
    const uint32_t lin0 = slice_lin0 + iA * nb;
    if (n_c <= 32u) {
        // few candidates: the first warp ranks them and writes them in order
        if (buf_n + n_c > a.K)
            flush_chunk<G>(a, ss, pbuf, buf_n, nseq, inner, w.status);
        if (tid < n_c) {
            const uint32_t key = cand[tid];
            uint32_t rank = 0;
            for (uint32_t m = 0; m < n_c; ++m)
                rank += cand[m] < key;
            pbuf[buf_n + rank] = make_uint4(lin0 + key, e, TV ? rowsA[key] : candv[tid], 0u);
        }
        buf_n += n_c;
        total += n_c;
        return;   // the caller's barrier follows before pbuf or the lists are used again
    }
    if (n_c <= kFusedCand) {
        // distinct keys: the rank of a key is the number of smaller ones
        for (uint32_t k = tid; k < n_c; k += bd) {
            const uint32_t key = cand[k];
            uint32_t rank = 0;
            for (uint32_t m = 0; m < n_c; ++m)
                rank += cand[m] < key;
            srt[rank] = key;
            srtv[rank] = TV ? rowsA[key] : candv[k];
        }
        // the sorted list is dense: append it to the chunk buffer as it is
        // (n_c <= kFusedCand <= K; a chunk is flushed with more than
        // K - kFusedCand entries, so the chunk bound of the rounds below holds)
        if (buf_n + n_c > a.K)
            flush_chunk<G>(a, ss, pbuf, buf_n, nseq, inner, w.status);   // its barriers order srt / srtv too
        else
            G::sync();
        for (uint32_t k = tid; k < n_c; k += bd)
            pbuf[buf_n + k] = make_uint4(lin0 + srt[k], e, srtv[k], 0u);
        buf_n += n_c;
        total += n_c;
        return;   // the caller's barrier follows before pbuf or the lists are used again
    }
    // rounds of rc threads, like the candidate rounds: a chunk is flushed
    // only when fewer than rc entries are free
    const uint32_t T = g.threshold, per_round = fused_round(bd, a.K);
    for (uint32_t r = 0; r < pr; ++r) {
        if (!((hotm >> r) & 1ull))
            continue;
        const uint32_t *row = r < split ? rowsA + (size_t)r * rs : rowsB + (size_t)(r - split) * rs;
        for (uint32_t j0 = 0; j0 < nb; j0 += per_round) {
            const uint32_t j = j0 + tid;
            uint32_t cnt = 0, pj[1], pv[1];
            if (tid < per_round && j < nb) {
                const uint32_t v = SMEM ? row[j] : __ldcg(row + j);
                if (v >= T) {
                    pj[0] = j;
                    pv[0] = v;
                    cnt = 1;
                }
            }
            if (G::sync_or(cnt)) {
                if (buf_n + per_round > a.K)
                    flush_chunk<G>(a, ss, pbuf, buf_n, nseq, inner, w.status);
                compact_round<G, false>(ss, pbuf, buf_n, cnt, pj, pv, lin0 + r * nb, e, nullptr);
                total += ss.round_total;
            }
        }
    }
}

// Rank-sort the n_c (<= kFusedCand) distinct keys r * n_b + j of cand into
// srt, with their votes read from the tile into srtv.  All threads of the
// group call it; the caller synchronises before srt / srtv are read.
template <class G, bool U16>
__device__ __forceinline__ void sort_tile_candidates(const Geom &g, const uint32_t *tile, uint32_t pitch,
                                                     const uint32_t *cand, uint32_t n_c, uint32_t *srt, uint32_t *srtv)
{
    for (uint32_t k = G::rank(); k < n_c; k += G::size()) {
        const uint32_t key = cand[k];
        uint32_t rank = 0;
        for (uint32_t m = 0; m < n_c; ++m)
            rank += cand[m] < key;
        const uint32_t rr = key / g.nb;
        srt[rank] = key;
        srtv[rank] = tile_cell(tile, pitch, U16, rr, key - rr * g.nb);
    }
}

// Write one pass from the tile to M_H, clear the tile, and emit its
// candidates (emit_pass).  empty_bar: arrived on once the tile is clear
// (the warp-specialised fill), or null.  All threads of the group call it.
template <class G, bool U16>
__device__ __forceinline__ void flush_emit_pass(const Geom &g, const Work &w, const ScanArgs &a, ScanSmem &ss,
                                                uint4 *pbuf, uint32_t &buf_n, uint32_t &nseq, uint32_t &total,
                                                const ChunkList &inner, uint32_t *tile, uint32_t pitch, uint32_t *dst,
                                                uint32_t pr, uint32_t iA, uint32_t slice_lin0, uint32_t e,
                                                const uint32_t *Ms, uint32_t *lists, uint32_t *s_hot, uint32_t *s_nc,
                                                uint64_t *empty_bar)
{
    uint32_t *cand = lists, *candv = lists + kFusedCand, *srt = lists + 2 * kFusedCand, *srtv = lists + 3 * kFusedCand;
    if (G::rank() == 0)
        s_hot[0] = s_hot[1] = *s_nc = 0u;
    G::sync();   // the pass's votes are complete (and the counters zero)
    flush_tile<U16, true, false, G>(g, tile, dst, pr, pitch, FlushList{s_hot, cand, candv, s_nc, kFusedCand});
    if (empty_bar)
        mbar_arrive(empty_bar);   // the tile is clear
    G::sync();                    // M_H rows of the pass and the lists visible to the group
    const uint64_t hotm = (uint64_t)s_hot[0] | ((uint64_t)s_hot[1] << 32);
    const uint32_t n_c = *s_nc;
    if (n_c)
        emit_pass<G>(g, w, a, ss, pbuf, buf_n, nseq, total, inner, cand, candv, srt, srtv, n_c, hotm, pr, iA,
                     slice_lin0, e, Ms + (size_t)iA * g.nb, nullptr, pr);
    G::sync();                    // lists and counters free for the next pass
}

// The same through the u32 staging buffers stg[0], stg[1] (hrows rows of
// n_b cells each; k_fill_bulk): the pass leaves in halves of hrows rows.
// Each half waits until the bulk copy that last read its buffer is done
// (thread 0's async-groups, all but the newest), is converted into the
// buffer while the candidates are listed, and is copied to M_H by thread 0
// with one bulk copy (the half's rows are contiguous in the buffer and in
// M_H); the threads then go on while the copy drains.  *bsel alternates the
// buffers across halves.  Hot rows of an overflowing pass are read back
// from the buffers.  dst: the pass's first M_H row.  All threads of the
// block call it.
template <bool U16>
__device__ __forceinline__ void bulk_flush_emit_pass(const Geom &g, const Work &w, const ScanArgs &a, ScanSmem &ss,
                                                     uint4 *pbuf, uint32_t &buf_n, uint32_t &nseq, uint32_t &total,
                                                     const ChunkList &inner, uint32_t *tile, uint32_t pitch,
                                                     uint32_t *dst, uint32_t pr, uint32_t iA, uint32_t slice_lin0,
                                                     uint32_t e, uint32_t *stg, uint32_t hrows, uint32_t &bsel,
                                                     uint32_t *lists, uint32_t *s_hot, uint32_t *s_nc)
{
    uint32_t *cand = lists, *candv = lists + kFusedCand, *srt = lists + 2 * kFusedCand, *srtv = lists + 3 * kFusedCand;
    const uint32_t tid = threadIdx.x, nb = g.nb;
    if (tid == 0)
        s_hot[0] = s_hot[1] = *s_nc = 0u;
    const uint32_t b0 = bsel;   // the first half's buffer; the second takes the other
    for (uint32_t h0 = 0; h0 < pr; h0 += hrows) {
        const uint32_t nr = min(hrows, pr - h0);
        uint32_t *S = stg + (size_t)bsel * hrows * nb;
        if (tid == 0)
            bulk_wait_read<1>();   // the copy that last read buffer bsel is done
        __syncthreads();           // (first half: the votes and the counter reset are done too)
        flush_tile<U16, true, false, BlockGroup, false>(g, tile, S, nr, pitch,
                                                        FlushList{s_hot, cand, candv, s_nc, kFusedCand}, h0);
        fence_proxy_async_smem();  // the buffer's generic writes, visible to the bulk copies
        __syncthreads();
        if (tid == 0) {
            bulk_store(dst + (size_t)h0 * nb, S, nr * nb * 4u);
            bulk_commit();
        }
        bsel ^= 1u;
    }
    const uint64_t hotm = (uint64_t)s_hot[0] | ((uint64_t)s_hot[1] << 32);
    const uint32_t n_c = *s_nc;
    if (n_c)
        emit_pass<BlockGroup, true>(g, w, a, ss, pbuf, buf_n, nseq, total, inner, cand, candv, srt, srtv, n_c, hotm,
                                    pr, iA, slice_lin0, e, stg + (size_t)b0 * hrows * nb,
                                    stg + (size_t)(b0 ^ 1u) * hrows * nb, hrows);
    __syncthreads();               // lists and counters free for the next pass
}

// The CTA's candidate bookkeeping once its range is done.
template <class G>
__device__ __forceinline__ void finish_candidates(const Work &w, const ScanArgs &a, ScanSmem &ss, const uint4 *pbuf,
                                                  uint32_t &buf_n, uint32_t &nseq, uint32_t total,
                                                  const ChunkList &inner, uint32_t cta)
{
    flush_chunk<G>(a, ss, pbuf, buf_n, nseq, inner, w.status);
    if (G::rank() == 0) {
        a.cta_nseq[cta] = min(nseq, a.seq_max);
        a.cta_total[cta] = total;
    }
}

// The body of both fused fills.  BULK (k_fill_bulk): the passes leave
// through two u32 staging buffers and bulk copies (bulk_flush_emit_pass),
// so the stores drain while the next votes run; else (k_fill_scan) the
// threads store each pass to M_H themselves (flush_emit_pass).
template <bool BULK>
__device__ __forceinline__ void fill_scan_body(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a)
{
    extern __shared__ uint4 sm4[];
    // layout: ScanSmem (256 B) | K entries | tile | [BULK: 2 staging buffers] | HC staged hits |
    //         B thresholds | candidate lists (keys, votes, sorted keys, sorted votes)
    ScanSmem &ss = *reinterpret_cast<ScanSmem *>(sm4);
    uint4 *pbuf = sm4 + 16;
    uint32_t *tile = reinterpret_cast<uint32_t *>(pbuf + a.K);
    uint32_t *stg = tile + c.tile_words;
    float4 *hs = reinterpret_cast<float4 *>(stg + (BULK ? staging_words(c, g.nb) : 0u));
    float *beta = reinterpret_cast<float *>(hs + c.HC);
    uint32_t *lists = reinterpret_cast<uint32_t *>(beta + c.beta_words);
    __shared__ uint32_t s_hot[2], s_nc;

    const uint32_t tid = threadIdx.x, bd = blockDim.x, nb = g.nb;
    for (uint32_t k = tid; k < c.tile_words / 4; k += bd)
        sm4[16 + a.K + k] = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t k = tid; k <= nb; k += bd)
        beta[k] = g.bth[k];
    grid_dep_wait();   // the unit lists of k_scatter
    const uint32_t cta = blockIdx.x;
    ChunkList inner = interior_list(a, cta);

    __shared__ unsigned long long s_rng[2];
    __shared__ uint32_t s_dyn;
    const uint64_t items = (uint64_t)w.n_events * g.n_slices * c.strips;
    const uint64_t n_dyn = c.dyn ? dyn_items(items, gridDim.x) : 0, n_static = items - n_dyn;
    uint64_t it0, it1;
    cta_items(g, w, c, cta, gridDim.x, n_static, it0, it1, s_rng);
    uint64_t cached_es = ~0ull;
    uint32_t cached_n = 0;
    uint32_t buf_n = 0, nseq = 0, total = 0;
    uint32_t bsel = 0;   // BULK: the staging buffer of the next half pass

    auto do_item = [&](const ItemCursor &cur) {
        const uint32_t k = cur.k;
        const uint64_t es = cur.es;
        const uint32_t s = cur.s;
        const uint32_t e = cur.e;
        const uint32_t l0 = __ldg(&w.slice_off[es]), l1 = __ldg(&w.slice_off[es + 1]);   // the unit's hits
        const uint32_t i0 = k * c.W;
        const uint32_t rows = min(c.W, g.na - i0);
        const bool u16 = (l1 - l0) < 65536u;
        const uint32_t rpass = u16 ? c.W : c.W / 2;
        const uint32_t pitch = u16 ? c.pitch16 : c.pitch32;
        const uint32_t slice_lin0 = s * g.na * nb;
        const uint32_t *Ms = w.M + (size_t)e * w.n_cells + slice_lin0;
        uint32_t *Mrow = w.M + (size_t)e * w.n_cells + ((size_t)s * g.na + i0) * g.nb;
        const uint32_t r = tid % rpass, hl = tid / rpass, hstride = bd / rpass;

        for (uint32_t p0 = 0; p0 < rows; p0 += rpass) {
            const uint32_t pr = min(rpass, rows - p0);
            const uint32_t iA = i0 + p0;
            // ---- vote (no barrier first: the previous pass, the previous item's
            // hand-out or the set-up ended with one) ---------------------------
            const uint32_t i = iA + r;
            vote_pass<BlockGroup, false, false>(g, w, tile, hs, beta, c.HC, es, l0, l1, cached_es, cached_n, u16, r, pr,
                                                i, hl, hstride, pitch, FlushList{});
            // ---- write the pass, clear the tile, emit its candidates --------
            if (BULK) {
                if (u16)
                    bulk_flush_emit_pass<true>(g, w, a, ss, pbuf, buf_n, nseq, total, inner, tile, pitch,
                                               Mrow + (size_t)p0 * nb, pr, iA, slice_lin0, e, stg, c.W / 2, bsel,
                                               lists, s_hot, &s_nc);
                else
                    bulk_flush_emit_pass<false>(g, w, a, ss, pbuf, buf_n, nseq, total, inner, tile, pitch,
                                                Mrow + (size_t)p0 * nb, pr, iA, slice_lin0, e, stg, c.W / 2, bsel,
                                                lists, s_hot, &s_nc);
            } else if (u16) {
                flush_emit_pass<BlockGroup, true>(g, w, a, ss, pbuf, buf_n, nseq, total, inner, tile, pitch,
                                                  Mrow + (size_t)p0 * nb, pr, iA, slice_lin0, e, Ms, lists, s_hot,
                                                  &s_nc, nullptr);
            } else {
                flush_emit_pass<BlockGroup, false>(g, w, a, ss, pbuf, buf_n, nseq, total, inner, tile, pitch,
                                                   Mrow + (size_t)p0 * nb, pr, iA, slice_lin0, e, Ms, lists, s_hot,
                                                   &s_nc, nullptr);
            }
        }
    };
    ItemCursor cur(g, c, it0);
    for (uint64_t item = it0; item < it1; ++item, cur.next(g, c))
        do_item(cur);
    finish_candidates<BlockGroup>(w, a, ss, pbuf, buf_n, nseq, total, inner, cta);
    if (c.dyn) {
        // handed-out items, each with its own list of chunks
        for (uint32_t d; (d = next_dyn_item(w, (uint32_t)n_dyn, &s_dyn)) < n_dyn;) {
            const uint32_t list = gridDim.x + d;
            inner = interior_list(a, list);
            buf_n = nseq = total = 0;
            do_item(ItemCursor(g, c, n_static + d));
            finish_candidates<BlockGroup>(w, a, ss, pbuf, buf_n, nseq, total, inner, list);
        }
    }
    if (BULK && threadIdx.x == 0)
        bulk_wait<0>();   // the last copies have written M_H (and read the staging) before the CTA ends
}

__global__ void __launch_bounds__(1024) k_fill_scan(Geom g, Work w, FillCfg c, ScanArgs a)
{
    fill_scan_body<false>(g, w, c, a);
}

__global__ void __launch_bounds__(1024) k_fill_bulk(Geom g, Work w, FillCfg c, ScanArgs a)
{
    fill_scan_body<true>(g, w, c, a);
}

// ---------------------------------------------------------------------------
// k_fill_tma: the fused fill with the tiles leaving by bulk copies.
//
// The tiles hold u32 counters in M_H's own layout (rows n_b cells apart, no
// swizzle), so a finished pass of W rows is one contiguous run of M_H and
// leaves the SM as a single bulk copy (cp.async.bulk, shared -> global) that
// one thread issues: no thread converts, stores or even reads the cells.
// Two tiles alternate: while the copy engine drains pass p's tile, the
// threads vote pass p + 1 into the other one; a tile is cleared once the
// copy that read it is done.  The votes themselves list the cells that
// reach the threshold (a returned count of T - 1), so no pass scans its
// tile for candidates.  The candidates go the way of k_fill_scan's (ranked,
// emitted as ordered entries, tested by k_peaks against the finished M_H).
// Needs n_b a multiple of 4 (16-byte rows); at most 64 rows per pass.
// ---------------------------------------------------------------------------

// A thread's share of the candidates q = r * nc + h of a pass over nc staged
// hits: q = tid, tid + blockDim, ..; (r0, h0) is its first, and each step
// adds dr rows and dh hits (carrying into r).  Fixed for a unit's staged
// hits, so the divisions are made once per staging, not once per pass.
struct FlatMap {
    uint32_t nc, r0, h0, dr, dh;
    __device__ __forceinline__ void set(uint32_t n)
    {
        nc = n;
        if (n) {
            r0 = threadIdx.x / n;
            h0 = threadIdx.x - r0 * n;
            dr = blockDim.x / n;
            dh = blockDim.x - dr * n;
        }
    }
};

// The votes of the staged hits hs[0 .. m.nc) into tile rows 0 .. pr - 1 (A
// bins iA ..): candidate q = r * nc + h goes to thread q % blockDim, so a
// warp's lanes take consecutive hits of one row (their B columns, and so
// their banks, are spread by the hits).  A vote that lifts its cell from
// T - 1 to T lists the cell as r * n_b + j.  AGG: warp-aggregated increments
// -- the lanes voting for the same cell find each other (match.any on the
// cell index) and their lowest lane adds their number with one atomic; the
// cell is listed by the add that takes it from below T to T or more.
template <bool AGG>
__device__ __forceinline__ void vote_flat(const Geom &g, uint32_t *tile, const float4 *hs, const float *beta,
                                          const FlatMap &m, uint32_t pr, uint32_t iA, const FlushList &L)
{
    const uint32_t nb = g.nb, nc = m.nc;
    if (nc == 0 || m.r0 >= pr)
        return;
    const uint32_t T = g.threshold, tm1 = T - 1u, lane = threadIdx.x & 31u;
    const float b_lo = beta[0], b_hi = beta[nb];
    uint32_t r = m.r0, h = m.h0;
#pragma unroll 2
    while (r < pr) {
        const float twoA = __fmul_rn(2.0f, a_centre(g, iA + r));
        const float4 hv = hs[h];
        const int j = vote_bin_tab(g, beta, b_lo, b_hi, twoA, hv.x, hv.y, hv.z);
        if (j >= 0) {
            const uint32_t key = r * nb + (uint32_t)j;
            if (AGG) {
                const uint32_t peers = __match_any_sync(__activemask(), key);
                if (lane == (uint32_t)(__ffs(peers) - 1)) {
                    const uint32_t n = (uint32_t)__popc(peers);
                    const uint32_t old = atomicAdd(&tile[key], n);
                    if (old < T && old + n >= T)
                        note_candidate(L, r, key);
                }
            } else if (atomicAdd(&tile[key], 1u) == tm1) {
                note_candidate(L, r, key);
            }
        }
        h += m.dh;
        r += m.dr;
        if (h >= nc) {
            h -= nc;
            ++r;
        }
    }
}

// One pass's votes from the hits of list entries l0 .. l1 of unit es,
// staged HC at a time (kept staged, with their FlatMap, for the unit's next
// passes when they fit, as vote_pass).  Starts with a block barrier in every
// case: the previous pass's clearing of this tile is complete.  All threads
// call it.
template <bool AGG>
__device__ __forceinline__ void vote_pass_flat(const Geom &g, const Work &w, uint32_t *tile, float4 *hs,
                                               const float *beta, uint32_t HC, uint64_t es, uint32_t l0, uint32_t l1,
                                               uint64_t &cached_es, FlatMap &cached, uint32_t pr, uint32_t iA,
                                               const FlushList &L)
{
    if (cached_es == es) {
        __syncthreads();
        vote_flat<AGG>(g, tile, hs, beta, cached, pr, iA, L);
        return;
    }
    cached_es = ~0ull;   // hs is about to be overwritten
    uint32_t pos = l0;
    bool first = true;
    while (first || pos < l1) {
        const uint32_t nsel = stage_hits<BlockGroup>(w, hs, HC, pos, l1);   // starts with a barrier
        FlatMap m;
        m.set(nsel);
        if (first && pos >= l1) {
            cached_es = es;
            cached = m;
        }
        first = false;
        vote_flat<AGG>(g, tile, hs, beta, m, pr, iA, L);
    }
}

// NT = 2 tiles rotate: after pass p's copy is issued, the copy of pass p - 1
// must have read its tile, which pass p + 1 then takes.  AGG: warp-aggregated
// vote increments (vote_flat).
template <bool AGG>
__global__ void __launch_bounds__(1024) k_fill_tma(Geom g, Work w, FillCfg c, ScanArgs a)
{
    constexpr int NT = 2;
    extern __shared__ uint4 sm4[];
    // layout: ScanSmem (256 B) | K entries | NT tiles | HC staged hits | B thresholds |
    //         candidate lists (keys, votes, sorted keys, sorted votes)
    ScanSmem &ss = *reinterpret_cast<ScanSmem *>(sm4);
    uint4 *pbuf = sm4 + 16;
    uint32_t *tiles = reinterpret_cast<uint32_t *>(pbuf + a.K);
    float4 *hs = reinterpret_cast<float4 *>(tiles + NT * c.tile_words);
    float *beta = reinterpret_cast<float *>(hs + c.HC);
    uint32_t *lists = reinterpret_cast<uint32_t *>(beta + c.beta_words);
    uint32_t *cand = lists, *candv = lists + kFusedCand, *srt = lists + 2 * kFusedCand,
             *srtv = lists + 3 * kFusedCand;
    __shared__ uint32_t s_hot[2], s_nc;

    const uint32_t tid = threadIdx.x, bd = blockDim.x, nb = g.nb;
    for (uint32_t k = tid; k < NT * c.tile_words / 4; k += bd)
        reinterpret_cast<uint4 *>(tiles)[k] = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t k = tid; k <= nb; k += bd)
        beta[k] = g.bth[k];
    if (tid == 0)
        s_hot[0] = s_hot[1] = s_nc = 0u;
    const uint32_t cta = blockIdx.x;
    ChunkList inner = interior_list(a, cta);

    // The static split reads only the unit offsets.  When k_bin wrote them
    // and k_scatter precedes this kernel (kSplitEarly), k_scatter lets it
    // launch only after k_bin has finished, so the split runs ahead of the
    // wait for k_scatter's lists; after k_bin_cluster the split is read
    // from what that kernel wrote (kSplitGiven), or computed after the wait.
    __shared__ unsigned long long s_rng[2];
    __shared__ uint32_t s_dyn;
    const uint64_t items = (uint64_t)w.n_events * g.n_slices * c.strips;
    const uint64_t n_dyn = c.dyn ? dyn_items(items, gridDim.x) : 0, n_static = items - n_dyn;
    uint64_t it0, it1;
    if (w.split_mode == kSplitEarly)
        cta_items(g, w, c, cta, gridDim.x, n_static, it0, it1, s_rng);
    grid_dep_wait();   // the unit lists (and, after k_bin_cluster, the offsets and split)
    if (w.split_mode == kSplitGiven && w.split_grid == gridDim.x && w.split_strips == c.strips &&
        w.split_vw == c.vote_weight && w.split_n_static == n_static) {
        it0 = __ldcg(&w.split[cta]);
        it1 = __ldcg(&w.split[cta + 1]);
    } else if (w.split_mode != kSplitEarly) {
        cta_items(g, w, c, cta, gridDim.x, n_static, it0, it1, s_rng);
    }
    uint64_t cached_es = ~0ull;
    FlatMap cached{};
    uint32_t buf_n = 0, nseq = 0, total = 0;
    uint32_t tsel = 0;   // the tile of the next pass

    auto do_item = [&](const ItemCursor &cur) {
        const uint64_t es = cur.es;
        const uint32_t e = cur.e;
        const uint32_t l0 = __ldg(&w.slice_off[es]), l1 = __ldg(&w.slice_off[es + 1]);   // the unit's hits
        const uint32_t iA = cur.k * c.W;
        const uint32_t pr = min(c.W, g.na - iA);
        const uint32_t slice_lin0 = cur.s * g.na * nb;
        uint32_t *tile = tiles + (size_t)tsel * c.tile_words;

        // ---- vote (tile tsel is clear, the lists empty) ------------------------
        vote_pass_flat<AGG>(g, w, tile, hs, beta, c.HC, es, l0, l1, cached_es, cached, pr, iA,
                       FlushList{s_hot, cand, candv, &s_nc, kFusedCand});
        fence_proxy_async_smem();   // the tile's counts, visible to the copy engine
        __syncthreads();            // votes and lists complete
        // ---- the pass leaves as one bulk copy ------------------------------------
        if (tid == 0) {
            bulk_store_evict_first(w.M + (size_t)e * w.n_cells + slice_lin0 + (size_t)iA * nb, tile, pr * nb * 4u);
            bulk_commit();
        }
        // ---- its candidates, votes read from the tile (the copy only reads it) --
        const uint32_t n_c = s_nc;
        const uint64_t hotm = (uint64_t)s_hot[0] | ((uint64_t)s_hot[1] << 32);
        if (n_c)
            emit_pass<BlockGroup, true, true>(g, w, a, ss, pbuf, buf_n, nseq, total, inner, cand, candv, srt, srtv,
                                              n_c, hotm, pr, iA, slice_lin0, e, tile, nullptr, pr);
        // ---- the next pass's tile: the copy that last read it is done -------------
        const uint32_t next = tsel + 1u == (uint32_t)NT ? 0u : tsel + 1u;
        if (tid == 0)
            bulk_wait_read<NT - 1>();
        __syncthreads();            // the lists are consumed; the next tile is free
        uint4 *nt = reinterpret_cast<uint4 *>(tiles + (size_t)next * c.tile_words);
#pragma unroll 4
        for (uint32_t k = tid; k < c.tile_words / 4; k += bd)
            nt[k] = make_uint4(0u, 0u, 0u, 0u);
        if (tid == 0)
            s_hot[0] = s_hot[1] = s_nc = 0u;
        tsel = next;                // the next pass's votes start with a barrier
    };
    // the first run-time item is claimed during the last static one, each
    // next one during the item before it (thread 0's claim stays in flight)
    const bool dyn = c.dyn && n_dyn > 0;
    uint32_t claim = 0;
    if (dyn && tid == 0 && it1 <= it0)
        claim = dyn_claim(w, (uint32_t)n_dyn);
    ItemCursor cur(g, c, it0);
    for (uint64_t item = it0; item < it1; ++item, cur.next(g, c)) {
        if (dyn && tid == 0 && item + 1 == it1)
            claim = dyn_claim(w, (uint32_t)n_dyn);
        do_item(cur);
    }
    finish_candidates<BlockGroup>(w, a, ss, pbuf, buf_n, nseq, total, inner, cta);
    if (dyn) {
        // handed-out items, each with its own list of chunks
        for (uint32_t d; (d = dyn_take(w, (uint32_t)n_dyn, claim, &s_dyn)) < n_dyn;) {
            if (tid == 0)
                claim = dyn_claim(w, (uint32_t)n_dyn);
            const uint32_t list = gridDim.x + d;
            inner = interior_list(a, list);
            buf_n = nseq = total = 0;
            do_item(ItemCursor(g, c, n_static + d));
            finish_candidates<BlockGroup>(w, a, ss, pbuf, buf_n, nseq, total, inner, list);
        }
    }
    if (tid == 0)
        bulk_wait<0>();   // the last copies have written M_H (and read the tiles) before the CTA ends
}

// ---------------------------------------------------------------------------
// k_fill_peaks: the fused fill without M_H in HBM (peaks-only fills).
//
// The passes are voted as in k_fill_scan, but the tile is not written out.
// The votes themselves list the cells that reach T (vote_rows with LIST),
// so no pass scans its tile for candidates: the listed cells are tested at
// once against the neighbours the tile holds, and the pass's first and last
// rows go to a small edge buffer.  A cell on the first (last) row of its
// pass whose row above (below) belongs to another pass is emitted with a
// flag; k_peaks finishes its test from the edge rows.  The output is the
// same ordered peak list; M_H is left as it was.
// ---------------------------------------------------------------------------

// Test of cell (r, j) with votes v against the neighbours inside the tile
// rows 0 .. pr - 1 (rule of Sec. 3 as read: > neighbours before it, >= after).
__device__ __forceinline__ bool tile_peak(const uint32_t *tile, uint32_t pitch, bool u16, uint32_t pr, uint32_t nb,
                                          uint32_t r, uint32_t j, uint32_t v)
{
    const bool hl = j > 0, hr = j + 1 < nb;
    if (r > 0) {
        if (hl && !(v > tile_cell(tile, pitch, u16, r - 1, j - 1))) return false;
        if (!(v > tile_cell(tile, pitch, u16, r - 1, j))) return false;
        if (hr && !(v > tile_cell(tile, pitch, u16, r - 1, j + 1))) return false;
    }
    if (hl && !(v > tile_cell(tile, pitch, u16, r, j - 1))) return false;
    if (hr && !(v >= tile_cell(tile, pitch, u16, r, j + 1))) return false;
    if (r + 1 < pr) {
        if (hl && !(v >= tile_cell(tile, pitch, u16, r + 1, j - 1))) return false;
        if (!(v >= tile_cell(tile, pitch, u16, r + 1, j))) return false;
        if (hr && !(v >= tile_cell(tile, pitch, u16, r + 1, j + 1))) return false;
    }
    return true;
}

// Copy the first and last rows of a voted pass (tile rows 0 and rows - 1)
// to edge[0, n_b) and edge[n_b, 2 n_b), 4 cells per thread and step when
// n_b % 4 == 0.  The tile is left as it is.
template <bool U16>
__device__ __forceinline__ void edge_rows(const Geom &g, const uint32_t *tile, uint32_t rows, uint32_t pitch,
                                          uint32_t *edge)
{
    const uint32_t tid = threadIdx.x, bd = blockDim.x, nb = g.nb;
    if ((nb & 3u) == 0) {
        const uint32_t q = nb >> 2;
        for (uint32_t u = tid; u < 2 * q; u += bd) {
            const uint32_t side = u >= q, c4 = u - side * q, r = side ? rows - 1 : 0;
            uint4 v;
            if (U16) {
                const uint2 pr =
                    *reinterpret_cast<const uint2 *>(&tile[r * pitch + ((2u * c4) ^ (row_hash(r) & 0x1Eu))]);
                v = make_uint4(pr.x & 0xffffu, pr.x >> 16, pr.y & 0xffffu, pr.y >> 16);
            } else {
                v = *reinterpret_cast<const uint4 *>(&tile[r * pitch + ((4u * c4) ^ (row_hash(r) & 0x1Cu))]);
            }
            reinterpret_cast<uint4 *>(edge)[u] = v;
        }
    } else {
        for (uint32_t u = tid; u < 2 * nb; u += bd) {
            const uint32_t side = u >= nb, j = u - side * nb;
            edge[u] = tile_cell(tile, pitch, U16, side ? rows - 1 : 0, j);
        }
    }
}

// Edge-flag bits of a peaks-only entry (in its .w): its test still needs
// the row above / below, which lies in another pass.
enum : uint32_t { EDGE_UP = 1u, EDGE_DN = 2u };

__global__ void __launch_bounds__(1024) k_fill_peaks(Geom g, Work w, FillCfg c, ScanArgs a)
{
    extern __shared__ uint4 sm4[];
    // layout as k_fill_scan
    ScanSmem &ss = *reinterpret_cast<ScanSmem *>(sm4);
    uint4 *pbuf = sm4 + 16;
    uint32_t *tile = reinterpret_cast<uint32_t *>(pbuf + a.K);
    float4 *hs = reinterpret_cast<float4 *>(tile + c.tile_words);
    float *beta = reinterpret_cast<float *>(hs + c.HC);
    uint32_t *lists = reinterpret_cast<uint32_t *>(beta + c.beta_words);
    uint32_t *cand = lists, *srt = lists + 2 * kFusedCand, *srtv = lists + 3 * kFusedCand;
    __shared__ uint32_t s_hot[2], s_nc;

    const uint32_t tid = threadIdx.x, bd = blockDim.x, nb = g.nb, T = g.threshold;
    if (tid == 0)
        s_hot[0] = s_hot[1] = s_nc = 0u;
    for (uint32_t k = tid; k < c.tile_words / 4; k += bd)
        sm4[16 + a.K + k] = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t k = tid; k <= nb; k += bd)
        beta[k] = g.bth[k];
    const uint32_t cta = blockIdx.x;
    ChunkList inner = interior_list(a, cta);

    // the static split as in k_fill_tma (Work::split_mode)
    __shared__ unsigned long long s_rng[2];
    __shared__ uint32_t s_dyn;
    const uint64_t items = (uint64_t)w.n_events * g.n_slices * c.strips;
    const uint64_t n_dyn = c.dyn ? dyn_items(items, gridDim.x) : 0, n_static = items - n_dyn;
    uint64_t it0, it1;
    if (w.split_mode == kSplitEarly)
        cta_items(g, w, c, cta, gridDim.x, n_static, it0, it1, s_rng);
    grid_dep_wait();   // the unit lists (and, after k_bin_cluster, the offsets and split)
    if (w.split_mode == kSplitGiven && w.split_grid == gridDim.x && w.split_strips == c.strips &&
        w.split_vw == c.vote_weight && w.split_n_static == n_static) {
        it0 = __ldcg(&w.split[cta]);
        it1 = __ldcg(&w.split[cta + 1]);
    } else if (w.split_mode != kSplitEarly) {
        cta_items(g, w, c, cta, gridDim.x, n_static, it0, it1, s_rng);
    }
    uint64_t cached_es = ~0ull;
    uint32_t cached_n = 0;
    uint32_t buf_n = 0, nseq = 0, total = 0;
    const uint32_t rc = fused_round(bd, a.K);

    auto do_item = [&](const ItemCursor &cur) {
        const uint32_t k = cur.k;
        const uint64_t es = cur.es;
        const uint32_t s = cur.s;
        const uint32_t e = cur.e;
        const uint32_t l0 = __ldg(&w.slice_off[es]), l1 = __ldg(&w.slice_off[es + 1]);
        const uint32_t i0 = k * c.W;
        const uint32_t rows = min(c.W, g.na - i0);
        const bool u16 = (l1 - l0) < 65536u;
        const uint32_t rpass = u16 ? c.W : c.W / 2;
        const uint32_t pitch = u16 ? c.pitch16 : c.pitch32;
        const uint32_t slice_lin0 = s * g.na * nb;
        const uint32_t r = tid % rpass, hl = tid / rpass, hstride = bd / rpass;

        for (uint32_t p0 = 0; p0 < rows; p0 += rpass) {
            const uint32_t pr = min(rpass, rows - p0);
            const uint32_t iA = i0 + p0;
            // ---- vote -------------------------------------------------------
            const uint32_t i = iA + r;
            const FlushList L{s_hot, lists, nullptr, &s_nc, kFusedCand};
            vote_pass<BlockGroup, true, true>(g, w, tile, hs, beta, c.HC, es, l0, l1, cached_es, cached_n, u16, r, pr,
                                              i, hl, hstride, pitch, L);
            __syncthreads();   // the pass's votes and their candidate list are complete
            const uint32_t n_c = s_nc;
            const uint64_t hotm = (uint64_t)s_hot[0] | ((uint64_t)s_hot[1] << 32);
            // ---- the pass's first and last rows to the edge buffer ------------
            const uint32_t pass = iA / rpass;
            uint32_t *edge = w.edge + ((size_t)es * w.edge_pass + pass) * 2 * nb;
            if (u16)
                edge_rows<true>(g, tile, pr, pitch, edge);
            else
                edge_rows<false>(g, tile, pr, pitch, edge);
            const bool up_out = iA > 0, dn_out = iA + pr < g.na;   // neighbours in other passes
            // ---- test against the tile, emit peaks and flagged edge cells ----
            if (n_c) {
                const bool fits = n_c <= kFusedCand;
                if (fits) {
                    if (u16)
                        sort_tile_candidates<BlockGroup, true>(g, tile, pitch, cand, n_c, srt, srtv);
                    else
                        sort_tile_candidates<BlockGroup, false>(g, tile, pitch, cand, n_c, srt, srtv);
                    __syncthreads();
                }
                // rounds of rc cells: the sorted list, or every cell of the hot rows
                const uint32_t m_total = fits ? n_c : pr * nb;
                for (uint32_t base = 0; base < m_total; base += rc) {
                    const uint32_t q = base + tid;
                    uint32_t has = 0;
                    uint4 ent = make_uint4(0u, 0u, 0u, 0u);
                    if (tid < rc && q < m_total) {
                        uint32_t key, v;
                        bool ok = true;
                        if (fits) {
                            key = srt[q];
                            v = srtv[q];
                        } else {
                            key = q;
                            const uint32_t rr = q / nb;
                            ok = (hotm >> rr) & 1ull;
                            v = ok ? tile_cell(tile, pitch, u16, rr, q - rr * nb) : 0u;
                            ok = ok && v >= T;
                        }
                        if (ok) {
                            const uint32_t rr = key / nb, j = key - rr * nb;
                            if (tile_peak(tile, pitch, u16, pr, nb, rr, j, v)) {
                                const uint32_t flags = (rr == 0 && up_out ? EDGE_UP : 0u) |
                                                       (rr == pr - 1 && dn_out ? EDGE_DN : 0u);
                                has = 1;
                                ent = make_uint4(slice_lin0 + iA * nb + key, e, v, flags);
                            }
                        }
                    }
                    if (__syncthreads_or(has)) {
                        if (buf_n + rc > a.K)
                            flush_chunk(a, ss, pbuf, buf_n, nseq, inner, w.status);
                        compact_entry<BlockGroup, false>(ss, pbuf, buf_n, has, ent, nullptr);
                        total += ss.round_total;
                    }
                }
            }
            __syncthreads();
            // ---- clear the tile and the lists for the next pass ----------------
            for (uint32_t q = tid; q < pr * pitch / 4; q += bd)
                reinterpret_cast<uint4 *>(tile)[q] = make_uint4(0u, 0u, 0u, 0u);
            if (tid == 0)
                s_hot[0] = s_hot[1] = s_nc = 0u;   // the next votes start with a barrier
        }
    };
    ItemCursor cur(g, c, it0);
    for (uint64_t item = it0; item < it1; ++item, cur.next(g, c))
        do_item(cur);
    finish_candidates<BlockGroup>(w, a, ss, pbuf, buf_n, nseq, total, inner, cta);
    if (c.dyn) {
        for (uint32_t d; (d = next_dyn_item(w, (uint32_t)n_dyn, &s_dyn)) < n_dyn;) {
            const uint32_t list = gridDim.x + d;
            inner = interior_list(a, list);
            buf_n = nseq = total = 0;
            do_item(ItemCursor(g, c, n_static + d));
            finish_candidates<BlockGroup>(w, a, ss, pbuf, buf_n, nseq, total, inner, list);
        }
    }
}

// ---------------------------------------------------------------------------
// k_fill_ws: the fused fill with warp specialisation, one CTA per SM.
//
// 1024 threads in two groups of 16 warps: the vote group stages hits and
// votes strip passes into one of two shared-memory tiles while the flush
// group writes the other tile to M_H, clears it and emits its candidates
// (exactly as k_fill_scan does).  Tiles change hands through mbarriers --
// FULL[b] (512 vote arrivals: tile b holds a pass) and EMPTY[b] (512 flush
// arrivals: tile b is clear again) -- with bounded waits, so the votes of
// pass p + 1 run while pass p streams to HBM.  Each group keeps to its own
// named barrier; a wait that gives up makes its whole group leave (decided
// by a group-wide vote) after flagging ST_WAIT_TIMEOUT, and the other
// group's waits then give up too.
// ---------------------------------------------------------------------------
using VoteGroup = WarpGroup<1, 0, 512>;
using FlushGroup = WarpGroup<2, 512, 512>;

// Geometry of one (event, slice, strip) work item.
struct ItemInfo {
    uint64_t es;
    uint32_t s, e, l0, l1, i0, rows, rpass, pitch;   // l0, l1: the unit's hit list
    bool u16;
};

__device__ __forceinline__ ItemInfo item_info(const Geom &g, const Work &w, const FillCfg &c, const ItemCursor &cur)
{
    ItemInfo t;
    const uint32_t k = cur.k;
    t.es = cur.es;
    t.s = cur.s;
    t.e = cur.e;
    t.l0 = __ldg(&w.slice_off[t.es]);
    t.l1 = __ldg(&w.slice_off[t.es + 1]);
    t.i0 = k * c.W;
    t.rows = min(c.W, g.na - t.i0);
    t.u16 = (t.l1 - t.l0) < 65536u;
    t.rpass = t.u16 ? c.W : c.W / 2;
    t.pitch = t.u16 ? c.pitch16 : c.pitch32;
    return t;
}

__global__ void __launch_bounds__(1024, 1) k_fill_ws(Geom g, Work w, FillCfg c, ScanArgs a)
{
    extern __shared__ uint4 sm4[];
    // layout: ScanSmem (256 B) | K entries | 2 tiles | HC staged hits | B thresholds |
    //         candidate lists | 4 mbarriers (FULL 0, FULL 1, EMPTY 0, EMPTY 1)
    ScanSmem &ss = *reinterpret_cast<ScanSmem *>(sm4);
    uint4 *pbuf = sm4 + 16;
    uint32_t *tiles = reinterpret_cast<uint32_t *>(pbuf + a.K);
    float4 *hs = reinterpret_cast<float4 *>(tiles + 2 * (size_t)c.tile_words);
    float *beta = reinterpret_cast<float *>(hs + c.HC);
    uint32_t *lists = reinterpret_cast<uint32_t *>(beta + c.beta_words);
    uint64_t *bars = reinterpret_cast<uint64_t *>(lists + 4 * kFusedCand);
    __shared__ uint32_t s_hot[2], s_nc;

    const uint32_t tid = threadIdx.x, nb = g.nb;
    for (uint32_t k = tid; k < c.tile_words / 2; k += blockDim.x)
        reinterpret_cast<uint4 *>(tiles)[k] = make_uint4(0u, 0u, 0u, 0u);
    for (uint32_t k = tid; k <= nb; k += blockDim.x)
        beta[k] = g.bth[k];
    if (tid == 0) {
        for (uint32_t q = 0; q < 4; ++q)
            mbar_init(&bars[q], VoteGroup::size());
        fence_mbar_init();
    }
    __syncthreads();   // the last block-wide barrier: the groups part here
    grid_dep_wait();   // the unit lists of k_scatter

    const uint32_t cta = blockIdx.x;
    __shared__ unsigned long long s_rng[2][2];

    if (tid < VoteGroup::size()) {
        // ---------------- vote group ----------------
        const uint32_t vr = VoteGroup::rank();
        uint64_t it0, it1;
        cta_items<VoteGroup>(g, w, c, cta, gridDim.x, (uint64_t)w.n_events * g.n_slices * c.strips, it0, it1,
                             s_rng[0]);
        uint64_t cached_es = ~0ull;
        uint32_t cached_n = 0, p = 0;
        ItemCursor cur(g, c, it0);
        for (uint64_t item = it0; item < it1; ++item, cur.next(g, c)) {
            const ItemInfo t = item_info(g, w, c, cur);
            const uint32_t r = vr % t.rpass, hl = vr / t.rpass, hstride = VoteGroup::size() / t.rpass;
            for (uint32_t p0 = 0; p0 < t.rows; p0 += t.rpass, ++p) {
                const uint32_t pr = min(t.rpass, t.rows - p0);
                const uint32_t b = p & 1u;
                uint32_t *tile = tiles + (size_t)b * c.tile_words;
                if (p >= 2) {
                    const bool ok = mbar_wait_bounded(&bars[2 + b], ((p >> 1) - 1u) & 1u);
                    if (VoteGroup::sync_or(!ok)) {
                        if (vr == 0)
                            atomicOr(w.status, (uint32_t)ST_WAIT_TIMEOUT);
                        return;
                    }
                }
                const uint32_t i = t.i0 + p0 + r;
                vote_pass<VoteGroup, false, false>(g, w, tile, hs, beta, c.HC, t.es, t.l0, t.l1, cached_es, cached_n,
                                                   t.u16, r, pr, i, hl, hstride, t.pitch, FlushList{});
                mbar_arrive(&bars[b]);   // tile b holds pass p
            }
        }
        return;
    }

    // ---------------- flush + emit group ----------------
    const uint32_t fr = FlushGroup::rank();
    uint64_t it0, it1;
    cta_items<FlushGroup>(g, w, c, cta, gridDim.x, (uint64_t)w.n_events * g.n_slices * c.strips, it0, it1,
                          s_rng[1]);
    const ChunkList inner = interior_list(a, cta);
    uint32_t buf_n = 0, nseq = 0, total = 0, p = 0;
    bool alive = true;
    ItemCursor cur(g, c, it0);
    for (uint64_t item = it0; item < it1 && alive; ++item, cur.next(g, c)) {
        const ItemInfo t = item_info(g, w, c, cur);
        const uint32_t slice_lin0 = t.s * g.na * nb;
        const uint32_t *Ms = w.M + (size_t)t.e * w.n_cells + slice_lin0;
        uint32_t *Mrow = w.M + (size_t)t.e * w.n_cells + ((size_t)t.s * g.na + t.i0) * nb;
        for (uint32_t p0 = 0; p0 < t.rows; p0 += t.rpass, ++p) {
            const uint32_t pr = min(t.rpass, t.rows - p0);
            const uint32_t b = p & 1u;
            uint32_t *tile = tiles + (size_t)b * c.tile_words;
            const bool ok = mbar_wait_bounded(&bars[b], (p >> 1) & 1u);
            if (FlushGroup::sync_or(!ok)) {
                if (fr == 0)
                    atomicOr(w.status, (uint32_t)ST_WAIT_TIMEOUT);
                alive = false;
                break;
            }
            if (t.u16)
                flush_emit_pass<FlushGroup, true>(g, w, a, ss, pbuf, buf_n, nseq, total, inner, tile, t.pitch,
                                                  Mrow + (size_t)p0 * nb, pr, t.i0 + p0, slice_lin0, t.e, Ms, lists,
                                                  s_hot, &s_nc, &bars[2 + b]);
            else
                flush_emit_pass<FlushGroup, false>(g, w, a, ss, pbuf, buf_n, nseq, total, inner, tile, t.pitch,
                                                   Mrow + (size_t)p0 * nb, pr, t.i0 + p0, slice_lin0, t.e, Ms, lists,
                                                   s_hot, &s_nc, &bars[2 + b]);
        }
    }
    finish_candidates<FlushGroup>(w, a, ss, pbuf, buf_n, nseq, total, inner, cta);
    (void)fr;
}

// ---------------------------------------------------------------------------
// k_peaks: after a fused fill (same grid), each CTA tests its candidate
// entries against their neighbours in the now complete M_H and compacts
// every chunk in place to its peaks (order kept), counting them per event.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_peaks(Geom g, Work w, FillCfg c, ScanArgs a, uint32_t peaks_only)
{
    grid_dep_wait();
    __shared__ uint32_t s_wsum[40];
    const uint32_t tid = threadIdx.x, bd = blockDim.x, cta = blockIdx.x;
    const uint32_t warp = tid >> 5, lane = tid & 31u, nw = (bd + 31) >> 5;
    const uint32_t nseq = a.cta_nseq[cta], sl = g.na * g.nb;
    uint32_t total = 0;
    for (uint32_t q = 0; q < nseq; ++q) {
        uint2 *dp = &a.desc[(size_t)cta * a.seq_max + q];
        const uint2 d = *dp;
        uint32_t kept = 0;
        for (uint32_t base = 0; base < d.y; base += bd) {
            const uint32_t k = base + tid;
            uint32_t has = 0;
            uint4 en = make_uint4(0u, 0u, 0u, 0u);
            if (k < d.y && d.x + k < a.entries_cap) {
                en = a.entries[d.x + k];
                const uint32_t s = en.x / sl, rem = en.x - s * sl, i = rem / g.nb, j = rem - i * g.nb;
                if (!peaks_only) {
                    const uint32_t *row = w.M + (size_t)en.y * w.n_cells + (size_t)(s * g.na + i) * g.nb;
                    has = is_peak_l2(row, i > 0 ? row - g.nb : nullptr, i + 1 < g.na ? row + g.nb : nullptr, j,
                                     g.nb, en.z) ? 1u : 0u;
                } else {
                    // the rows above / below from the edge rows of the neighbouring passes
                    const uint32_t u = en.y * g.n_slices + s;
                    const bool u16 = (__ldg(&w.slice_off[u + 1]) - __ldg(&w.slice_off[u])) < 65536u;
                    const uint32_t rpass = u16 ? c.W : c.W / 2, pass = i / rpass;
                    const uint32_t *eu = w.edge + (size_t)u * w.edge_pass * 2 * g.nb;
                    const uint32_t *up = (en.w & EDGE_UP) ? eu + ((size_t)(pass - 1) * 2 + 1) * g.nb : nullptr;
                    const uint32_t *dn = (en.w & EDGE_DN) ? eu + ((size_t)(pass + 1) * 2) * g.nb : nullptr;
                    const bool hl = j > 0, hr = j + 1 < g.nb;
                    const uint32_t v = en.z;
                    bool ok = true;
                    if (up)
                        ok = (!hl || v > __ldcg(up + j - 1)) && v > __ldcg(up + j) && (!hr || v > __ldcg(up + j + 1));
                    if (dn)
                        ok = ok && (!hl || v >= __ldcg(dn + j - 1)) && v >= __ldcg(dn + j) &&
                             (!hr || v >= __ldcg(dn + j + 1));
                    has = ok ? 1u : 0u;
                    en.w = 0u;
                }
            }
            // stable compaction: every read of this round happens before the
            // barrier, every write after, and no write passes its own read
            const uint32_t incl = warp_incl_scan(has);
            if (lane == 31u)
                s_wsum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                const uint32_t v = lane < nw ? s_wsum[lane] : 0u;
                const uint32_t vi = warp_incl_scan(v);
                s_wsum[lane] = vi - v;
                if (lane == 31u)
                    s_wsum[32] = vi;
            }
            __syncthreads();
            if (has) {
                a.entries[d.x + kept + s_wsum[warp] + incl - 1] = en;
                atomicAdd(&a.ev_count[en.y], 1u);
            }
            kept += s_wsum[32];
            __syncthreads();
        }
        if (tid == 0)
            dp->y = kept;
        total += kept;
    }
    if (tid == 0)
        a.cta_total[cta] = total;
}

// Ascending bitonic sort of n <= kCand words in shared memory (block-wide).
__device__ void sort_u32(uint32_t *s, uint32_t n)
{
    if (n < 2)
        return;
    uint32_t P = 1;
    while (P < n)
        P <<= 1;
    for (uint32_t i = n + threadIdx.x; i < P; i += blockDim.x)
        s[i] = 0xffffffffu;
    __syncthreads();
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const uint32_t x = s[i], y = s[l];
                    if ((x > y) == ((i & k) == 0)) {
                        s[i] = y;
                        s[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Test sorted candidate cells (run-local indices from global row g0) against
// their neighbours in M_H and append the peaks in order.
__device__ void test_candidates(const Geom &g, const Work &w, const ScanArgs &a, ScanSmem &ss, uint4 *pbuf,
                                uint32_t &buf_n, uint32_t &nseq, uint32_t &total, uint64_t g0,
                                const uint32_t *cand, uint32_t n)
{
    const uint32_t tid = threadIdx.x, bd = blockDim.x, nb = g.nb;
    const uint64_t rows_ev = (uint64_t)g.n_slices * g.na;
    for (uint32_t base = 0; base < n; base += bd) {
        const uint32_t k = base + tid;
        uint32_t has = 0;
        uint4 ent = make_uint4(0u, 0u, 0u, 0u);
        if (k < n) {
            const uint32_t idx = cand[k];
            const uint64_t gr = g0 + idx / nb;
            const uint32_t j = idx % nb;
            const uint32_t i = (uint32_t)(gr % g.na);
            const uint32_t ev = (uint32_t)(gr / rows_ev);
            const uint32_t *row = w.M + gr * nb;
            const uint32_t v = row[j];
            if (is_peak(row, i > 0 ? row - nb : nullptr, i + 1 < g.na ? row + nb : nullptr, j, nb, v)) {
                has = 1;
                ent = make_uint4((uint32_t)((gr - (uint64_t)ev * rows_ev) * nb) + j, ev, v, 0u);
            }
        }
        if (__syncthreads_or(has)) {
            if (buf_n + bd > a.K)
                flush_chunk(a, ss, pbuf, buf_n, nseq, interior_list(a, blockIdx.x), w.status);
            compact_entry(ss, pbuf, buf_n, has, ent, a.ev_count);
            total += ss.round_total;
        }
    }
}

// Register-streaming scan (n_b % 4 == 0): many resident warps per SM, each
// thread keeps kLdgUPT independent 16-byte streaming loads in flight; a chunk
// of a.R rows (kLdgUPT 16-byte units per thread) costs one block vote.

__global__ void __launch_bounds__(256) k_scan_ldg(Geom g, Work w, ScanArgs a)
{
    grid_dep_wait();
    extern __shared__ uint4 sm4[];
    ScanSmem &ss = *reinterpret_cast<ScanSmem *>(sm4);
    uint4 *pbuf = sm4 + 16;
    const uint32_t tid = threadIdx.x, bd = blockDim.x;
    const uint32_t nb = g.nb, nb4 = nb >> 2, T = g.threshold;
    const uint64_t G = (uint64_t)g.n_slices * g.na * w.n_events;
    const uint64_t g0 = G * blockIdx.x / gridDim.x, g1 = G * (blockIdx.x + 1) / gridDim.x;
    const uint32_t RC = a.R;
    uint32_t buf_n = 0, nseq = 0, total = 0;
    // pass 1: stream the run with no block barrier; collect the cells >= T
    // (run-local index) in a shared list, and mark their chunks (RC rows) in
    // a shared bitmap for when the list overflows
    uint32_t *hot = reinterpret_cast<uint32_t *>(pbuf + a.K);
    uint32_t *cand = hot + a.hot_words;
    __shared__ uint32_t s_ncand;
    const uint64_t n_chunks = (g1 - g0 + RC - 1) / RC;
    for (uint32_t k = tid; k < (n_chunks + 31) / 32; k += bd)
        hot[k] = 0u;
    if (tid == 0)
        s_ncand = 0u;
    __syncthreads();
    const uint4 *run = reinterpret_cast<const uint4 *>(w.M + g0 * nb);
    const uint64_t n4 = (g1 - g0) * nb4, per_chunk = (uint64_t)RC * nb4;
    for (uint64_t u0 = 0; u0 < n4; u0 += (uint64_t)kLdgUPT * bd) {
        uint4 v[kLdgUPT];
#pragma unroll
        for (uint32_t q = 0; q < kLdgUPT; ++q) {
            const uint64_t u = u0 + (uint64_t)q * bd + tid;
            v[q] = u < n4 ? __ldcs(run + u) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (uint32_t q = 0; q < kLdgUPT; ++q)
            if (max(max(v[q].x, v[q].y), max(v[q].z, v[q].w)) >= T) {
                const uint64_t u = u0 + (uint64_t)q * bd + tid;
                const uint64_t c = u / per_chunk;
                atomicOr(&hot[c >> 5], 1u << (c & 31u));
                const uint32_t vv[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
                for (uint32_t m = 0; m < 4; ++m)
                    if (vv[m] >= T) {
                        const uint32_t p = atomicAdd(&s_ncand, 1u);
                        if (p < kCand)
                            cand[p] = (uint32_t)(4 * u + m);
                    }
            }
    }
    __syncthreads();
    const uint32_t n_cand = s_ncand;
    if (n_cand <= kCand && (g1 - g0) * nb < (1ull << 32)) {
        // pass 2: the candidates in linear order, tested one per thread
        sort_u32(cand, n_cand);
        test_candidates(g, w, a, ss, pbuf, buf_n, nseq, total, g0, cand, n_cand);
    } else {
        // too many: detailed pass over the marked chunks
        for (uint64_t c = 0; c < n_chunks; ++c) {
            if (!((hot[c >> 5] >> (c & 31u)) & 1u))
                continue;
            const uint64_t ra = g0 + c * RC, rb = min(ra + RC, g1);
            scan_rows_slow<4>(g, w, a, ss, pbuf, buf_n, nseq, total, ra, rb, w.M, 0);
        }
    }
    flush_chunk(a, ss, pbuf, buf_n, nseq, interior_list(a, blockIdx.x), w.status);
    if (tid == 0) {
        a.cta_nseq[blockIdx.x] = min(nseq, a.seq_max);
        a.cta_total[blockIdx.x] = total;
    }
}

// ---------------------------------------------------------------------------
// k_order: one warp per list of chunks (a scan CTA's or a fused-fill list),
// eight lists per CTA; a list's rank is the peak total of the lists before it.
// ---------------------------------------------------------------------------
// The 32-byte output record of entry {lin within event, event, votes, .}.
__device__ __forceinline__ Peak peak_record(const Geom &g, const uint4 &en)
{
    const uint32_t lin = en.x;
    const uint32_t s = lin / (g.na * g.nb);
    const uint32_t rem = lin - s * (g.na * g.nb);
    const uint32_t i = rem / g.nb, j = rem - i * g.nb;
    Peak pk;
    pk.itheta = s / g.np;
    pk.iphi = s - pk.itheta * g.np;
    pk.ia = i;
    pk.ib = j;
    pk.votes = en.z;
    pk.a_c = a_centre(g, i);
    pk.b_c = b_centre(g, j);
    pk.event = en.y;
    return pk;
}

__global__ void __launch_bounds__(256) k_order(Geom g, Work w, ScanArgs a, OrderArgs o)
{
    grid_dep_wait();
    extern __shared__ uint32_t smo[];
    uint32_t *ev_base = smo;                  // n_events + 1
    uint32_t *red = ev_base + w.n_events + 1; // 40
    __shared__ uint32_t s_tot[32], s_last;
    const uint32_t tid = threadIdx.x, bd = blockDim.x, warp = tid >> 5, lane = tid & 31u, nw = bd >> 5;
    // one list per warp: lists c0 .. c0 + nw - 1
    const uint32_t c0 = blockIdx.x * nw, c = c0 + warp;
    const bool valid = c < a.grid;
    const uint32_t nseq = valid ? a.cta_nseq[c] : 0u, mine = valid ? a.cta_total[c] : 0u;
    const uint2 d0 = nseq ? a.desc[(size_t)c * a.seq_max] : make_uint2(0u, 0u);
    // one event or one list over all events: the rank within the event is the
    // global rank (no per-event bases)
    const bool global_rank = o.compact || w.n_events == 1;
    if (lane == 0)
        s_tot[warp] = mine;
    const bool any = __syncthreads_or(mine != 0);   // a CTA whose lists hold no peaks writes nothing

    // rank of the CTA's first list: the totals of the lists before it
    uint32_t part = 0;
    if (any)
        for (uint32_t q0 = 0; q0 < c0; q0 += 4 * bd) {   // four loads per thread in flight
            uint32_t v[4];
#pragma unroll
            for (uint32_t k = 0; k < 4; ++k) {
                const uint32_t q = q0 + k * bd + tid;
                v[k] = q < c0 ? a.cta_total[q] : 0u;
            }
            part += (v[0] + v[1]) + (v[2] + v[3]);
        }
    part = warp_incl_scan(part);
    if (lane == 31u)
        red[warp] = part;
    if (any && !global_rank)
        for (uint32_t e = tid; e < w.n_events; e += bd)
            ev_base[e] = o.ev_count[e];
    __syncthreads();
    uint32_t P = 0;
    for (uint32_t q = 0; q < nw; ++q)
        P += red[q];
    for (uint32_t q = 0; q < warp; ++q)   // the CTA's lists before this warp's
        P += s_tot[q];
    __syncthreads();
    if (any && !global_rank)
        block_exclusive_scan(ev_base, w.n_events, red);

    for (uint32_t q = 0; q < (mine ? nseq : 0u); ++q) {
        const uint2 d = q == 0 ? d0 : a.desc[(size_t)c * a.seq_max + q];
        for (uint32_t k = lane; k < d.y; k += 32u) {
            if (d.x + k >= a.entries_cap)
                break;
            const uint4 en = a.entries[d.x + k];
            const uint32_t e = en.y;
            const uint32_t pos = global_rank ? P + k : P + k - ev_base[e];
            if (pos < o.capacity)
                o.out[o.compact ? (size_t)pos : (size_t)e * o.capacity + pos] = peak_record(g, en);
        }
        P += d.y;
    }
    if (global_rank) {
        // no other CTA reads the per-event counts: the first one publishes and
        // resets them (and the entry counter), and no CTA waits for the others
        if (blockIdx.x == 0) {
            for (uint32_t e = tid; e < w.n_events; e += bd) {
                o.counts[e] = o.ev_count[e];
                o.ev_count[e] = 0u;
            }
            if (tid == 0)
                *o.g_count = 0u;
        }
        return;
    }
    if (blockIdx.x == 0)
        for (uint32_t e = tid; e < w.n_events; e += bd)
            o.counts[e] = o.ev_count[e];

    // Every CTA read the per-event counts: the last CTA to finish resets the
    // counters for the next scan.
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(o.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        for (uint32_t e = tid; e < w.n_events; e += bd)
            o.ev_count[e] = 0u;
        if (tid == 0) {
            *o.g_count = 0u;
            *o.ticket = 0u;
        }
    }
}

} // namespace htk

// ---------------------------------------------------------------------------
// Launchers (host).
// ---------------------------------------------------------------------------
namespace htk {

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) only when a launch needs
// more than was already allowed for the kernel on this device: the attribute
// call is a driver round trip that would otherwise cost every launch.
static cudaError_t allow_smem(const void *kernel, size_t bytes)
{
    constexpr int kSlots = 16, kDevs = 64;
    static std::atomic<const void *> keys[kSlots];
    static std::atomic<int> allowed[kSlots][kDevs];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    int slot = -1;
    for (int i = 0; i < kSlots && slot < 0; ++i) {
        const void *k = keys[i].load(std::memory_order_acquire);
        if (k == kernel)
            slot = i;
        else if (!k) {
            const void *expect = nullptr;
            if (keys[i].compare_exchange_strong(expect, kernel) || expect == kernel)
                slot = i;
        }
    }
    if (slot < 0)
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    std::atomic<int> &a = allowed[slot][dev];
    if ((int)bytes <= a.load(std::memory_order_acquire))
        return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) {
        int cur = a.load();
        while ((int)bytes > cur && !a.compare_exchange_weak(cur, (int)bytes)) {
        }
    }
    return e;
}

// Launch with programmatic stream serialisation allowed (see grid_dep_wait).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), uint32_t grid, uint32_t block, size_t smem,
                              cudaStream_t st, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

cudaError_t launch_bin(const Geom &g, const Work &w, uint32_t grid, cudaStream_t st)
{
    const size_t smem = w.hit_off ? ((size_t)w.n_events + 1) * 4 : 0;
    if (smem > 32 * 1024) {
        cudaError_t e = allow_smem((const void *)k_bin, smem);
        if (e != cudaSuccess)
            return e;
    }
    return launch_pdl(k_bin, grid, 256, smem, st, g, w);
}

cudaError_t launch_scatter(const Geom &g, const Work &w, uint32_t grid, cudaStream_t st)
{
    return launch_pdl(k_scatter, grid, 256, 0, st, g, w);
}

size_t bin_cluster_smem_bytes(const Geom &g, uint32_t n_events)
{
    return ((size_t)3 * n_events * g.n_slices + 1 + n_events + 1) * 4;
}

bool bin_cluster_supported(size_t smem)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kBinClusterMax);
    cfg.blockDim = dim3(kBinClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kBinClusterMax;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (allow_smem((const void *)k_bin_cluster, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveClusters(&n, (const void *)k_bin_cluster, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

cudaError_t launch_bin_cluster(const Geom &g, const Work &w, uint32_t cs, cudaStream_t st)
{
    const size_t smem = bin_cluster_smem_bytes(g, w.n_events);   // <= kBinClusterSmem, allowed by bin_cluster_supported
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kBinClusterThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k_bin_cluster, g, w);
}

size_t fill_scan_smem_bytes(const FillCfg &c, const ScanArgs &a, uint32_t nb)
{
    return 16 * sizeof(uint4) + (size_t)a.K * sizeof(uint4) + (size_t)c.tile_words * 4 +
           (size_t)staging_words(c, nb) * 4 + (size_t)c.HC * 16 + (size_t)c.beta_words * 4 +
           (size_t)4 * kFusedCand * 4;
}

cudaError_t launch_fill_scan(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                             cudaStream_t st)
{
    const size_t smem = fill_scan_smem_bytes(c, a, g.nb);
    const void *k = c.bulk ? (const void *)k_fill_bulk : (const void *)k_fill_scan;
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    return c.bulk ? launch_pdl(k_fill_bulk, grid, c.threads, smem, st, g, w, c, a)
                  : launch_pdl(k_fill_scan, grid, c.threads, smem, st, g, w, c, a);
}

size_t fill_ws_smem_bytes(const FillCfg &c, const ScanArgs &a)
{
    return 16 * sizeof(uint4) + (size_t)a.K * sizeof(uint4) + (size_t)2 * c.tile_words * 4 + (size_t)c.HC * 16 +
           (size_t)c.beta_words * 4 + (size_t)4 * kFusedCand * 4 + 4 * sizeof(uint64_t);
}

cudaError_t launch_fill_ws(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                           cudaStream_t st)
{
    const size_t smem = fill_ws_smem_bytes(c, a);
    cudaError_t e = allow_smem((const void *)k_fill_ws, smem);
    if (e != cudaSuccess)
        return e;
    return launch_pdl(k_fill_ws, grid, kWsThreads, smem, st, g, w, c, a);
}

cudaError_t fill_ws_occupancy(const FillCfg &c, const ScanArgs &a, int *blocks_per_sm)
{
    const size_t smem = fill_ws_smem_bytes(c, a);
    cudaError_t e = allow_smem((const void *)k_fill_ws, smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_fill_ws, kWsThreads, smem);
}

cudaError_t launch_peaks(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                         bool peaks_only, cudaStream_t st)
{
    return launch_pdl(k_peaks, grid, 256, 0, st, g, w, c, a, peaks_only ? 1u : 0u);
}

cudaError_t launch_fill_peaks(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                              cudaStream_t st)
{
    const size_t smem = fill_scan_smem_bytes(c, a, g.nb);
    cudaError_t e = allow_smem((const void *)k_fill_peaks, smem);
    if (e != cudaSuccess)
        return e;
    return launch_pdl(k_fill_peaks, grid, c.threads, smem, st, g, w, c, a);
}

size_t fill_tma_smem_bytes(const FillCfg &c, const ScanArgs &a)
{
    return 16 * sizeof(uint4) + (size_t)a.K * sizeof(uint4) + (size_t)2 * c.tile_words * 4 +
           (size_t)c.HC * 16 + (size_t)c.beta_words * 4 + (size_t)4 * kFusedCand * 4;
}

cudaError_t launch_fill_tma(const Geom &g, const Work &w, const FillCfg &c, const ScanArgs &a, uint32_t grid,
                            cudaStream_t st)
{
    const size_t smem = fill_tma_smem_bytes(c, a);
    const void *k = c.vote_agg ? (const void *)k_fill_tma<true> : (const void *)k_fill_tma<false>;
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    return c.vote_agg ? launch_pdl(k_fill_tma<true>, grid, c.threads, smem, st, g, w, c, a)
                      : launch_pdl(k_fill_tma<false>, grid, c.threads, smem, st, g, w, c, a);
}

cudaError_t fill_tma_occupancy(const FillCfg &c, const ScanArgs &a, int *blocks_per_sm)
{
    const size_t smem = fill_tma_smem_bytes(c, a);
    const void *k = c.vote_agg ? (const void *)k_fill_tma<true> : (const void *)k_fill_tma<false>;
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, c.threads, smem);
}

cudaError_t fill_scan_occupancy(const FillCfg &c, const ScanArgs &a, uint32_t nb, int *blocks_per_sm)
{
    const size_t smem = fill_scan_smem_bytes(c, a, nb);
    const void *k = c.bulk ? (const void *)k_fill_bulk : (const void *)k_fill_scan;
    cudaError_t e = allow_smem(k, smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, c.threads, smem);
}

size_t fill_smem_bytes(const FillCfg &c)
{
    return (size_t)c.tile_words * 4 + (size_t)c.HC * 16 + (size_t)c.beta_words * 4;
}

cudaError_t launch_fill_priv(const Geom &g, const Work &w, const FillCfg &c, uint32_t grid,
                             cudaStream_t st)
{
    const size_t smem = fill_smem_bytes(c);
    cudaError_t e = allow_smem((const void *)k_fill_priv, smem);
    if (e != cudaSuccess)
        return e;
    return launch_pdl(k_fill_priv, grid, c.threads, smem, st, g, w, c);
}

cudaError_t launch_clear(uint32_t *M, uint64_t words, uint32_t grid, cudaStream_t st)
{
    return launch_pdl(k_clear, grid, 512, 0, st, M, words);
}

cudaError_t launch_fill_naive(const Geom &g, const Work &w, uint32_t num_sms, cudaStream_t st)
{
    // a block over A; as many blocks as are resident at once (2048 threads per SM)
    const uint32_t threads = g.na >= 1024 ? 1024 : ((g.na + 31) / 32) * 32;
    const size_t smem = ((size_t)g.nb + 1) * 4 <= 48u * 1024u ? ((size_t)g.nb + 1) * 4 : 0;
    return launch_pdl(k_fill_naive, num_sms * (2048 / threads), threads, smem, st, g, w);
}

size_t scan_smem_bytes(const ScanArgs &a)
{
    return 16 * sizeof(uint4) + (size_t)a.K * sizeof(uint4) + (size_t)a.S * a.slot_words * 4 +
           (size_t)a.hot_words * 4 + (a.hot_words ? (size_t)kCand * 4 : 0);
}

static const void *scan_kernel(int kind)
{
    switch (kind) {
    case SCAN_BULK:
        return (const void *)k_scan_tma;
    case SCAN_LDG:
        return (const void *)k_scan_ldg;
    default:
        return (const void *)k_scan_direct;
    }
}

cudaError_t launch_scan(const Geom &g, const Work &w, const ScanArgs &a, int kind, cudaStream_t st)
{
    const size_t smem = scan_smem_bytes(a);
    cudaError_t e = allow_smem((const void *)scan_kernel(kind), smem);
    if (e != cudaSuccess)
        return e;
    if (kind == SCAN_BULK)
        return launch_pdl(k_scan_tma, a.grid, 256, smem, st, g, w, a);
    if (kind == SCAN_LDG)
        return launch_pdl(k_scan_ldg, a.grid, 256, smem, st, g, w, a);
    return launch_pdl(k_scan_direct, a.grid, 256, smem, st, g, w, a);
}



// ---------------------------------------------------------------------------
// k_wait_probe: the failure path of the bounded waits, on demand.  One
// thread waits on a shared-memory mbarrier that nothing arrives at, giving
// up after limit_ns (at most kWaitNs) or kWaitIters polls, and flags
// ST_WAIT_TIMEOUT exactly as a real wait that gave up does.
// ---------------------------------------------------------------------------
__global__ void k_wait_probe(uint32_t *status, uint64_t limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0)
        return;
    mbar_init(&bar, 1u);   // one arrival expected, none will come
    fence_mbar_init();
    const uint64_t t0 = global_ns();
    bool done = false;
    for (uint32_t it = 0; it < kWaitIters && !done; ++it) {
        done = mbar_try_wait(&bar, 0u);
        if ((it & 255u) == 255u && global_ns() - t0 > limit_ns)
            break;
    }
    if (!done)
        atomicOr(status, (uint32_t)ST_WAIT_TIMEOUT);
}

cudaError_t launch_wait_probe(uint32_t *status, uint32_t limit_ms, cudaStream_t st)
{
    const uint64_t ns = (uint64_t)limit_ms * 1000000ull;
    k_wait_probe<<<1, 32, 0, st>>>(status, ns < kWaitNs ? ns : kWaitNs);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// k_peaks4d: the 4-D (80-neighbour) maxima rule as a filter of the 2-D list.
//
// A cell's 8 neighbours in its own (A, B) slice are among its 80 neighbours
// in (theta, phi, A, B), so every 4-D peak is a 2-D peak: the filter takes
// the 2-D peaks (ascending linear index) and keeps those that also beat the
// up to 72 cells of the adjacent slices -- strictly the ones in an earlier
// slice (smaller linear index), with >= the ones in a later slice; phi does
// not wrap.  One warp per peak: its lanes read the 72 cells at once (three
// rounds of 32) and a warp vote decides; the keep flags go to `keep`, and
// the last CTA to finish (ticket) compacts the kept peaks in order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_peaks4d(Geom g, const uint32_t *M, const Peak *in, const uint32_t *n_in,
                                                 uint32_t cap_in, uint8_t *keep, Peak *out, uint32_t cap_out,
                                                 uint32_t *n_out, uint32_t *ticket, uint32_t *status)
{
    __shared__ uint32_t s_warp[32], s_total, s_last;
    grid_dep_wait();   // the 2-D list of k_order
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5, nw = blockDim.x >> 5;
    const uint32_t n_all = __ldcg(n_in);
    const uint32_t n = min(n_all, cap_in);
    const int nt = (int)g.nt, np = (int)g.np, na = (int)g.na, nb = (int)g.nb;
    for (uint32_t q = blockIdx.x * nw + wid; q < n; q += gridDim.x * nw) {
        const Peak p = in[q];
        const int t = (int)p.itheta, f = (int)p.iphi, i = (int)p.ia, j = (int)p.ib;
        bool ok = true;
#pragma unroll
        for (uint32_t round = 0; round < 3; ++round) {
            const uint32_t k = lane + 32u * round;   // neighbour k: slice k / 9, cell k % 9
            if (k < 72u) {
                const uint32_t sl = k / 9u, cell = k - sl * 9u;
                const uint32_t ts = sl < 4u ? sl : sl + 1u;   // the 3 x 3 (theta, phi) offsets but (0, 0)
                const int dt = (int)(ts / 3u) - 1, df = (int)(ts % 3u) - 1;
                const int tt = t + dt, ff = f + df, ii = i + (int)(cell / 3u) - 1, jj = j + (int)(cell % 3u) - 1;
                if (tt >= 0 && tt < nt && ff >= 0 && ff < np && ii >= 0 && ii < na && jj >= 0 && jj < nb) {
                    const uint32_t w = M[(((size_t)tt * np + ff) * na + ii) * (size_t)nb + jj];
                    const bool before = dt < 0 || (dt == 0 && df < 0);
                    ok = ok && (before ? p.votes > w : p.votes >= w);
                }
            }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (lane == 0)
            keep[q] = ok ? 1u : 0u;
    }
    // the last CTA to finish compacts the kept peaks in order
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    if (n_all > cap_in && tid == 0)
        atomicOr(status, (uint32_t)ST_SCRATCH_OVERFLOW);   // the 2-D list was cut: the filter would miss peaks
    uint32_t base = 0;
    for (uint32_t r0 = 0; r0 < n; r0 += blockDim.x) {
        const uint32_t q = r0 + tid;
        const bool kq = q < n && __ldcg(&keep[q]) != 0u;
        const uint32_t bal = __ballot_sync(0xffffffffu, kq);
        if (lane == 0)
            s_warp[wid] = __popc(bal);
        __syncthreads();
        if (wid == 0) {
            const uint32_t c = lane < nw ? s_warp[lane] : 0u;
            const uint32_t incl = warp_incl_scan(c);
            if (lane < nw)
                s_warp[lane] = incl - c;   // exclusive prefix of the warp totals
            if (lane == 31)
                s_total = incl;
        }
        __syncthreads();
        const uint32_t pos = base + s_warp[wid] + __popc(bal & ((1u << lane) - 1u));
        if (kq && pos < cap_out)
            out[pos] = in[q];
        base += s_total;
        __syncthreads();   // s_warp, s_total free for the next round
    }
    if (tid == 0) {
        *n_out = base;
        *ticket = 0u;
    }
}

cudaError_t launch_peaks4d(const Geom &g, const uint32_t *M, const Peak *in, const uint32_t *n_in, uint32_t cap_in,
                           uint8_t *keep, Peak *out, uint32_t cap_out, uint32_t *n_out, uint32_t *ticket,
                           uint32_t *status, uint32_t grid, cudaStream_t st)
{
    return launch_pdl(k_peaks4d, grid, 256u, (size_t)0, st, g, M, in, n_in, cap_in, keep, out, cap_out, n_out,
                      ticket, status);
}

// ---------------------------------------------------------------------------
// k_atomic_rate: the L2-atomic roofline the naive fill is measured against.
// Every thread adds 1 to per_thread words of buf picked by a linear
// congruential sequence of its own (masked to the footprint, a power of two
// words); the results are unused, so the adds are reductions performed in L2.
// ---------------------------------------------------------------------------
__global__ void k_atomic_rate(uint32_t *buf, uint32_t mask, uint32_t per_thread, uint32_t seed)
{
    uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u ^ seed;
    for (uint32_t i = 0; i < per_thread; ++i) {
        x = x * 1664525u + 1013904223u;
        atomicAdd(&buf[(x >> 4) & mask], 1u);
    }
}

cudaError_t launch_atomic_rate(uint32_t *buf, uint32_t mask, uint32_t per_thread, uint32_t seed, uint32_t grid,
                               cudaStream_t st)
{
    k_atomic_rate<<<grid, 256, 0, st>>>(buf, mask, per_thread, seed);
    return cudaGetLastError();
}

cudaError_t launch_order(const Geom &g, const Work &w, const ScanArgs &a, const OrderArgs &o,
                         cudaStream_t st)
{
    const size_t smem = (w.n_events + 1 + 40) * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = allow_smem((const void *)k_order, smem);
        if (e != cudaSuccess)
            return e;
    }
    // one list per warp, eight per CTA
    return launch_pdl(k_order, (a.grid + 7) / 8, 256, smem, st, g, w, a, o);
}

cudaError_t scan_occupancy(int kind, size_t smem, int *blocks_per_sm)
{
    const void *k = scan_kernel(kind);
    cudaError_t e = allow_smem((const void *)k, smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, 256, smem);
}

cudaError_t fill_occupancy(const FillCfg &c, int *blocks_per_sm)
{
    const size_t smem = fill_smem_bytes(c);
    cudaError_t e = allow_smem((const void *)k_fill_priv, smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_fill_priv, c.threads, smem);
}

} // namespace htk
