// Device-side definitions shared by the Hough-Transform kernels.
//
// Every floating-point operation on the vote path uses an explicit
// round-to-nearest intrinsic (__fadd_rn, __fsub_rn, __fmul_rn, __fdiv_rn,
// __fsqrt_rn): these are never contracted into FMA, so the FP32 result of each
// step is the IEEE-754 binary32 result the C ABI documents.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace htk {

// Status word bits (device -> host).
enum : uint32_t {
    ST_WAIT_TIMEOUT = 1u,      // a bounded mbarrier wait gave up
    ST_SCRATCH_OVERFLOW = 2u,  // peak scratch or descriptor table too small
    ST_BAD_ARG = 4u            // a kernel saw an impossible size
};

// Per-binning constants (by value in every launch).
struct Geom {
    uint32_t nt, np, na, nb, wt, wp;
    uint32_t n_slices;      // nt * np
    uint32_t phi_full;      // phi range is the full circle: wrap the window
    uint32_t max_admit;     // slices one hit can enter
    uint32_t threshold;
    float a_min, b_min, da, db, nbf;
    float inv_db;           // 1 / dB, only to estimate a bin before the exact table test
    const float *et;        // device: nt + 1 theta pseudo-angle edges
    const float *ep;        // device: np + 1 phi pseudo-angle edges
    const float *bth;       // device: nb + 1 B-bin thresholds (see bin_from_thresholds)
};

// Device buffers of one batch of events (a single-event context is a batch
// of one).  Event e owns M[e * n_cells ...] and the hits [hit_off[e],
// hit_off[e + 1]) of the concatenated arrays.
struct Work {
    const float *x, *y, *z;     // concatenated hits
    const uint32_t *hit_off;    // [n_events + 1] or nullptr: one event, n_hits0 hits
    uint32_t n_hits0;           // with hit_off: the bound every offset is clamped to (staging size)
    uint32_t n_events;
    float4 *hits4;              // per hit: {x, x^2 + y^2, 2y, event (bits)}
    uint32_t *codes;            // per hit: (itheta << 16) | iphi, or kDropped
    uint32_t *M;                // vote matrices
    uint64_t n_cells;           // per event
    uint32_t *status;
    uint32_t *ctr;              // counter block (htk::CTR_*)
    // hits grouped by (event, slice) unit u = e * n_slices + s
    uint32_t *slice_cnt;        // [n_events * n_slices] hits per unit (k_bin counts, k_scatter clears)
    uint32_t *slice_fill;       // [n_events * n_slices] scatter cursors (k_bin's last block clears)
    uint32_t *slice_off;        // [n_events * n_slices + 1] exclusive prefix of slice_cnt
    float4 *list;               // list_cap hit records {x, x^2 + y^2, 2y, event}, unit by unit
    uint32_t list_cap;
    // peaks-only fills: the first and last row of every strip pass,
    // [unit][edge_pass][2][n_b] (pass p of a unit covers rows p * rpass ..)
    uint32_t *edge;
    uint32_t edge_pass;
    // Where a fill's static split (the static items of every CTA) comes from:
    // kSplitAfterWait: computed after the fill's dependency wait;
    // kSplitEarly: computed before it (k_scatter let the fill launch only
    //   after its own wait for k_bin, so the unit offsets are complete);
    // kSplitGiven: read from split[] after the wait, where k_bin_cluster put
    //   it for a fill of split_grid CTAs, split_strips strips per unit, vote
    //   weight split_vw and split_n_static static items (a fill of another
    //   shape computes its own).
    uint32_t split_mode;
    uint32_t split_grid, split_strips, split_vw;
    uint64_t split_n_static;
    uint64_t *split;            // [split_grid + 1] first static item of every fill CTA
};

constexpr uint32_t kSplitAfterWait = 0, kSplitEarly = 1, kSplitGiven = 2;

constexpr uint32_t kDropped = 0xffffffffu;


// One peak as the scan emits it: {lin within event, event, votes, 0}.
// Output record (matches ht_peak of the C ABI, 32 bytes).
struct Peak {
    uint32_t itheta, iphi, ia, ib, votes;
    float a_c, b_c;
    uint32_t event;
};

// Hit range of event e, clamped to [0, n_hits0] so that offsets written by
// a caller on the device can never send a kernel outside the staging.
__device__ __forceinline__ uint32_t ev_hit_begin(const Work &w, uint32_t e)
{
    return w.hit_off ? min(w.hit_off[e], w.n_hits0) : 0u;
}
__device__ __forceinline__ uint32_t ev_hit_end(const Work &w, uint32_t e)
{
    return w.hit_off ? max(min(w.hit_off[e + 1], w.n_hits0), ev_hit_begin(w, e)) : w.n_hits0;
}

// ---------------------------------------------------------------------------
// Pseudo-angles.  Polar: rho/(z+rho) for z >= 0, else 1 + (-z)/(rho-z); 0 on
// +z, 1 in the transverse plane, 2 on -z.  Azimuthal: the quadrant "diamond
// angle" of (u, v) = (-x, -y), 0 at phi = -pi rising to 4 at phi = +pi.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float theta_pseudo(float rho, float z)
{
    if (z >= 0.0f)
        return __fdiv_rn(rho, __fadd_rn(z, rho));
    return __fadd_rn(1.0f, __fdiv_rn(-z, __fsub_rn(rho, z)));
}

__device__ __forceinline__ float phi_pseudo(float x, float y)
{
    const float u = -x, v = -y;
    if (v >= 0.0f) {
        if (u >= 0.0f)
            return __fdiv_rn(v, __fadd_rn(u, v));
        return __fadd_rn(1.0f, __fdiv_rn(-u, __fadd_rn(-u, v)));
    }
    if (u < 0.0f)
        return __fadd_rn(2.0f, __fdiv_rn(-v, __fadd_rn(-u, -v)));
    return __fadd_rn(3.0f, __fdiv_rn(u, __fadd_rn(u, -v)));
}

// Number of edges e[1..n-1] that are <= D (edges non-decreasing): the bin.
__device__ __forceinline__ uint32_t edge_bin(float D, const float *e, uint32_t n)
{
    uint32_t lo = 1, hi = n;            // search in [1, n)
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (D >= e[mid])
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo - 1;
}

// Bin code of one hit: (itheta << 16) | iphi of its own slice, or kDropped
// (rho == 0, NaN, or outside the angle ranges).  Also returns r2 = x^2 + y^2.
__device__ __forceinline__ uint32_t bin_code(const Geom &g, const float *et, const float *ep, float x,
                                             float y, float z, float &r2)
{
    r2 = __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y));
    const float rho = __fsqrt_rn(r2);
    if (!(rho > 0.0f))
        return kDropped;
    const float dt = theta_pseudo(rho, z);
    const float dp = phi_pseudo(x, y);
    if (!(dt >= et[0] && dt <= et[g.nt]))
        return kDropped;
    if (!(dp >= ep[0] && dp <= ep[g.np]))
        return kDropped;
    return (edge_bin(dt, et, g.nt) << 16) | edge_bin(dp, ep, g.np);
}

// Is slice (ts, ps) among the slices a hit of bin code `code` votes in: its
// own bin, +-win_theta (clipped), +-win_phi (cyclic on the full circle,
// clipped otherwise), each slice at most once.
__device__ __forceinline__ bool admits(const Geom &g, uint32_t code, uint32_t ts, uint32_t ps)
{
    if (code == kDropped)
        return false;
    const uint32_t it = code >> 16, ip = code & 0xffffu;
    const uint32_t dt = ts > it ? ts - it : it - ts;
    if (dt > g.wt)
        return false;
    uint32_t dp = ps > ip ? ps - ip : ip - ps;
    if (g.phi_full && g.np - dp < dp)
        dp = g.np - dp;
    return dp <= g.wp;
}

// Visit every slice id (itheta * n_phi + iphi) a hit of bin code `code` votes in.
template <class F>
__device__ __forceinline__ void for_each_slice(const Geom &g, uint32_t code, F &&f)
{
    if (code == kDropped)
        return;
    const uint32_t it = code >> 16, ip = code & 0xffffu;
    const uint32_t t0 = it > g.wt ? it - g.wt : 0u, t1 = min(it + g.wt, g.nt - 1);
    for (uint32_t t = t0; t <= t1; ++t) {
        if (g.phi_full && 2 * g.wp + 1 >= g.np) {
            for (uint32_t p = 0; p < g.np; ++p)
                f(t * g.np + p);
        } else if (g.phi_full) {
            for (int32_t d = -(int32_t)g.wp; d <= (int32_t)g.wp; ++d) {
                int32_t p = (int32_t)ip + d;
                if (p < 0)
                    p += (int32_t)g.np;
                else if (p >= (int32_t)g.np)
                    p -= (int32_t)g.np;
                f(t * g.np + (uint32_t)p);
            }
        } else {
            const uint32_t p0 = ip > g.wp ? ip - g.wp : 0u, p1 = min(ip + g.wp, g.np - 1);
            for (uint32_t p = p0; p <= p1; ++p)
                f(t * g.np + p);
        }
    }
}

// A bin centre A_i = a_min + ((float)i + 0.5) * dA.
__device__ __forceinline__ float a_centre(const Geom &g, uint32_t i)
{
    return __fadd_rn(g.a_min, __fmul_rn(__fadd_rn(__uint2float_rn(i), 0.5f), g.da));
}
__device__ __forceinline__ float b_centre(const Geom &g, uint32_t j)
{
    return __fadd_rn(g.b_min, __fmul_rn(__fadd_rn(__uint2float_rn(j), 0.5f), g.db));
}

// The vote of one (hit, A bin): returns the B bin, or -1 if out of range.
//   B = (r2 - (2 A) x) / d,  t = (B - b_min) / dB,  bin = floor(t) if 0 <= t < N_B.
__device__ __forceinline__ int vote_bin(const Geom &g, float twoA, float x, float r2, float d)
{
    const float num = __fsub_rn(r2, __fmul_rn(twoA, x));
    const float B = __fdiv_rn(num, d);
    const float t = __fdiv_rn(__fsub_rn(B, g.b_min), g.db);
    if (t >= 0.0f && t < g.nbf)
        return (int)__float2uint_rz(t);
    return -1;
}

// The B bin of the vote from the threshold table beta[0 .. nb]: beta[k] is
// the smallest float B whose bin floor(fl(fl(B - b_min) / dB)) is >= k, so
// the bin is max{k : beta[k] <= B} and the vote is in range iff
// beta[0] <= B < beta[nb] (NaN fails).  Identical to the division rule for
// every float B; an estimate from 1/dB is corrected by table compares.
__device__ __forceinline__ int bin_from_thresholds(const Geom &g, const float *beta, float b_lo, float b_hi, float B)
{
    if (!(B >= b_lo && B < b_hi))   // b_lo = beta[0], b_hi = beta[n_b]
        return -1;
    int j = (int)((B - g.b_min) * g.inv_db);
    j = max(0, min(j, (int)g.nb - 1));
    while (B < beta[j])
        --j;
    while (B >= beta[j + 1])
        ++j;
    return j;
}

// The vote of one (hit, A bin) with the threshold table: B = (r2 - (2A) x) / d
// by IEEE division, then its bin (or -1).
__device__ __forceinline__ int vote_bin_tab(const Geom &g, const float *beta, float b_lo, float b_hi, float twoA,
                                            float x, float r2, float d)
{
    const float num = __fsub_rn(r2, __fmul_rn(twoA, x));
    const float B = __fdiv_rn(num, d);
    return bin_from_thresholds(g, beta, b_lo, b_hi, B);
}

// ---------------------------------------------------------------------------
// mbarrier + bulk-copy (TMA, non-tensor) wrappers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> this CTA's shared memory, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 1-D bulk copy this CTA's shared memory -> global, in the issuing thread's
// current bulk async-group.  dst, src 16-byte aligned; bytes a multiple of
// 16.  The source must have been written before a fence.proxy.async by the
// writing threads and a barrier.
__device__ __forceinline__ void bulk_store(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

// bulk_store with an L2 evict-first policy: the written lines are the first
// to leave L2 (the destination is written once and read back only in part).
__device__ __forceinline__ void bulk_store_evict_first(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("{\n\t.reg .b64 pol;\n\t"
                 "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
                 "cp.async.bulk.global.shared::cta.bulk_group.L2::cache_hint [%0], [%1], %2, pol;\n\t}" ::"l"(dst),
                 "r"(smem_addr(src)), "r"(bytes)
                 : "memory");
}

// Close the issuing thread's current bulk async-group.
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until at most N of the issuing thread's bulk async-groups are still
// reading their shared-memory sources (the writes may still be in flight).
template <int N>
__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

// Wait until at most N of the issuing thread's bulk async-groups are
// incomplete (their writes performed).
template <int N>
__device__ __forceinline__ void bulk_wait()
{
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// One arrival (release semantics, CTA scope) on a barrier initialised with
// the number of arriving threads.
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: gives up after kWaitIters polls or about one second.
constexpr uint32_t kWaitIters = 1u << 24;
constexpr uint64_t kWaitNs = 1000000000ull;

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it < kWaitIters; ++it) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((it & 255u) == 0 && global_ns() - t0 > kWaitNs)
            return false;
    }
    return false;
}

} // namespace htk
