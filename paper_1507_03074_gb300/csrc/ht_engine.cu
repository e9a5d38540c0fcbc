// Engine: resident workspace and launch shapes for the two steps.
#include "ht_engine.h"
#include "ht_geom.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

namespace hte {

static uint32_t round_up(uint32_t v, uint32_t m) { return (v + m - 1) / m * m; }

static const size_t kSmemMax = 227 * 1024;     // per CTA on sm_100-class parts
static const uint32_t kScanThreads = 256;
static const uint32_t kPeakBuf = 1024;         // K: entries buffered per scan / seam CTA
static const uint32_t kFusedPeakBuf = 512;     // K of a fused-fill CTA (at least its block)

const char *const kKernelNames[K_NKINDS] = {"k_bin", "k_scatter", "k_fill_priv", "k_fill_scan", "k_fill_ws",
                                             "k_fill_peaks", "k_peaks", "k_clear", "k_fill_naive", "k_scan",
                                             "k_order", "k_peaks4d", "k_fill_tma", "k_bin_cluster"};

// ---------------------------------------------------------------------------
// Profiling
// ---------------------------------------------------------------------------
static cudaEvent_t prof_event(Engine &E)
{
    if (!E.prof.pool.empty()) {
        cudaEvent_t ev = E.prof.pool.back();
        E.prof.pool.pop_back();
        return ev;
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreate(&ev) != cudaSuccess)
        return nullptr;
    return ev;
}

cudaError_t prof_collect(Engine &E)
{
    Prof &P = E.prof;
    if (P.pending.empty())
        return cudaSuccess;
    cudaError_t e = cudaEventSynchronize(P.pending.back().b);
    if (e != cudaSuccess)
        return e;
    for (auto &r : P.pending) {
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, r.a, r.b)) != cudaSuccess)
            return e;
        P.ms[r.kind] += ms;
        P.n[r.kind] += 1;
        P.pool.push_back(r.a);
        P.pool.push_back(r.b);
    }
    P.pending.clear();
    return cudaSuccess;
}

cudaError_t prof_enable(Engine &E, bool on)
{
    cudaError_t e = prof_collect(E);
    E.prof.on = on;
    if (on)
        for (int k = 0; k < K_NKINDS; ++k) {
            E.prof.ms[k] = 0.0;
            E.prof.n[k] = 0;
        }
    return e;
}

// Record around one launch when profiling is on.
struct ProfScope {
    Engine &E;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(Engine &E_, int k, cudaStream_t s) : E(E_), kind(k), st(s)
    {
        if (E.prof.on && (a = prof_event(E)))
            cudaEventRecord(a, st);
    }
    ~ProfScope()
    {
        if (!a)
            return;
        cudaEvent_t b = prof_event(E);
        if (!b)
            return;
        cudaEventRecord(b, st);
        E.prof.pending.push_back({kind, a, b});
        if (E.prof.pending.size() >= 4096)
            prof_collect(E);
    }
};

template <class T>
static cudaError_t dalloc(T **p, size_t bytes, size_t *acc)
{
    *acc += bytes;
    return cudaMalloc(reinterpret_cast<void **>(p), bytes ? bytes : 16);
}

// Chunk descriptors a CTA owning `rows` rows may need when a row yields at
// most per_row entries (peaks: ceil(n_b / 2), as no two peaks are
// neighbours; fused-fill candidates: n_b); every chunk but the last holds at
// least K - per_round entries.
static uint32_t chunks_for(uint64_t rows, uint32_t per_row, uint32_t K, uint32_t per_round)
{
    return (uint32_t)std::min<uint64_t>(rows * per_row / (K - per_round) + 2, 1u << 20);
}

ht_status engine_configure(Engine &E, std::string *why)
{
    const ht_binning &b = E.b;
    const Tuning &t = E.tune;
    const htk::Geom &g = E.geom;
    char buf[256];

    // --- privatised fill -------------------------------------------------
    htk::FillCfg f{};
    f.threads = t.fill_threads ? t.fill_threads : 512;
    if (f.threads != 256 && f.threads != 512 && f.threads != 1024) {
        *why = "fill_threads must be 256, 512 or 1024";
        return HT_E_INVAL;
    }
    if (t.vote_agg > 1) {
        *why = "fill_vote_agg must be 0 (plain shared-memory atomics) or 1 (warp-aggregated)";
        return HT_E_INVAL;
    }
    if (t.bin_cluster > 2) {
        *why = "bin_cluster must be 0 (auto), 1 (one cluster launch) or 2 (two launches)";
        return HT_E_INVAL;
    }
    if (t.fused > 5) {
        *why = "fused must be 0 (auto), 1 (on), 2 (off), 3 (warp-specialised), 4 (bulk-copy staging) or "
               "5 (bulk-copy tiles)";
        return HT_E_INVAL;
    }
    f.HC = std::max(t.fill_HC ? t.fill_HC : 2048u, 2 * f.threads);   // hits staged per chunk
    f.pitch16 = round_up((b.n_b + 1) / 2, 32);
    f.pitch32 = round_up(b.n_b, 32);
    f.beta_words = round_up(b.n_b + 1, 4);
    f.dyn = 1;   // the last items are handed out at run time (htk::dyn_items)
    f.vote_weight = htk::kVoteWeight;
    const size_t beta_bytes = (size_t)f.beta_words * 4;
    if (t.fill_W && (t.fill_W & (t.fill_W - 1))) {
        *why = "fill_rows must be a power of two";
        return HT_E_INVAL;
    }
    // with the bulk-copy-tile fill (asked for, or automatic where n_b allows
    // it) fill_rows sizes its tiles; the other fills (accumulating, peaks-only)
    // keep their own tile height
    bool tma_mode = (t.fused == 5 || t.fused == 0) && (b.n_b & 3u) == 0 && b.n_b <= 4096;
    if (tma_mode && t.fill_W) {
        // a requested tile height the bulk-copy-tile fill cannot hold leaves it to the others
        htk::FillCfg probe = f;
        probe.W = t.fill_W;
        probe.tile_words = t.fill_W * b.n_b;
        probe.HC = 2 * f.threads;
        htk::ScanArgs tmp{};
        tmp.K = std::max<uint32_t>(kFusedPeakBuf, f.threads);
        tma_mode = t.fill_W <= 64 && htk::fill_tma_smem_bytes(probe, tmp) <= kSmemMax;
    }
    uint32_t W = tma_mode ? 0u : t.fill_W;
    if (!W) {
        // aim at ~64 KB tiles so that two CTAs share an SM
        W = 32;
        while (W > 2 && (size_t)W * f.pitch16 * 4 > 64 * 1024)
            W >>= 1;
    }
    while (W > 2 && (size_t)W * f.pitch16 * 4 + (size_t)f.HC * 16 + beta_bytes > kSmemMax)
        W >>= 1;
    f.W = W;
    f.tile_words = W * f.pitch16;
    f.strips = (b.n_a + W - 1) / W;
    E.fill_priv_ok = (W >= 2) && (f.threads % W == 0) && htk::fill_smem_bytes(f) <= kSmemMax;
    E.fill = f;
    if (E.fill_priv_ok) {
        int occ = 0;
        cudaError_t e = htk::fill_occupancy(f, &occ);
        if (e != cudaSuccess || occ < 1) {
            std::snprintf(buf, sizeof buf, "fill occupancy query failed: %s", cudaGetErrorString(e));
            *why = buf;
            return HT_E_CUDA;
        }
        if (t.fill_blocks_per_sm)
            occ = std::min<int>(occ, (int)t.fill_blocks_per_sm);
        E.fill_grid = (uint32_t)E.num_sms * (uint32_t)occ;
    }
    E.clear_grid = (uint32_t)E.num_sms * 4;
    E.bin_cluster = htk::bin_cluster_supported(htk::kBinClusterSmem) ? 1 : 0;

    // --- fused fill + maxima ---------------------------------------------------
    // A smaller peak buffer than the scan's (the tile needs the room); k_seam
    // keeps kPeakBuf in its own launch.
    E.fused_ok = false;
    E.fused_capped = false;
    E.fused_K = std::max<uint32_t>(kFusedPeakBuf, f.threads);
    if (E.fill_priv_ok && t.fused != 2 && W <= 64 && b.n_b <= 4096) {
        htk::ScanArgs tmp{};
        tmp.K = E.fused_K;
        htk::FillCfg ff = f;
        const bool bulk = t.fused == 4;
        if (bulk) {
            // one CTA of 1024 threads per SM: the tile, two u32 staging
            // buffers of W / 2 rows and as many staged hits as still fit
            ff.bulk = 1;
            ff.threads = t.fill_threads ? t.fill_threads : 1024;
            ff.dyn = 1;
            E.fused_K = std::max<uint32_t>(kFusedPeakBuf, ff.threads);
            tmp.K = E.fused_K;
            if (t.fill_HC) {
                ff.HC = t.fill_HC;   // as asked (no two-blocks minimum here)
            } else {
                ff.HC = 2048;
                while (ff.HC > 256 && htk::fill_scan_smem_bytes(ff, tmp, b.n_b) > kSmemMax)
                    ff.HC -= 256;
            }
        }
        // two CTAs per SM if a staging size (a multiple of the block, at
        // least two blocks' worth) allows it, unless tuned explicitly
        int occ = 0;
        auto occupancy = [&](const htk::FillCfg &c) {
            int o = 0;
            if (htk::fill_scan_smem_bytes(c, tmp, b.n_b) > kSmemMax ||
                htk::fill_scan_occupancy(c, tmp, b.n_b, &o) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            return o;
        };
        occ = occupancy(ff);
        while (!bulk && !t.fill_HC && occ < 2 && ff.HC > 2 * ff.threads) {
            ff.HC -= ff.threads;
            occ = occupancy(ff);
        }
        if (bulk && ((b.n_b & 3u) || ff.threads % W || W < 2))
            occ = 0;   // rows must start on 16 bytes; the block must cover whole rows
        E.fused_fill = ff;
        if (occ >= 1) {
            E.fused_capped = t.fill_blocks_per_sm && (int)t.fill_blocks_per_sm < occ;
            if (t.fill_blocks_per_sm)
                occ = std::min<int>(occ, (int)t.fill_blocks_per_sm);
            E.fused_ok = true;
            E.fused_grid = (uint32_t)E.num_sms * (uint32_t)occ;
        }
    }
    // --- warp-specialised fused fill: two tiles, one CTA per SM -------------------
    E.ws_ok = false;
    if (E.fill_priv_ok && t.fused == 3 && W <= 64 && b.n_b <= 4096 &&
        (!t.fill_threads || t.fill_threads == htk::kWsThreads / 2)) {
        htk::ScanArgs tmp{};
        tmp.K = E.fused_K;
        htk::FillCfg wf = f;
        wf.dyn = 0;   // both thread groups walk the same static range
        wf.threads = htk::kWsThreads / 2;
        wf.HC = std::max(wf.HC, 2 * wf.threads);
        while (!t.fill_HC && wf.HC > 2 * wf.threads && htk::fill_ws_smem_bytes(wf, tmp) > kSmemMax)
            wf.HC -= wf.threads;
        int occ = 0;
        if (wf.threads % W == 0 && htk::fill_ws_smem_bytes(wf, tmp) <= kSmemMax &&
            htk::fill_ws_occupancy(wf, tmp, &occ) == cudaSuccess && occ >= 1) {
            E.ws_ok = true;
            E.ws_fill = wf;
            E.ws_grid = (uint32_t)E.num_sms * (uint32_t)occ;
        } else {
            cudaGetLastError();
        }
    }
    if (t.fused == 3 && !E.ws_ok) {
        *why = "the warp-specialised fused fill does not fit this binning and tuning";
        return HT_E_INVAL;
    }
    E.use_ws = E.ws_ok;
    // --- fused fill with bulk-copy tiles: two u32 tiles in M_H's layout ----------
    E.tma_ok = false;
    E.tma_capped = false;
    // the default fused fill wherever it fits (fused 0 = auto)
    if (E.fill_priv_ok && (t.fused == 5 || t.fused == 0) && (b.n_b & 3u) == 0 && b.n_b <= 4096) {
        htk::FillCfg tf = f;
        tf.threads = t.fill_threads ? t.fill_threads : 512;
        uint32_t Wt = t.fill_W;
        if (!Wt) {
            // two tiles of about 64 KB together
            Wt = 32;
            while (Wt > 1 && (size_t)2 * Wt * b.n_b * 4 > 64 * 1024)
                Wt >>= 1;
        }
        Wt = std::min<uint32_t>(Wt, 64);   // the hot-row mask holds 64 rows
        tf.W = Wt;
        tf.strips = (b.n_a + Wt - 1) / Wt;
        tf.tile_words = Wt * b.n_b;
        tf.vote_agg = t.vote_agg;
        tf.bulk = 0;
        tf.dyn = 1;
        tf.HC = std::max(t.fill_HC ? t.fill_HC : 2048u, 2 * tf.threads);
        htk::ScanArgs tmp{};
        tmp.K = std::max<uint32_t>(kFusedPeakBuf, tf.threads);
        auto occupancy = [&](const htk::FillCfg &c) {
            int o = 0;
            if (htk::fill_tma_smem_bytes(c, tmp) > kSmemMax || htk::fill_tma_occupancy(c, tmp, &o) != cudaSuccess) {
                cudaGetLastError();
                return 0;
            }
            return o;
        };
        int occ = occupancy(tf);
        while (!t.fill_HC && occ < 2 && tf.HC > 2 * tf.threads) {
            tf.HC -= tf.threads;
            occ = occupancy(tf);
        }
        E.tma_capped = false;
        if (occ >= 1) {
            E.tma_capped = t.fill_blocks_per_sm && (int)t.fill_blocks_per_sm < occ;
            if (t.fill_blocks_per_sm)
                occ = std::min<int>(occ, (int)t.fill_blocks_per_sm);
            E.tma_ok = true;
            E.tma_fill = tf;
            E.tma_K = tmp.K;
            E.tma_grid = (uint32_t)E.num_sms * (uint32_t)occ;
        }
    }
    if (t.fused == 5 && !E.tma_ok) {
        *why = "the bulk-copy-tile fused fill needs n_b a multiple of 4 (at most 4096) and tiles that fit";
        return HT_E_INVAL;
    }
    E.use_tma = E.tma_ok;
    if ((t.fused == 1 || t.fused == 4) && !E.fused_ok) {
        *why = "the fused fill does not fit this binning and tuning";
        return HT_E_INVAL;
    }

    // --- scan variant and shape --------------------------------------------
    htk::ScanArgs &s = E.scan;
    const size_t row_bytes = (size_t)b.n_b * 4;
    const size_t fixed = 16 * 16 + (size_t)kPeakBuf * 16;
    const bool vec = (b.n_b & 3u) == 0;
    s.K = kPeakBuf;
    int kind = !vec ? htk::SCAN_DIRECT
             : t.scan_kind == 1 ? htk::SCAN_BULK
             : t.scan_kind == 3 ? htk::SCAN_DIRECT : htk::SCAN_LDG;
    if (kind == htk::SCAN_BULK) {
        const size_t target = t.scan_stage_bytes ? t.scan_stage_bytes : (row_bytes >= 8192 ? 65536 : 32768);
        uint32_t rows = (uint32_t)std::max<size_t>(3, target / row_bytes);     // R + 2
        uint32_t S = t.scan_slots ? std::min<uint32_t>(std::max<uint32_t>(t.scan_slots, 2), 8) : 4;
        while (S > 2 && fixed + (size_t)S * rows * row_bytes > kSmemMax)
            --S;
        while (rows > 3 && fixed + (size_t)S * rows * row_bytes > kSmemMax)
            --rows;
        if (fixed + (size_t)S * rows * row_bytes <= kSmemMax && rows * row_bytes < (1u << 20)) {
            s.S = S;
            s.R = rows - 2;
            s.slot_words = rows * b.n_b;
        } else {
            kind = htk::SCAN_LDG;
        }
    }
    if (kind != htk::SCAN_BULK) {
        s.S = 0;
        s.slot_words = 0;
        // streaming: a chunk is kLdgUPT 16-byte units per thread
        s.R = kind == htk::SCAN_LDG ? std::max<uint32_t>(1, htk::kLdgUPT * kScanThreads / (b.n_b / 4)) : 16;
    }
    E.scan_kind = kind;
    const uint64_t G_max = (uint64_t)g.n_slices * g.na * E.max_events;
    {   // bitmap words for the streaming scan at one CTA per SM (the longest run)
        const uint64_t rows1 = (G_max + E.num_sms - 1) / E.num_sms + 1;
        s.hot_words = kind == htk::SCAN_LDG ? (uint32_t)((rows1 + s.R - 1) / s.R / 32 + 2) : 0;
    }
    int occ = 0;
    cudaError_t e = htk::scan_occupancy(kind, htk::scan_smem_bytes(s), &occ);
    if (e != cudaSuccess || occ < 1) {
        std::snprintf(buf, sizeof buf, "scan occupancy query failed: %s", cudaGetErrorString(e));
        *why = buf;
        return HT_E_CUDA;
    }
    if (t.scan_blocks_per_sm)
        occ = std::min<int>(occ, (int)t.scan_blocks_per_sm);
    E.scan_grid_max = (uint32_t)E.num_sms * (uint32_t)occ;

    // --- chunk bookkeeping for the largest launch (max_events events) ---------
    const uint32_t scan_grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(E.scan_grid_max, G_max));
    const uint64_t items_max = (uint64_t)E.max_events * g.n_slices * f.strips;
    const uint32_t fused_grid = E.fused_ok ? (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(E.fused_grid, items_max)) : 0;
    const uint32_t ws_grid = E.ws_ok ? (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(E.ws_grid, items_max)) : 0;
    const uint64_t items_tma = E.tma_ok ? (uint64_t)E.max_events * g.n_slices * E.tma_fill.strips : 0;
    const uint32_t tma_grid =
        E.tma_ok ? (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(E.tma_grid, items_tma)) : 0;
    // the fused fill's candidate lists: one per CTA plus one per handed-out item
    const uint32_t fused_lists = fused_grid + (uint32_t)htk::dyn_items(items_max, fused_grid);
    const uint32_t tma_lists = E.tma_ok ? tma_grid + (uint32_t)htk::dyn_items(items_tma, tma_grid) : 0;
    const uint32_t grid_cap = std::max(std::max(std::max(scan_grid, fused_lists), ws_grid), tma_lists);
    uint32_t seq = chunks_for((G_max + scan_grid - 1) / scan_grid + 1, (g.nb + 1) / 2, s.K, 2 * kScanThreads);
    // the cost-balanced split gives a CTA at most `spread` times the items of
    // an even split (every strip costs at least its n_b-per-row writing share)
    const double hits_per_unit = (double)std::max<uint32_t>(E.max_hits, 1) * E.max_admit /
                                 ((double)E.max_events * g.n_slices);
    const double spread = 1.0 + std::max(htk::kVoteWeight, htk::kPeaksVoteWeight) * hits_per_unit / g.nb;
    auto rows_per_cta = [&](uint32_t grid) {
        return (uint64_t)(std::ceil((double)items_max / grid * spread) + 2) * f.W + 1;
    };
    if (E.fused_ok) {
        const uint64_t fused_rows = rows_per_cta(fused_grid);
        seq = std::max(seq, chunks_for(fused_rows, g.nb, E.fused_K,
                                       htk::fused_round(E.fused_fill.threads, E.fused_K)));
    }
    if (E.tma_ok) {
        const uint64_t tma_rows = (uint64_t)(std::ceil((double)items_tma / tma_grid * spread) + 2) * E.tma_fill.W + 1;
        seq = std::max(seq, chunks_for(tma_rows, g.nb, E.tma_K, htk::fused_round(E.tma_fill.threads, E.tma_K)));
    }
    if (E.ws_ok) {
        const uint64_t ws_rows = rows_per_cta(ws_grid);
        seq = std::max(seq, chunks_for(ws_rows, g.nb, E.fused_K, htk::fused_round(E.ws_fill.threads, E.fused_K)));
    }
    s.seq_max = seq;
    const size_t desc_b = (size_t)grid_cap * seq * 8;
    const size_t cta_b = (size_t)grid_cap * 2 * 4;
    const size_t need = desc_b + cta_b;
    if (need > E.book_bytes || grid_cap != E.grid_cap) {
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
            *why = std::string("synchronise before re-allocation: ") + cudaGetErrorString(e);
            return HT_E_CUDA;
        }
        if (need > E.book_bytes) {
            cudaFree(E.d_book);
            E.d_book = nullptr;
            E.book_bytes = 0;
            if ((e = cudaMalloc(&E.d_book, need)) != cudaSuccess) {
                cudaGetLastError();
                *why = std::string("scan bookkeeping allocation failed: ") + cudaGetErrorString(e);
                return HT_E_NOMEM;
            }
            E.book_bytes = need;
        }
        // cudaMemset of device memory is asynchronous (legacy default stream),
        // and the objects' streams do not wait for that stream: wait here
        if ((e = cudaMemset(E.d_book, 0, need)) != cudaSuccess ||
            (e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess) {
            *why = std::string("scan bookkeeping initialisation failed: ") + cudaGetErrorString(e);
            return HT_E_CUDA;
        }
        E.grid_cap = grid_cap;
    }
    char *p = static_cast<char *>(E.d_book);
    s.desc = reinterpret_cast<uint2 *>(p);
    uint32_t *cta = reinterpret_cast<uint32_t *>(p + desc_b);
    s.cta_nseq = cta;
    s.cta_total = cta + grid_cap;
    s.grid = scan_grid;
    E.fused_valid = false;
    return HT_OK;
}

ht_status engine_create(Engine &E, const ht_binning *b, const ht_ranges *r, uint32_t threshold,
                        uint32_t max_events, uint32_t max_hits, const Tuning *tune, std::string *why)
{
    char buf[256];
    if (!htg::validate(b, r, threshold, why))
        return HT_E_INVAL;
    if (max_events < 1 || max_events > 4096) {
        *why = "need 1 <= max_events <= 4096";
        return HT_E_INVAL;
    }
    if (max_hits > (1u << 26)) {
        *why = "max_hits must be <= 2^26";
        return HT_E_INVAL;
    }
    E.b = *b;
    E.r = *r;
    E.threshold = threshold;
    E.max_events = max_events;
    E.max_hits = max_hits;
    E.max_admit = htg::max_admit(*b);
    E.n_cells = (uint64_t)b->n_theta * b->n_phi * b->n_a * b->n_b;
    if (tune)
        E.tune = *tune;

    cudaError_t e = cudaGetDevice(&E.device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&E.num_sms, cudaDevAttrMultiProcessorCount, E.device);
    if (e != cudaSuccess) {
        std::snprintf(buf, sizeof buf, "no usable CUDA device: %s", cudaGetErrorString(e));
        *why = buf;
        return HT_E_CUDA;
    }

    E.et.resize(b->n_theta + 1);
    E.ep.resize(b->n_phi + 1);
    htg::theta_edges(r->theta_min, r->theta_max, b->n_theta, E.et.data());
    htg::phi_edges(r->phi_min, r->phi_max, b->n_phi, E.ep.data());

    htk::Geom &g = E.geom;
    g.nt = b->n_theta;
    g.np = b->n_phi;
    g.na = b->n_a;
    g.nb = b->n_b;
    g.wt = b->win_theta;
    g.wp = b->win_phi;
    g.n_slices = b->n_theta * b->n_phi;
    g.phi_full = htg::phi_is_full_circle(r->phi_min, r->phi_max) ? 1u : 0u;
    g.max_admit = E.max_admit;
    g.threshold = threshold;
    g.a_min = r->a_min;
    g.b_min = r->b_min;
    // dA = fl((a_max - a_min) / n_a), dB likewise, in FP32
    g.da = htg::delta(r->a_min, r->a_max, b->n_a);
    g.db = htg::delta(r->b_min, r->b_max, b->n_b);
    g.nbf = (float)b->n_b;
    g.inv_db = (float)(1.0 / (double)g.db);
    E.bth.resize(b->n_b + 1);
    htg::b_thresholds(g.b_min, g.db, b->n_b, E.bth.data());

    ht_status st = engine_configure(E, why);
    if (st != HT_OK) {
        engine_destroy(E);
        return st;
    }

    // Entries are the fused fill's candidates (cells >= T) or the scan's
    // peaks; both hold >= T votes each, so there are at most votes / T of
    // them (and no more than the cells).
    htk::ScanArgs &s = E.scan;
    const uint64_t slack = 2ull * 1024;
    const uint64_t by_votes = (uint64_t)std::max<uint32_t>(max_hits, 1) * E.max_admit * g.na / threshold + 1;
    const uint64_t by_cells = E.n_cells * max_events;
    s.entries_cap = (uint32_t)std::min<uint64_t>(std::min(by_votes, by_cells) + slack, 0xffffffffull);

    size_t acc = 0;
    const size_t hits_cap = (size_t)std::max<uint32_t>(max_hits, 1);
    const uint32_t ctr_words = engine_ctr_words(E);
    const size_t units = (size_t)max_events * g.n_slices;
    const uint64_t list_cap = std::min<uint64_t>((uint64_t)hits_cap * E.max_admit, 0xffffffffull);
    E.split_cap = (uint32_t)E.num_sms * 32 + 1;   // a fill grid of up to 32 CTAs per SM
    E.list_cap = (uint32_t)list_cap;
    if ((e = dalloc(&E.d_edges, (E.et.size() + E.ep.size() + E.bth.size()) * 4, &acc)) != cudaSuccess ||
        (e = dalloc(&E.d_M, (size_t)E.n_cells * 4 * max_events + 256, &acc)) != cudaSuccess ||
        (e = dalloc(&E.d_hits4, hits_cap * 16, &acc)) != cudaSuccess ||
        (e = dalloc(&E.d_codes, hits_cap * 4, &acc)) != cudaSuccess ||
        (e = dalloc(&E.d_slice, (3 * units + 1) * 4, &acc)) != cudaSuccess ||
        (e = dalloc(&E.d_list, (size_t)list_cap * 16, &acc)) != cudaSuccess ||
        (e = dalloc(&E.d_entries, (size_t)s.entries_cap * 16, &acc)) != cudaSuccess ||
        (e = dalloc(&E.d_ctr, (size_t)ctr_words * 4, &acc)) != cudaSuccess ||
        (e = dalloc(&E.d_split, (size_t)E.split_cap * 8, &acc)) != cudaSuccess) {
        std::snprintf(buf, sizeof buf, "device allocation of %zu bytes failed: %s", acc,
                      cudaGetErrorString(e));
        *why = buf;
        cudaGetLastError();
        engine_destroy(E);
        return HT_E_NOMEM;
    }
    E.device_bytes = acc + E.book_bytes;
    g.et = E.d_edges;
    g.ep = E.d_edges + E.et.size();
    g.bth = E.d_edges + E.et.size() + E.ep.size();
    if ((e = cudaMemcpy(E.d_edges, E.et.data(), E.et.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(E.d_edges + E.et.size(), E.ep.data(), E.ep.size() * 4, cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(E.d_edges + E.et.size() + E.ep.size(), E.bth.data(), E.bth.size() * 4,
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(E.d_ctr, 0, (size_t)ctr_words * 4)) != cudaSuccess ||
        (e = cudaMemset(E.d_slice, 0, (3 * units + 1) * 4)) != cudaSuccess ||
        (e = cudaMemset(E.d_M, 0, (size_t)E.n_cells * 4 * max_events)) != cudaSuccess ||
        // the memsets are asynchronous on the legacy default stream, which the
        // objects' non-blocking streams do not wait for: finish them here
        (e = cudaStreamSynchronize(cudaStreamLegacy)) != cudaSuccess) {
        std::snprintf(buf, sizeof buf, "device initialisation failed: %s", cudaGetErrorString(e));
        *why = buf;
        engine_destroy(E);
        return HT_E_CUDA;
    }
    s.entries = E.d_entries;
    s.g_count = E.d_ctr + htk::CTR_ENTRIES;
    s.ev_count = E.d_ctr + htk::CTR_EVENTS;
    return HT_OK;
}

ht_status engine_ensure_any_matrix(Engine &E, std::string *why)
{
    const htk::Geom &g = E.geom;
    const uint64_t by_space = (uint64_t)g.n_slices * ((g.na + 1) / 2) * ((g.nb + 1) / 2) * E.max_events +
                              2ull * 1024;
    E.fused_valid = false;
    if (by_space <= E.scan.entries_cap)
        return HT_OK;
    if (by_space > 0xffffffffull) {
        *why = "matrix too large for an arbitrary-content peak scan";
        return HT_E_NOMEM;
    }
    uint4 *p = nullptr;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMalloc(&p, by_space * 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *why = std::string("peak scratch allocation failed: ") + cudaGetErrorString(e);
        return HT_E_NOMEM;
    }
    cudaFree(E.d_entries);
    E.device_bytes += (by_space - E.scan.entries_cap) * 16;
    E.d_entries = p;
    E.scan.entries = p;
    E.scan.entries_cap = (uint32_t)by_space;
    return HT_OK;
}

void engine_destroy(Engine &E)
{
    prof_collect(E);
    for (cudaEvent_t ev : E.prof.pool)
        cudaEventDestroy(ev);
    E.prof.pool.clear();
    cudaFree(E.d_edges);
    cudaFree(E.d_M);
    cudaFree(E.d_hits4);
    cudaFree(E.d_codes);
    cudaFree(E.d_slice);
    cudaFree(E.d_split);
    cudaFree(E.d_list);
    cudaFree(E.d_edge);
    cudaFree(E.d_entries);
    cudaFree(E.d_book);
    cudaFree(E.d_ctr);
    E.d_edges = nullptr;
    E.d_M = nullptr;
    E.d_hits4 = nullptr;
    E.d_codes = nullptr;
    E.d_slice = nullptr;
    E.d_split = nullptr;
    E.d_list = nullptr;
    E.d_edge = nullptr;
    E.edge_pass = 0;
    E.d_entries = nullptr;
    E.d_book = nullptr;
    E.d_ctr = nullptr;
    E.book_bytes = 0;
}

static htk::Work make_work(Engine &E, const float *x, const float *y, const float *z,
                           const uint32_t *d_hit_off, uint32_t n_hits0, uint32_t n_events)
{
    htk::Work w{};
    w.x = x;
    w.y = y;
    w.z = z;
    w.hit_off = d_hit_off;
    w.n_hits0 = n_hits0;
    w.n_events = n_events;
    w.hits4 = E.d_hits4;
    w.codes = E.d_codes;
    w.M = E.d_M;
    w.n_cells = E.n_cells;
    w.status = engine_status(E);
    w.ctr = E.d_ctr;
    const size_t units = (size_t)E.max_events * E.geom.n_slices;
    w.slice_cnt = E.d_slice;
    w.slice_fill = E.d_slice + units;
    w.slice_off = E.d_slice + 2 * units;
    w.list = E.d_list;
    w.list_cap = E.list_cap;
    w.edge = E.d_edge;
    w.edge_pass = E.edge_pass;
    w.split_mode = E.split_mode;
    w.split_grid = E.split_grid;
    w.split_strips = E.split_strips;
    w.split_vw = E.split_vw;
    w.split_n_static = E.split_n_static;
    w.split = E.d_split;
    return w;
}

// When engine_vote's next fill for these flags is one whose work split
// k_bin_cluster can hand over -- the bulk-copy-tile fill (k_fill_tma) or the
// peaks-only fill (k_fill_peaks) -- its configuration and grid, and whether
// fill_blocks_per_sm holds it below its occupancy (the fill checks the shape
// and splits by itself on a mismatch).
static bool split_fill_next(const Engine &E, uint32_t n_events, uint32_t flags, htk::FillCfg &ff, uint32_t &grid,
                            bool &capped)
{
    if ((flags & (HT_FILL_NAIVE | HT_ACCUMULATE)) || !E.fill_priv_ok)
        return false;
    const bool peaks_only = (flags & HT_PEAKS_ONLY) && E.fused_ok && E.d_edge &&
                            E.edge_pass * std::max<uint32_t>(1, E.fused_fill.W / 2) >= E.geom.na;
    uint32_t g0;
    if (peaks_only) {
        ff = E.fused_fill;
        ff.vote_weight = htk::kPeaksVoteWeight;
        g0 = E.fused_grid;
        capped = E.fused_capped;
    } else {
        if (!E.use_tma || E.use_ws)
            return false;
        ff = E.tma_fill;
        ff.vote_weight = htk::kVoteWeight;
        g0 = E.tma_grid;
        capped = E.tma_capped;
    }
    ff.accumulate = 0u;
    const uint64_t items = (uint64_t)n_events * E.geom.n_slices * ff.strips;
    grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(g0, items));
    return grid + 1 <= E.split_cap;
}

cudaError_t engine_fill(Engine &E, const float *x, const float *y, const float *z,
                        const uint32_t *d_hit_off, uint32_t n_hits0, uint32_t n_events,
                        uint32_t n_total, uint32_t flags, cudaStream_t st)
{
    E.fused_valid = false;
    htk::FillCfg ff{};
    uint32_t grid = 0;
    bool capped = false;
    const bool split_next = split_fill_next(E, n_events, flags, ff, grid, capped);
    const bool want_cluster = E.tune.bin_cluster == 1 || (E.tune.bin_cluster == 0 && split_next && !capped);
    const bool cluster = want_cluster && E.bin_cluster > 0 &&
                         n_total <= htk::kBinClusterMax * htk::kBinClusterThreads * htk::kBinClusterHPT &&
                         htk::bin_cluster_smem_bytes(E.geom, n_events) <= htk::kBinClusterSmem;
    cudaError_t e;
    if (cluster) {
        // few hits: binning and unit lists in one cluster launch, one CTA per
        // kBinClusterThreads hits (two hits a thread past kBinClusterMax CTAs)
        if (split_next) {
            const uint64_t items = (uint64_t)n_events * E.geom.n_slices * ff.strips;
            E.split_mode = htk::kSplitGiven;
            E.split_grid = grid;
            E.split_strips = ff.strips;
            E.split_vw = ff.vote_weight;
            E.split_n_static = items - (ff.dyn ? htk::dyn_items(items, grid) : 0);
        } else {
            E.split_mode = htk::kSplitAfterWait;   // the offsets come from the launch right before the fill
        }
        const htk::Work w = make_work(E, x, y, z, d_hit_off, n_hits0, n_events);
        const uint32_t cs = std::min<uint32_t>(
            htk::kBinClusterMax, std::max<uint32_t>(1u, (n_total + htk::kBinClusterThreads - 1) / htk::kBinClusterThreads));
        {
            ProfScope ps(E, K_BIN_CLUSTER, st);
            e = htk::launch_bin_cluster(E.geom, w, cs, st);
        }
        if (e != cudaSuccess)
            return e;
        ++E.launches;
    } else {
        E.split_mode = htk::kSplitEarly;
        const htk::Work w = make_work(E, x, y, z, d_hit_off, n_hits0, n_events);
        const uint32_t bgrid = std::max<uint32_t>(1, std::min<uint32_t>((n_total + 255) / 256, E.num_sms * 8));
        {
            ProfScope ps(E, K_BIN, st);
            e = htk::launch_bin(E.geom, w, bgrid, st);
        }
        if (e != cudaSuccess)
            return e;
        ++E.launches;
        {
            ProfScope ps(E, K_SCATTER, st);
            e = htk::launch_scatter(E.geom, w, bgrid, st);
        }
        if (e != cudaSuccess)
            return e;
        ++E.launches;
    }
    E.ctr_dirty = false;   // the binning zeroed the counters
    E.last_hit_off = d_hit_off;
    E.last_n_hits0 = n_hits0;
    E.last_n_events = n_events;
    E.last_accumulate = (flags & HT_ACCUMULATE) != 0;
    return engine_vote(E, d_hit_off, n_hits0, n_events, flags, st);
}

cudaError_t engine_vote(Engine &E, const uint32_t *d_hit_off, uint32_t n_hits0, uint32_t n_events, uint32_t flags,
                        cudaStream_t st)
{
    htk::Work w = make_work(E, nullptr, nullptr, nullptr, d_hit_off, n_hits0, n_events);
    cudaError_t e;
    E.fused_valid = false;
    const bool accumulate = (flags & HT_ACCUMULATE) != 0;
    if ((flags & HT_FILL_NAIVE) || !E.fill_priv_ok) {
        if (!accumulate) {
            ProfScope ps(E, K_CLEAR, st);
            if ((e = htk::launch_clear(E.d_M, E.n_cells * n_events, E.clear_grid, st)) != cudaSuccess)
                return e;
            ++E.launches;
        }
        ProfScope ps(E, K_FILL_NAIVE, st);
        e = htk::launch_fill_naive(E.geom, w, (uint32_t)E.num_sms, st);
        ++E.launches;
        return e;
    }
    htk::FillCfg f = E.fill;
    f.accumulate = accumulate ? 1u : 0u;
    const uint64_t items = (uint64_t)n_events * E.geom.n_slices * f.strips;
    const bool peaks_only = (flags & HT_PEAKS_ONLY) && E.fused_ok && E.d_edge &&
                            E.edge_pass * std::max<uint32_t>(1, E.fused_fill.W / 2) >= E.geom.na;
    if ((E.use_ws || E.use_tma || E.fused_ok) && !accumulate) {
        htk::ScanArgs a = E.scan;
        const bool ws = E.use_ws && !peaks_only;
        const bool tma = !ws && E.use_tma && !peaks_only;
        a.K = tma ? E.tma_K : E.fused_K;
        htk::FillCfg ff = ws ? E.ws_fill : tma ? E.tma_fill : E.fused_fill;
        ff.accumulate = 0u;
        ff.vote_weight = peaks_only ? htk::kPeaksVoteWeight : htk::kVoteWeight;
        const uint64_t items_ff = (uint64_t)n_events * E.geom.n_slices * ff.strips;
        const uint32_t grid = (uint32_t)std::max<uint64_t>(
            1, std::min<uint64_t>(ws ? E.ws_grid : tma ? E.tma_grid : E.fused_grid, items_ff));
        const uint32_t lists = grid + (ff.dyn ? (uint32_t)htk::dyn_items(items_ff, grid) : 0u);
        {
            ProfScope ps(E, ws ? K_FILL_WS : tma ? K_FILL_TMA : peaks_only ? K_FILL_PEAKS : K_FILL_SCAN, st);
            e = ws ? htk::launch_fill_ws(E.geom, w, ff, a, grid, st)
               : tma ? htk::launch_fill_tma(E.geom, w, ff, a, grid, st)
               : peaks_only ? htk::launch_fill_peaks(E.geom, w, ff, a, grid, st)
                            : htk::launch_fill_scan(E.geom, w, ff, a, grid, st);
        }
        ++E.launches;
        if (e == cudaSuccess) {
            ProfScope ps(E, K_PEAKS, st);
            e = htk::launch_peaks(E.geom, w, ff, a, lists, peaks_only, st);
            ++E.launches;
        }
        if (e == cudaSuccess) {
            E.fused_valid = true;
            E.ctr_dirty = true;
            E.fused_grid_used = lists;
            E.fused_events = n_events;
        }
        return e;
    }
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(E.fill_grid, items));
    ProfScope ps(E, K_FILL_PRIV, st);
    e = htk::launch_fill_priv(E.geom, w, f, grid, st);
    ++E.launches;
    return e;
}

cudaError_t engine_scan(Engine &E, uint32_t n_events, htk::Peak *out, uint32_t capacity,
                        uint32_t *counts, cudaStream_t st, bool compact)
{
    htk::Work w = make_work(E, nullptr, nullptr, nullptr, nullptr, 0, n_events);
    htk::ScanArgs a = E.scan;
    htk::OrderArgs o{};
    o.out = out;
    o.capacity = capacity;
    o.counts = counts;
    o.ev_count = E.d_ctr + htk::CTR_EVENTS;
    o.ticket = E.d_ctr + htk::CTR_OTICKET;
    o.g_count = E.d_ctr + htk::CTR_ENTRIES;
    o.compact = compact ? 1u : 0u;
    cudaError_t e;
    if (E.fused_valid && E.fused_events == n_events) {
        // the fused fill already found the peaks: only order them
        a.grid = E.fused_grid_used;
        E.fused_valid = false;
    } else {
        if (E.ctr_dirty) {
            // an unconsumed fused fill left its counters: start from zero
            e = cudaMemsetAsync(E.d_ctr + htk::CTR_ENTRIES, 0,
                                (engine_ctr_words(E) - htk::CTR_ENTRIES) * sizeof(uint32_t), st);
            if (e != cudaSuccess)
                return e;
        }
        E.fused_valid = false;
        const uint64_t G = (uint64_t)E.geom.n_slices * E.geom.na * n_events;
        a.grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(a.grid, G));
        {
            ProfScope ps(E, K_SCAN, st);
            e = htk::launch_scan(E.geom, w, a, E.scan_kind, st);
        }
        if (e != cudaSuccess)
            return e;
        ++E.launches;
    }
    {
        ProfScope ps(E, K_ORDER, st);
        e = htk::launch_order(E.geom, w, a, o, st);
    }
    ++E.launches;
    E.ctr_dirty = false;   // the order kernel's last CTA zeroes them
    return e;
}

cudaError_t engine_scan4d(Engine &E, htk::Peak *p2, uint8_t *keep, uint32_t p2_cap, uint32_t *p2_count,
                          htk::Peak *out, uint32_t capacity, uint32_t *counts, cudaStream_t st)
{
    cudaError_t e = engine_scan(E, 1, p2, p2_cap, p2_count, st);
    if (e != cudaSuccess)
        return e;
    {
        ProfScope ps(E, K_PEAKS4D, st);
        e = htk::launch_peaks4d(E.geom, E.d_M, p2, p2_count, p2_cap, keep, out, capacity, counts,
                                E.d_ctr + htk::CTR_P4TICKET, E.d_ctr + htk::CTR_STATUS, (uint32_t)E.num_sms * 2u,
                                st);
    }
    ++E.launches;
    return e;
}

// ---------------------------------------------------------------------------
// Autotuner
// ---------------------------------------------------------------------------
ht_status engine_autotune(Engine &E, uint32_t reps, cudaStream_t st, double *best_us, std::string *why)
{
    if (!E.last_n_events) {
        *why = "autotune needs a previous fill (it re-times that fill's hits)";
        return HT_E_INVAL;
    }
    if (E.last_accumulate) {
        *why = "autotune re-runs the last fill alone: not after an accumulating fill";
        return HT_E_INVAL;
    }
    reps = std::max<uint32_t>(reps, 1);
    const uint32_t n_events = E.last_n_events;
    uint32_t *d_counts = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&d_counts, (size_t)n_events * 4)) != cudaSuccess ||
        (e = cudaEventCreate(&t0)) != cudaSuccess || (e = cudaEventCreate(&t1)) != cudaSuccess) {
        cudaFree(d_counts);
        cudaGetLastError();
        *why = std::string("autotune set-up failed: ") + cudaGetErrorString(e);
        return HT_E_NOMEM;
    }
    const Tuning user = E.tune;
    const bool prof_on = E.prof.on;
    E.prof.on = false;

    // candidates: fused / two-kernel fill, tile rows, threads, scan variant
    std::vector<Tuning> cands;
    const uint32_t rows_opts[] = {16, 32};
    const uint32_t thr_opts[] = {256, 512};
    for (uint32_t fused = 1; fused <= 5; ++fused)
        for (uint32_t W : rows_opts)
            for (uint32_t th : thr_opts)
                for (uint32_t kind = 1; kind <= (fused == 2 ? 2u : 1u); ++kind) {
                    if (fused == 5) {
                        // the bulk-copy-tile kernel: its own row counts (0 = two 64 KB tiles)
                        if (th == thr_opts[0])
                            continue;
                        for (uint32_t Wt : {0u, W / 2})
                            for (uint32_t tt : {512u, 1024u}) {
                                Tuning t = user;
                                t.fused = 5;
                                t.fill_W = Wt;
                                t.fill_threads = tt;
                                cands.push_back(t);
                            }
                        continue;
                    }
                    if (fused == 3 && th != htk::kWsThreads / 2)
                        continue;                // one group size for the warp-specialised kernel
                    if (fused == 4 && th != thr_opts[0])
                        continue;                // the bulk-store kernel: its own block size (1024)
                    Tuning t = user;
                    t.fused = fused;
                    t.fill_W = W;
                    t.fill_threads = fused == 4 ? 0u : th;
                    t.scan_kind = fused == 2 ? (kind == 1 ? 2u : 1u) : user.scan_kind;
                    cands.push_back(t);
                }

    double best = 1e30;
    Tuning chosen = user;
    ht_status st_out = HT_OK;
    for (const Tuning &t : cands) {
        E.tune = t;
        std::string w2;
        if (engine_configure(E, &w2) != HT_OK)
            continue;                            // shape does not fit this binning
        bool ok = true;
        float ms = 0.f;
        for (uint32_t r = 0; r < reps + 2 && ok; ++r) {
            if (r == 2 && cudaEventRecord(t0, st) != cudaSuccess)
                ok = false;
            ok = ok && engine_vote(E, E.last_hit_off, E.last_n_hits0, n_events, 0u, st) == cudaSuccess &&
                 engine_scan(E, n_events, nullptr, 0u, d_counts, st) == cudaSuccess;
        }
        ok = ok && cudaEventRecord(t1, st) == cudaSuccess && cudaEventSynchronize(t1) == cudaSuccess &&
             cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess;
        if (!ok) {
            *why = std::string("autotune run failed: ") + cudaGetErrorString(cudaGetLastError());
            st_out = HT_E_CUDA;
            break;
        }
        const double us = 1e3 * ms / reps / n_events;
        if (us < best) {
            best = us;
            chosen = t;
        }
    }
    E.tune = st_out == HT_OK ? chosen : user;
    std::string w3;
    if (engine_configure(E, &w3) != HT_OK && st_out == HT_OK) {
        *why = w3;
        st_out = HT_E_CUDA;
    }
    // leave M_H and the peak state as a fill with the chosen tuning leaves them
    if (st_out == HT_OK && engine_vote(E, E.last_hit_off, E.last_n_hits0, n_events, 0u, st) != cudaSuccess) {
        *why = "autotune final fill failed";
        st_out = HT_E_CUDA;
    }
    cudaStreamSynchronize(st);
    E.prof.on = prof_on;
    cudaFree(d_counts);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (best_us)
        *best_us = best;
    return st_out;
}

ht_status engine_set_tuning(Engine &E, const ht_tuning &t, bool *poisoned, std::string *why)
{
    if (t.scan_kind > HT_SCAN_DIRECT) {
        *why = "unknown scan_kind";
        return HT_E_INVAL;
    }
    Tuning old = E.tune;
    Tuning &n = E.tune;
    n.fill_W = t.fill_rows;
    n.fill_threads = t.fill_threads;
    n.fill_HC = t.fill_hits_staged;
    n.fill_blocks_per_sm = t.fill_blocks_per_sm;
    n.scan_kind = t.scan_kind;
    n.scan_stage_bytes = t.scan_stage_bytes;
    n.scan_slots = t.scan_slots;
    n.scan_blocks_per_sm = t.scan_blocks_per_sm;
    n.fused = t.fill_fused_scan;
    n.vote_agg = t.fill_vote_agg;
    n.bin_cluster = t.bin_cluster;
    ht_status s = engine_configure(E, why);
    if (s != HT_OK) {
        E.tune = old;
        std::string why2;
        if (engine_configure(E, &why2) != HT_OK)
            *poisoned = true;
    }
    return s;
}

void engine_get_tuning(const Engine &E, ht_tuning *t)
{
    t->fill_rows = E.fill.W;
    t->fill_threads = E.fill.threads;
    t->fill_hits_staged = E.fill.HC;
    t->fill_blocks_per_sm = E.num_sms ? E.fill_grid / (uint32_t)E.num_sms : 0;
    t->scan_kind = E.scan_kind == htk::SCAN_BULK ? HT_SCAN_BULK
                 : E.scan_kind == htk::SCAN_LDG ? HT_SCAN_STREAM : HT_SCAN_DIRECT;
    t->scan_stage_bytes = E.scan.slot_words * 4;
    t->scan_slots = E.scan.S;
    t->scan_blocks_per_sm = E.num_sms ? E.scan_grid_max / (uint32_t)E.num_sms : 0;
    t->fill_fused_scan = E.use_ws ? 3u : E.use_tma ? 5u : E.fused_ok ? (E.fused_fill.bulk ? 4u : 1u) : 2u;
    t->fill_vote_agg = E.use_tma ? E.tma_fill.vote_agg : 0u;
    t->bin_cluster = E.tune.bin_cluster ? E.tune.bin_cluster : (E.use_tma && !E.tma_capped) ? 1u : 2u;
    if (E.use_tma) {
        t->fill_rows = E.tma_fill.W;
        t->fill_threads = E.tma_fill.threads;
        t->fill_hits_staged = E.tma_fill.HC;
        t->fill_blocks_per_sm = E.num_sms ? E.tma_grid / (uint32_t)E.num_sms : 0;
    }
}

cudaError_t prof_read(Engine &E, ht_kernel_time *out, uint32_t cap, uint32_t *n)
{
    cudaError_t e = prof_collect(E);
    if (e != cudaSuccess)
        return e;
    uint32_t k = 0;
    for (int i = 0; i < K_NKINDS; ++i) {
        if (k < cap) {
            std::memset(&out[k], 0, sizeof(ht_kernel_time));
            std::strncpy(out[k].name, kKernelNames[i], sizeof(out[k].name) - 1);
            out[k].launches = E.prof.n[i];
            out[k].total_ms = E.prof.ms[i];
        }
        ++k;
    }
    *n = k;
    return cudaSuccess;
}

cudaError_t engine_set_phi_edges(Engine &E, const float *ep)
{
    std::copy(ep, ep + E.ep.size(), E.ep.begin());
    // a pageable-source copy may still be in flight when cudaMemcpy returns,
    // on the legacy stream the object's streams do not wait for
    cudaError_t e = cudaMemcpy(E.d_edges + E.et.size(), E.ep.data(), E.ep.size() * 4, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? cudaStreamSynchronize(cudaStreamLegacy) : e;
}

ht_status engine_ensure_edges(Engine &E, std::string *why)
{
    // passes per unit at the smallest pass height (u32 tiles: W / 2 rows)
    const uint32_t rpass_min = std::max<uint32_t>(1, E.fused_fill.W / 2);
    const uint32_t passes = (E.geom.na + rpass_min - 1) / rpass_min;
    if (E.d_edge && E.edge_pass >= passes)
        return HT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        *why = std::string("synchronise before allocation: ") + cudaGetErrorString(e);
        return HT_E_CUDA;
    }
    cudaFree(E.d_edge);
    E.d_edge = nullptr;
    E.edge_pass = 0;
    const size_t bytes = (size_t)E.max_events * E.geom.n_slices * passes * 2 * E.geom.nb * 4;
    if ((e = cudaMalloc(&E.d_edge, bytes)) != cudaSuccess) {
        cudaGetLastError();
        *why = std::string("edge-row buffer allocation failed: ") + cudaGetErrorString(e);
        return HT_E_NOMEM;
    }
    E.edge_pass = passes;
    E.device_bytes += bytes;
    return HT_OK;
}

} // namespace hte
