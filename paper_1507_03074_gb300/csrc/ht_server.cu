// C ABI: the serving loop (ht_server_*, ht_submit, ht_poll).
//
// Requests (one event each) queue on the host; a worker thread packs the
// waiting requests of one (binning, ranges, threshold) into a micro-batch
// and runs it on a free lane -- a Runner (resident vote matrices, staging,
// mapped pinned outputs) with its own stream -- through the same graph-
// replayed kernel sequence as ht_batch_run.  Several lanes run at once, so
// requests that arrive while others are on the GPU start as soon as a lane
// frees up, and their work overlaps on the device.  An event recorded behind
// each micro-batch tells the worker that it is done; while any lane is busy,
// or for kIdleSpin after the last activity, the worker polls those events
// and the queue instead of sleeping, so neither a completion nor an arrival
// waits for a thread to be woken.  Lanes of larger matrices get streams of
// higher priority: a long fill is not stretched by the short ones that start
// beside it (the latency tail is the long events').
//
// Locking: `mu` guards the queues and requests and is never held across a
// CUDA call.
#include "ht_geom.h"
#include "ht_runner.h"
#include "ht_trace.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

namespace hte {
ht_status report(ht_status s, const std::string &msg);   // ht_api.cu
}

namespace {

using Clock = std::chrono::steady_clock;

struct Key {
    ht_binning b;
    ht_ranges r;
    uint32_t threshold;
    bool operator==(const Key &o) const
    {
        return std::memcmp(&b, &o.b, sizeof b) == 0 && std::memcmp(&r, &o.r, sizeof r) == 0 &&
               threshold == o.threshold;
    }
};

struct Request {
    uint64_t ticket = 0;
    Key key{};
    uint32_t n = 0;
    std::vector<float> xyz;          // x | y | z
    Clock::time_point t_submit, t_done;
    std::atomic<bool> done{false};   // set under mu; read without it while a poller spins
    ht_status status = HT_OK;
    uint32_t n_found = 0;
    std::vector<ht_peak> peaks;      // the first min(n_found, room) peaks
};

struct Lane {
    Key key{};
    hte::Runner R;
    cudaStream_t st = nullptr;
    uint32_t events = 0;             // micro-batch size
    uint64_t bytes = 0;              // device memory held
    bool busy = false;
    cudaEvent_t done_ev = nullptr;   // recorded behind the running micro-batch
    std::vector<Request *> reqs;     // the running micro-batch
    Clock::time_point last_used;
    struct ht_server *srv = nullptr;
};

} // namespace

struct ht_server {
    ht_server_cfg cfg{};
    int device = 0;
    std::mutex mu;                   // queues, requests, stats
    std::condition_variable done_cv; // pollers
    std::deque<Request *> waiting;
    std::unordered_map<uint64_t, Request *> tickets;
    uint64_t next_ticket = 1;
    std::vector<std::unique_ptr<Lane>> lanes;   // owned by the worker
    uint64_t lane_bytes = 0;
    bool stop = false;
    // wake-up of the worker (submit, host functions)
    std::mutex wake_mu;
    std::condition_variable wake_cv;
    bool wake = false;
    std::thread worker;
    // stats
    uint64_t submitted = 0, completed = 0, in_flight = 0, micro_batches = 0, batched_events = 0;
    std::vector<double> lat_us;
};

namespace {

void wake_worker(ht_server *s)
{
    {
        std::lock_guard<std::mutex> g(s->wake_mu);
        s->wake = true;
    }
    s->wake_cv.notify_one();
}

uint64_t matrix_bytes(const Key &k)
{
    return (uint64_t)k.b.n_theta * k.b.n_phi * k.b.n_a * k.b.n_b * 4;
}

// Device memory of a lane with `events` events: matrices, hit workspace and
// staging, the peak scratch (bounded like the engine bounds it) and a margin
// for the bookkeeping.
uint64_t lane_estimate(const ht_server_cfg &, const Key &k, uint32_t events, uint32_t max_hits)
{
    const ht_binning &b = k.b;
    const uint64_t admit = (2ull * b.win_theta + 1) * (2ull * b.win_phi + 1);
    const uint64_t by_votes = (uint64_t)max_hits * admit * b.n_a / k.threshold + 1;
    const uint64_t by_space = (uint64_t)b.n_theta * b.n_phi * ((b.n_a + 1) / 2) * ((b.n_b + 1) / 2) * events;
    return matrix_bytes(k) * events + (uint64_t)max_hits * 64 + std::min(by_votes, by_space) * 16 + (32ull << 20);
}

uint32_t lane_hits(const ht_server_cfg &c, uint32_t events)
{
    return std::max<uint32_t>(c.max_hits_per_event, std::min<uint64_t>((uint64_t)events * 6000, 1u << 26));
}

// Results of a finished micro-batch into its requests.
void harvest(ht_server *s, Lane &l)
{
    hte::TraceRange tr("ht_server harvest");
    hte::Runner &R = l.R;
    std::string why;
    const uint32_t status = R.h_counts[R.E.max_events];
    ht_status st = hte::runner_status(R, status, l.st, &why);
    const uint32_t n_ev = (uint32_t)l.reqs.size();
    std::vector<uint32_t> counts(R.h_counts, R.h_counts + n_ev);
    uint64_t off = 0;
    for (uint32_t e = 0; e < n_ev; ++e) {
        Request *q = l.reqs[e];
        q->status = st;
        if (st == HT_OK) {
            q->n_found = counts[e];
            const uint64_t b0 = std::min<uint64_t>(off, R.capacity), b1 = std::min<uint64_t>(off + counts[e], R.capacity);
            q->peaks.assign(reinterpret_cast<const ht_peak *>(R.h_out) + b0,
                            reinterpret_cast<const ht_peak *>(R.h_out) + b1);
            for (auto &p : q->peaks)
                p.event = 0;
            if (b1 - b0 < counts[e])
                q->status = HT_TRUNCATED;
        }
        off += counts[e];
    }
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        for (Request *q : l.reqs) {
            q->t_done = now;
            q->done = true;
            if (s->lat_us.size() < (1u << 22))
                s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - q->t_submit).count());
            ++s->completed;
            --s->in_flight;
        }
    }
    s->done_cv.notify_all();
    l.reqs.clear();
    l.busy = false;
    l.last_used = now;
}

// (worker thread only; the vector changes under mu for the stats reader)
void free_lane(ht_server *s, size_t i)
{
    Lane &l = *s->lanes[i];
    cudaStreamSynchronize(l.st);
    hte::runner_destroy(l.R);
    cudaEventDestroy(l.done_ev);
    cudaStreamDestroy(l.st);
    std::lock_guard<std::mutex> g(s->mu);
    s->lane_bytes -= l.bytes;
    s->lanes.erase(s->lanes.begin() + (long)i);
}

// Stream priority of a lane: one level above the lowest per doubling of its
// matrix beyond 64 MiB, capped at the device's highest (the 256 MiB paper
// binning two levels up, the 4 GiB upgrade binning at the top).
int lane_priority(const Key &k)
{
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int up = 0;
    for (uint64_t b = matrix_bytes(k); b > (64ull << 20); b >>= 1)
        ++up;
    return std::max(greatest, least - up);
}

// A new lane for key k, within the budget (freeing idle lanes of other
// binnings if needed).  nullptr if it cannot be had now; *never is set when
// even a one-event lane can never fit.
Lane *make_lane(ht_server *s, const Key &k, bool *never)
{
    const ht_server_cfg &c = s->cfg;
    *never = false;
    // events per lane: what a fair share of the budget holds, 1 .. max_batch
    const uint64_t share = c.hbm_budget_bytes / (2ull * c.n_streams);
    uint32_t events = (uint32_t)std::min<uint64_t>(c.max_batch, std::max<uint64_t>(1, share / matrix_bytes(k)));
    uint64_t need = lane_estimate(c, k, events, lane_hits(c, events));
    if (lane_estimate(c, k, 1, lane_hits(c, 1)) > c.hbm_budget_bytes) {
        *never = true;
        return nullptr;
    }
    while (events > 1 && need > c.hbm_budget_bytes) {
        events /= 2;
        need = lane_estimate(c, k, events, lane_hits(c, events));
    }
    // free idle lanes of other binnings, least recently used first
    while (s->lane_bytes + need > c.hbm_budget_bytes) {
        size_t victim = SIZE_MAX;
        for (size_t i = 0; i < s->lanes.size(); ++i) {
            const Lane &l = *s->lanes[i];
            if (!l.busy && !(l.key == k) && (victim == SIZE_MAX || l.last_used < s->lanes[victim]->last_used))
                victim = i;
        }
        if (victim == SIZE_MAX)
            return nullptr;   // wait for busy lanes to finish
        free_lane(s, victim);
    }
    std::unique_ptr<Lane> l(new Lane());
    l->key = k;
    l->srv = s;
    l->events = events;
    std::string why;
    const uint32_t hits = lane_hits(c, events);
    if (hte::runner_create(l->R, &k.b, &k.r, k.threshold, events, hits, events * 8192u, &why) != HT_OK) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaStreamCreateWithPriority(&l->st, cudaStreamNonBlocking, lane_priority(k)) != cudaSuccess) {
        cudaGetLastError();
        hte::runner_destroy(l->R);
        return nullptr;
    }
    if (cudaEventCreateWithFlags(&l->done_ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        cudaStreamDestroy(l->st);
        hte::runner_destroy(l->R);
        return nullptr;
    }
    if (c.fill_blocks_per_sm) {
        ht_tuning t{};
        t.fill_blocks_per_sm = c.fill_blocks_per_sm;
        bool poisoned = false;
        if (hte::engine_set_tuning(l->R.E, t, &poisoned, &why) != HT_OK) {
            cudaGetLastError();
            cudaEventDestroy(l->done_ev);
            cudaStreamDestroy(l->st);
            hte::runner_destroy(l->R);
            return nullptr;
        }
    }
    if ((c.flags & HT_PEAKS_ONLY) && hte::engine_ensure_edges(l->R.E, &why) != HT_OK) {
        cudaGetLastError();
        cudaEventDestroy(l->done_ev);
        cudaStreamDestroy(l->st);
        hte::runner_destroy(l->R);
        return nullptr;
    }
    l->bytes = std::max<uint64_t>(need, l->R.E.device_bytes);
    l->last_used = Clock::now();
    std::lock_guard<std::mutex> g(s->mu);
    s->lane_bytes += l->bytes;
    s->lanes.push_back(std::move(l));
    return s->lanes.back().get();
}

// Stage a micro-batch into the lane and enqueue it.
bool dispatch(ht_server *s, Lane &l, std::vector<Request *> &&reqs)
{
    hte::TraceRange tr("ht_server micro-batch");
    hte::Runner &R = l.R;
    const size_t mh = R.E.max_hits;
    uint32_t off = 0;
    R.h_off[0] = 0;
    for (size_t e = 0; e < reqs.size(); ++e) {
        const Request *q = reqs[e];
        const size_t nb = (size_t)q->n * 4;
        std::memcpy(R.h_xyz + off, q->xyz.data(), nb);
        std::memcpy(R.h_xyz + mh + off, q->xyz.data() + q->n, nb);
        std::memcpy(R.h_xyz + 2 * mh + off, q->xyz.data() + 2 * (size_t)q->n, nb);
        off += q->n;
        R.h_off[e + 1] = off;
    }
    l.reqs = std::move(reqs);
    l.busy = true;
    cudaError_t e = hte::runner_enqueue(R, (uint32_t)l.reqs.size(), off, true, true, l.st,
                                        s->cfg.flags & (uint32_t)HT_PEAKS_ONLY);
    if (e == cudaSuccess)
        e = cudaEventRecord(l.done_ev, l.st);
    return e == cudaSuccess;
}

void fail_requests(ht_server *s, std::vector<Request *> &reqs, ht_status st)
{
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> g(s->mu);
        for (Request *q : reqs) {
            q->status = st;
            q->done = true;
            q->t_done = now;
            ++s->completed;
            --s->in_flight;
        }
    }
    s->done_cv.notify_all();
    reqs.clear();
}

// One pass: dispatch what can start now.  Returns true if anything started.
bool schedule(ht_server *s)
{
    bool started = false;
    std::vector<Key> blocked;        // binnings waiting for memory in this pass
    auto is_blocked = [&](const Key &k) {
        for (const Key &b : blocked)
            if (b == k)
                return true;
        return false;
    };
    for (;;) {
        // the oldest waiting request with a free lane, or room for a new one
        Lane *lane = nullptr;
        Key key{};
        bool any = false;
        {
            std::lock_guard<std::mutex> g(s->mu);
            for (Request *q : s->waiting) {
                if (is_blocked(q->key))
                    continue;
                uint32_t n_key = 0;
                for (auto &l : s->lanes)
                    if (l->key == q->key) {
                        ++n_key;
                        if (!l->busy && !lane)
                            lane = l.get();
                    }
                if (lane || n_key < s->cfg.n_streams) {
                    key = q->key;
                    any = true;
                    break;
                }
            }
        }
        if (!any)
            return started;
        if (!lane) {
            bool never = false;
            lane = make_lane(s, key, &never);
            if (!lane) {
                if (never) {
                    // this binning never fits the budget: fail its waiting requests
                    std::vector<Request *> bad;
                    {
                        std::lock_guard<std::mutex> g(s->mu);
                        for (auto it = s->waiting.begin(); it != s->waiting.end();) {
                            if ((*it)->key == key) {
                                bad.push_back(*it);
                                ++s->in_flight;
                                it = s->waiting.erase(it);
                            } else {
                                ++it;
                            }
                        }
                    }
                    fail_requests(s, bad, HT_E_NOMEM);
                } else {
                    blocked.push_back(key);   // wait for memory; others may still start
                }
                continue;
            }
        }
        // the lane's micro-batch: waiting requests of its key, oldest first
        std::vector<Request *> take;
        {
            std::lock_guard<std::mutex> g(s->mu);
            uint64_t hits = 0;
            for (auto it = s->waiting.begin(); it != s->waiting.end() && take.size() < lane->events;) {
                Request *q = *it;
                if (q->key == key && hits + q->n <= lane->R.E.max_hits) {
                    hits += q->n;
                    take.push_back(q);
                    ++s->in_flight;
                    it = s->waiting.erase(it);
                } else {
                    ++it;
                }
            }
            if (!take.empty()) {
                ++s->micro_batches;
                s->batched_events += take.size();
            }
        }
        if (take.empty())
            return started;
        if (!dispatch(s, *lane, std::move(take))) {
            cudaGetLastError();
            fail_requests(s, lane->reqs, HT_E_CUDA);
            lane->busy = false;
            continue;
        }
        started = true;
    }
}

// How long ht_poll spins on its request before it sleeps on the condition
// variable (at most its timeout).
constexpr auto kPollSpin = std::chrono::microseconds(2000);

// How long the worker keeps polling after its last dispatch, completion or
// wake-up before it sleeps on the condition variable.
constexpr auto kIdleSpin = std::chrono::microseconds(2000);

void worker_main(ht_server *s)
{
    cudaSetDevice(s->device);
    Clock::time_point last = Clock::now();
    for (;;) {
        bool stopping;
        {
            std::lock_guard<std::mutex> g(s->mu);
            stopping = s->stop;
        }
        for (auto &l : s->lanes) {
            if (!l->busy)
                continue;
            const cudaError_t q = cudaEventQuery(l->done_ev);
            if (q == cudaErrorNotReady)
                continue;
            if (q != cudaSuccess)
                cudaGetLastError();   // a failed micro-batch: its status word reports it
            harvest(s, *l);
            last = Clock::now();
        }
        bool busy_any = false;
        for (auto &l : s->lanes)
            busy_any = busy_any || l->busy;
        if (stopping && !busy_any)
            break;
        if (!stopping && schedule(s)) {
            busy_any = true;
            last = Clock::now();
        }
        if (busy_any || Clock::now() - last < kIdleSpin) {
            std::this_thread::yield();
            continue;
        }
        std::unique_lock<std::mutex> lk(s->wake_mu);
        s->wake_cv.wait_for(lk, std::chrono::milliseconds(2), [&] { return s->wake; });
        if (s->wake)
            last = Clock::now();
        s->wake = false;
    }
    while (!s->lanes.empty())
        free_lane(s, s->lanes.size() - 1);
}

} // namespace

extern "C" {

ht_status ht_server_create(const ht_server_cfg *cfg, ht_server **out)
{
    if (!out)
        return hte::report(HT_E_INVAL, "out is NULL");
    *out = nullptr;
    ht_server_cfg c = cfg ? *cfg : ht_server_cfg{};
    int dev = 0;
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess)
        return hte::report(HT_E_CUDA, std::string("no usable CUDA device: ") + cudaGetErrorString(e));
    if (!c.hbm_budget_bytes)
        c.hbm_budget_bytes = (uint64_t)(0.8 * (double)free_b);
    if (!c.n_streams)
        c.n_streams = 4;
    if (!c.max_batch)
        c.max_batch = 16;
    if (!c.max_hits_per_event)
        c.max_hits_per_event = 65536;
    if (!c.queue_depth)
        c.queue_depth = 65536;
    if (c.flags & ~(uint32_t)HT_PEAKS_ONLY)
        return hte::report(HT_E_INVAL, "server flags: 0 or HT_PEAKS_ONLY");
    if (c.n_streams > 64 || c.max_batch > 4096 || c.max_hits_per_event > (1u << 24) || c.fill_blocks_per_sm > 32)
        return hte::report(HT_E_INVAL,
                           "n_streams <= 64, max_batch <= 4096, max_hits_per_event <= 2^24, fill_blocks_per_sm <= 32");
    ht_server *s = new (std::nothrow) ht_server();
    if (!s)
        return hte::report(HT_E_NOMEM, "host allocation failed");
    s->cfg = c;
    s->device = dev;
    try {
        s->worker = std::thread(worker_main, s);
    } catch (...) {
        delete s;
        return hte::report(HT_E_NOMEM, "could not start the worker thread");
    }
    *out = s;
    return HT_OK;
}

ht_status ht_server_destroy(ht_server *s)
{
    if (!s)
        return HT_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    wake_worker(s);
    if (s->worker.joinable())
        s->worker.join();
    for (auto &kv : s->tickets)
        delete kv.second;
    delete s;
    return HT_OK;
}

ht_status ht_submit(ht_server *s, const ht_binning *binning, const ht_ranges *ranges, uint32_t threshold,
                    const float *x, const float *y, const float *z, uint32_t n_hits, uint64_t *ticket)
{
    if (!s || !ticket || !binning || !ranges || (n_hits && (!x || !y || !z)))
        return hte::report(HT_E_INVAL, "NULL argument");
    std::string why;
    if (!htg::validate(binning, ranges, threshold, &why))
        return hte::report(HT_E_INVAL, why);
    if (n_hits > s->cfg.max_hits_per_event)
        return hte::report(HT_E_INVAL, "more hits than max_hits_per_event");
    std::unique_ptr<Request> q(new (std::nothrow) Request());
    if (!q)
        return hte::report(HT_E_NOMEM, "host allocation failed");
    q->key = Key{*binning, *ranges, threshold};
    q->n = n_hits;
    q->xyz.resize((size_t)n_hits * 3);
    std::memcpy(q->xyz.data(), x, (size_t)n_hits * 4);
    std::memcpy(q->xyz.data() + n_hits, y, (size_t)n_hits * 4);
    std::memcpy(q->xyz.data() + 2 * (size_t)n_hits, z, (size_t)n_hits * 4);
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->stop)
            return hte::report(HT_E_STATE, "server is shutting down");
        if (s->waiting.size() >= s->cfg.queue_depth)
            return hte::report(HT_E_BUSY, "queue_depth requests are already waiting");
        q->ticket = s->next_ticket++;
        q->t_submit = Clock::now();
        *ticket = q->ticket;
        s->tickets[q->ticket] = q.get();
        s->waiting.push_back(q.release());
        ++s->submitted;
    }
    wake_worker(s);
    return HT_OK;
}

ht_status ht_poll(ht_server *s, uint64_t ticket, ht_peak *out, uint32_t capacity, uint32_t *n_found,
                  uint32_t timeout_us)
{
    if (!s || !n_found || (capacity && !out))
        return hte::report(HT_E_INVAL, "NULL argument");
    const Clock::time_point t_end = Clock::now() + std::chrono::microseconds(timeout_us);
    const Clock::time_point spin_end = std::min(t_end, Clock::now() + kPollSpin);
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end())
        return hte::report(HT_E_INVAL, "unknown ticket");
    Request *q = it->second;
    // spin briefly (the result is usually near), then sleep on the condition
    while (!q->done.load(std::memory_order_acquire) && Clock::now() < spin_end) {
        lk.unlock();
        std::this_thread::yield();
        lk.lock();
        it = s->tickets.find(ticket);   // another poller of the same ticket may have taken it
        if (it == s->tickets.end())
            return hte::report(HT_E_INVAL, "unknown ticket");
    }
    if (!q->done)
        s->done_cv.wait_until(lk, t_end, [&] { return q->done.load(); });
    if (!q->done)
        return HT_PENDING;
    s->tickets.erase(it);
    lk.unlock();
    ht_status st = q->status;
    if (st == HT_OK || st == HT_TRUNCATED) {
        *n_found = q->n_found;
        const size_t k = std::min<size_t>(q->peaks.size(), capacity);
        if (k)
            std::memcpy(out, q->peaks.data(), k * sizeof(ht_peak));
        if (q->n_found > capacity)
            st = HT_TRUNCATED;
    } else {
        *n_found = 0;
        hte::report(st, st == HT_E_NOMEM ? "the event's vote matrix never fits the server's memory budget"
                                         : "the micro-batch of this request failed on the device");
    }
    delete q;
    return st;
}

ht_status ht_server_get_stats(ht_server *s, ht_server_stats *out, int reset)
{
    if (!s || !out)
        return hte::report(HT_E_INVAL, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = s->submitted;
    out->completed = s->completed;
    out->waiting = s->waiting.size();
    out->in_flight = s->in_flight;
    out->micro_batches = s->micro_batches;
    out->mean_batch = s->micro_batches ? (double)s->batched_events / (double)s->micro_batches : 0.0;
    out->lanes = (uint32_t)s->lanes.size();
    out->lane_bytes = s->lane_bytes;
    if (!s->lat_us.empty()) {
        std::vector<double> v = s->lat_us;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = v.back();
        double sum = 0;
        for (double d : v)
            sum += d;
        out->mean_us = sum / (double)v.size();
    }
    if (reset) {
        s->lat_us.clear();
        s->micro_batches = 0;
        s->batched_events = 0;
    }
    return HT_OK;
}

} // extern "C"
