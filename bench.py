"""Benchmark of the Hough-Transform hot path on GB300 (one JSON line).

Workload: paper-scale events (Sec. 2: <= 5000 hits on a 12-layer barrel,
M_H binned 4 x 16 x 1024 x 1024), synthetic and seeded: 396 helix tracks +
238 noise hits = 4990 hits per event, threshold 10.  One step = one event
through the whole hot path: slice admission + counting sort, vote fill
(privatised), threshold + local-maxima scan and ordered compaction.

  value   events/s with hits already resident in HBM (device pointers).
          Events go round-robin to --contexts contexts, each with its own
          stream, so that one event's small kernels and its fill's ragged
          end overlap the next event's work; every event still runs through
          its own per-event launches; the fills take the faster in flight of
          the single-event launch shape and the same at one CTA per SM (two
          events' fills then share every SM).  CUDA events on a stream that forks to
          and joins the launching streams bracket the timed steps; every
          step's peak count is checked.  `one_context` is the same with one
          context (one event at a time).
  e2e     the same through the C ABI with host buffers: every step copies
          its hits host->device (ht_fill from host arrays) and its peak list
          and count come back into that step's own slot of pinned host memory
          (ht_find_maxima writing there); the calls are issued back to back
          over the same contexts and the host waits once, at the end.  The
          blocking per-call path (one context, ht_find_maxima into host
          memory, one round trip per event) is reported beside it with its
          latencies.
  roofline  the dominant kernel's algorithmic bytes / live launch time.
  cpu_baseline  the CPU oracle on a bounded sample of the same workload.

`--impl reference` times the CPU oracle (the reference arm) instead.
Under torchrun each rank runs its own events (independent replicas, weak
scaling); rank 0 prints max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1507_03074_gb300 import synth  # noqa: E402

WORKLOAD = "paper-scale event: 4990 hits (396 tracks + 238 noise), M_H 4x16x1024x1024 u32, threshold 10"
METRIC = "events/s"
N_POOL = 8              # distinct resident events cycled through the steps
THRESHOLD = 10
EVENTS_PER_STEP = 64    # one step = one group of events through the whole hot path
L2_NOTE = "inputs larger than L2: each event writes a 256 MiB M_H (L2 129 MB), read back at its candidates"


def bench_config(events_per_step):
    """The workload a line is measured on (the same dict in both arms)."""
    return {"workload": WORKLOAD, "events_per_step": events_per_step, "l2": L2_NOTE,
            "parallelism": "replicas (one per GPU, no collective)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--events-per-step", type=int, default=EVENTS_PER_STEP,
                    help="paper-scale events in one step (spread round-robin over the contexts)")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--naive", action="store_true", help="time the naive global-atomic fill")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and serving measurements")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--serving-seconds", type=float, default=1.5, help="arrival window per serving rate")
    ap.add_argument("--contexts", type=int, default=8, help="contexts (events in flight) of the timed steps")
    ap.add_argument("--tuning", default=None,
                    help="JSON launch shape (ht_tuning fields) for the timed steps, e.g. '{\"fill_vote_agg\": 1}'; "
                         "implies --no-autotune")
    ap.add_argument("--peaks-only", action="store_true",
                    help="time the peaks-only fills (HT_PEAKS_ONLY: M_H not written) in the headline steps")
    ap.add_argument("--components-only", action="store_true",
                    help="print only the component timings (two-kernel path, naive fill, L2 atomics), "
                         "--steps events each")
    a = ap.parse_args()
    if a.naive and a.peaks_only:
        ap.error("--naive and --peaks-only exclude each other")
    return a


# ---------------------------------------------------------------------------
# Distributed plumbing (replicas only; no collective on the data path)
# ---------------------------------------------------------------------------

def dist_init(n):
    """Rank and world size from the launcher's environment; one process per
    GPU over NCCL (gloo where no GPU is visible, e.g. the CPU reference arm)."""
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    if world > 1:
        import torch.distributed as dist
        import torch
        if torch.cuda.is_available():
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """The largest of every rank's v (the slowest replica's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_event_seeds(rank, n=None):
    """Seeds of a replica's resident events: disjoint across ranks."""
    n = N_POOL if n is None else n
    return [1 + rank * 1000 + k for k in range(n)]


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------

REASON_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
               0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
               0x100: "display_clock_setting"}


class ClockSampler:
    def __init__(self, index=0):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.samples = []
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            try:
                self.samples.append((float(parts[0]), float(parts[1]), float(parts[2]), int(parts[3], 16)))
            except Exception:
                pass

    def summary(self):
        s = getattr(self, "samples", [])
        if not s:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        busy = [x for x in s if not (x[3] & 0x1)] or s
        reasons = set()
        for x in busy:
            for bit, name in REASON_BITS.items():
                if x[3] & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(x[0] for x in busy), "sm_max_mhz": max(x[1] for x in s),
                "power_w_max": max(x[2] for x in s), "reasons": sorted(reasons), "samples": len(s)}


# ---------------------------------------------------------------------------
# Peaks and profile summaries
# ---------------------------------------------------------------------------

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def strip_comments(src):
    """C/CUDA source without its comments, trailing blanks and empty lines
    (the kernel sources hold no comment marker inside a string literal)."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.split("\n") if line.strip())


def kernel_source_hash():
    """Hash of the kernel sources' code (comments excluded), which keys the
    committed DRAM traffic figure to the kernels it was measured on."""
    h = hashlib.sha256()
    for f in ("ht_kernels.cu", "ht_device.cuh", "ht_internal.h"):
        with open(os.path.join(ROOT, "paper_1507_03074_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was captured from the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("kernel_source_hash") != kernel_source_hash():
        return None
    k = d.get("kernels", {}).get(kernel)
    return None if k is None else k.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------

def run_ours(args, rank, world):
    import torch
    from paper_1507_03074_gb300 import ht

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    events = [synth.paper_event(seed=sd) for sd in rank_event_seeds(rank)]
    max_hits = max(e.n_hits for e in events)
    ctx = ht.Context(b, r, threshold=THRESHOLD, max_hits=max_hits)
    st = torch.cuda.Stream()
    cap = 1 << 16
    dev = []
    with torch.cuda.stream(st):
        for e in events:
            dev.append(tuple(torch.from_numpy(a).cuda() for a in (e.x, e.y, e.z)))
        out = torch.empty(cap * 8, dtype=torch.int32, device="cuda")
        cnt = torch.empty(1, dtype=torch.int32, device="cuda")
        M = torch.empty(b.n_cells, dtype=torch.int32, device="cuda")
    st.synchronize()

    # votes per pool event (outside the timed region)
    votes, peaks, cands = [], [], []
    for k in range(N_POOL):
        ctx.fill(*dev[k], naive=args.naive, stream=st)
        ctx.find_maxima(capacity=cap, out=out, count=cnt, stream=st)
        ctx.matrix_into(M, stream=st)
        st.synchronize()
        votes.append(int(M.to(torch.int64).sum().item()))
        peaks.append(int(cnt.item()))
        cands.append(ctx.last_admitted() * b.n_a)
    ctx.sync()
    del M
    if args.components_only:
        res = None
        if rank == 0:
            res = {"components": run_components(dev, b, r, max_hits, float(np.mean(votes)), measured_peaks()[0],
                                                steps=args.steps)}
        ctx.close()
        return res
    # pick launch shapes on this workload (outside the timed region)
    if args.tuning:
        ctx.set_tuning(**json.loads(args.tuning))
    tuning = ctx.get_tuning() if args.no_autotune or args.tuning else ctx.autotune(reps=5)[0]

    # events in flight: one context (and stream) per event slot, round-robin
    C = max(1, args.contexts)
    E = max(1, args.events_per_step)
    ctxs = [ctx] + [ht.Context(b, r, threshold=THRESHOLD, max_hits=max_hits) for _ in range(C - 1)]
    for c in ctxs[1:]:
        c.set_tuning(**tuning)
    sts = [st] + [torch.cuda.Stream() for _ in range(C - 1)]
    with torch.cuda.stream(st):
        outs = [out] + [torch.empty(cap * 8, dtype=torch.int32, device="cuda") for _ in range(C - 1)]
        cnts = [cnt] + [torch.empty(1, dtype=torch.int32, device="cuda") for _ in range(C - 1)]
    st.synchronize()

    def event(i, count=None):
        """Event i of the run: context i % C, pool event i % N_POOL."""
        c = i % C
        ctxs[c].fill(*dev[i % N_POOL], naive=args.naive, peaks_only=args.peaks_only, stream=sts[c])
        ctxs[c].find_maxima(capacity=cap, out=outs[c], count=cnts[c] if count is None else count, stream=sts[c])

    def event1(i):
        ctx.fill(*dev[i % N_POOL], naive=args.naive, peaks_only=args.peaks_only, stream=st)
        ctx.find_maxima(capacity=cap, out=out, count=cnt, stream=st)

    # the launch shape of the events in flight (outside the timed region): the
    # single-event choice, or the same fill at one CTA per SM so that two
    # events' fills share every SM, whichever a short in-flight run finds faster
    tun_fl = tuning if args.no_autotune or C == 1 else pick_in_flight(ctxs, sts, event, tuning)
    for c in ctxs:
        c.set_tuning(**tun_fl)
    for i in range(max(args.warmup * E, C)):
        event(i)
    torch.cuda.synchronize()

    # ---- device-resident timed region --------------------------------------
    # The headline: K steps of E events each between two CUDA events on a
    # stream that forks to and joins the contexts' streams, nothing else
    # recorded in between (per-event marks and per-kernel events would sit
    # between the dependent launches).  Each event's peak count lands in its
    # own word.
    K = args.steps
    NE = K * E
    ev_counts = torch.full((NE,), -1, dtype=torch.int32, device="cuda")
    count_views = [ev_counts[i:i + 1] for i in range(NE)]
    main = torch.cuda.Stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        launches0 = sum(c.launches for c in ctxs)
        ev0.record(main)
        for s in sts:
            s.wait_stream(main)
        for i in range(NE):
            event(i, count_views[i])
        for s in sts:
            main.wait_stream(s)
        ev1.record(main)
        main.synchronize()
        launches = sum(c.launches for c in ctxs) - launches0
        torch.cuda.synchronize()
        got = ev_counts.cpu().numpy()
        steps_ok = all(int(got[i]) == peaks[i % N_POOL] for i in range(NE))
        barrier(world)
        # the same events with one context: one event at a time on one stream,
        # at the single-event launch shape
        ctx.set_tuning(**tuning)
        for i in range(args.warmup * E):
            event1(i)
        e1a, e1b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e1a.record(st)
            for i in range(NE):
                event1(i)
            e1b.record(st)
        st.synchronize()
        one_ms = e1a.elapsed_time(e1b)
        barrier(world)
        # per-event latency and per-kernel device times: one context again
        # with a CUDA event after every event and around every kernel
        NP = min(max(NE // 4, 400), 2000)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(NP + 1)]
        ctx.profile(True)
        with torch.cuda.stream(st):
            marks[0].record(st)
            for i in range(NP):
                event1(i)
                marks[i + 1].record(st)
        st.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
        torch.cuda.synchronize()
        barrier(world)
        # e2e, blocking: host buffers through the C ABI, one round trip per event
        NB = min(max(NE // 8, 400), 3000)
        host_cap = 4096
        e2e_times = []
        n_peaks_e2e = 0
        t0 = time.perf_counter()
        for i in range(NB):
            e = events[i % N_POOL]
            ts = time.perf_counter()
            ctx.fill(e.x, e.y, e.z)
            pk, n = ctx.find_maxima(capacity=host_cap)
            e2e_times.append(time.perf_counter() - ts)
            n_peaks_e2e += len(pk)
        e2e_s = time.perf_counter() - t0
        ctx.set_tuning(**tun_fl)
        # e2e, pipelined: the same calls over the contexts (each on its own
        # stream with its own pinned staging), at least as many events as the
        # headline and at least 400 or a quarter second's worth; each event's
        # count lands in its own word of pinned host memory and its peaks in a
        # ring of pinned slots; one wait at the end
        rate_est = NE / max(ev0.elapsed_time(ev1) / 1e3, 1e-9)
        N2 = max(NE, 400, int(0.25 * rate_est))
        slot_cap, ring = 1024, 256
        res_pk = torch.zeros((ring, slot_cap * 8), dtype=torch.int32, pin_memory=True)
        res_n = torch.zeros(N2, dtype=torch.int32, pin_memory=True)
        for c in ctxs:
            c.sync()
        t0 = time.perf_counter()
        for i in range(N2):
            e = events[i % N_POOL]
            c = ctxs[i % C]
            c.fill(e.x, e.y, e.z)
            c.find_maxima(capacity=slot_cap, out=res_pk[i % ring], count=res_n[i:i + 1])
        for c in ctxs:
            c.sync()
        e2e_pipe_s = time.perf_counter() - t0
        got_n = res_n.numpy().astype(np.int64)
        pipe_ok = all(int(got_n[i]) == peaks[i % N_POOL] for i in range(N2))
        n_peaks_pipe = int(np.minimum(got_n, slot_cap).sum())
    total_ms = ev0.elapsed_time(ev1)
    per_event = [marks[i].elapsed_time(marks[i + 1]) for i in range(NP)]

    t_dev = max_over_ranks(total_ms / 1e3, world)
    t_one = max_over_ranks(one_ms / 1e3, world)
    t_e2e = max_over_ranks(e2e_s, world)
    t_e2e_pipe = max_over_ranks(e2e_pipe_s, world)
    if rank != 0:
        for c in ctxs:
            c.close()
        return None

    kern = {kname: round(ms / n * 1e3, 2) for kname, (n, ms) in prof.items() if n}
    # dominant kernel: largest total device time
    dom = max(((kname, ms) for kname, (n, ms) in prof.items() if n), key=lambda t: t[1])[0]
    hbm_peak, peak_src = measured_peaks()
    cells_bytes = b.n_cells * 4
    algo = {"k_fill_priv": cells_bytes, "k_fill_scan": cells_bytes, "k_fill_ws": cells_bytes,
            "k_fill_bulk": cells_bytes, "k_fill_tma": cells_bytes, "k_scan": cells_bytes, "k_clear": cells_bytes}
    n_dom, ms_dom = prof[dom]
    avg_s = ms_dom / n_dom / 1e3
    value = NE * world / t_dev
    roofline = None
    if algo.get(dom):
        ach = algo[dom] / avg_s / 1e9
        roofline = {"kernel": dom, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak,
                    "unit": "GB/s", "frac": round(ach / hbm_peak, 4), "traffic": profiled_traffic(dom),
                    "algorithmic_bytes_per_launch": algo[dom], "avg_launch_us": round(avg_s * 1e6, 2),
                    "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs), burst",
                    "launch_time_from": "one-context pass, single-event launch shape",
                    "in_flight": {"gbs": round(algo[dom] * value / world / 1e9, 1),
                                  "frac": round(algo[dom] * value / world / 1e9 / hbm_peak, 4)}}
    mean_votes = float(np.mean(votes))

    res = {
        "metric": METRIC, "value": round(value, 2), "unit": "events/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(t_dev * 1e3 / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded helix events; the paper's dataset is not available)",
        "config": bench_config(E),
        "gpu_launches": int(launches),
        "results_checked": bool(steps_ok),
        "e2e": {"value": round(N2 * world / t_e2e_pipe, 2), "unit": "events/s", "events": N2,
                "h2d_bytes_per_step": int(E * 12 * np.mean([e.n_hits for e in events])),
                "d2h_bytes_per_step": int(E * (4 + 32 * n_peaks_pipe / N2)),
                "api": "ht_fill(host) + ht_find_maxima(pinned host out), round-robin over the contexts",
                "results_checked": bool(pipe_ok),
                "blocking_per_call": {"value": round(NB * world / t_e2e, 2), "events": NB,
                                      "p50_ms": round(float(np.percentile(e2e_times, 50)) * 1e3, 4),
                                      "p99_ms": round(float(np.percentile(e2e_times, 99)) * 1e3, 4)}},
        "roofline": roofline,
        "clocks": clk.summary(),
        "run": {"events_per_step": E, "contexts_in_flight": C, "in_flight_tuning": tun_fl, "tuning": tuning,
                "fill": "naive" if args.naive else "privatised", "peaks_only": bool(args.peaks_only),
                "arithmetic": "f32 vote arithmetic (IEEE round-to-nearest, no FMA), u32 vote counters"},
        "one_context": {"value": round(NE * world / t_one, 2), "us_per_event": round(t_one * 1e6 / NE, 2)},
        "gvotes_per_s": round(value * mean_votes / 1e9, 3),
        "gcandidates_per_s": round(value * float(np.mean(cands)) / 1e9, 3),
        "votes_per_event": int(mean_votes), "peaks_per_event": float(np.mean(peaks)),
        "latency_ms": {"device_p50": round(float(np.percentile(per_event, 50)), 4),
                       "device_p99": round(float(np.percentile(per_event, 99)), 4), "events": NP},
        "kernels_us": kern,
    }
    for c in ctxs:
        c.set_tuning(**tuning)
    n_x = min(max(NE, 400), 4000)     # events per timed extra
    if not args.no_extras and world == 1:
        res["peaks_only"] = run_peaks_only(ctxs, dev, outs, cnts, cap, sts, n_x, 2 * C, peaks)
        res["maxima_4d"] = run_maxima4d(ctxs, dev, outs, cnts, cap, sts, n_x, 2 * C)
        res["readout"] = run_readout(ctx, events, b, r)
        res["sectors"] = run_sectors(dev, b, r, max_hits, n_x // 4, 2 * C, peaks)
        res["upgrade"] = run_upgrade(hbm_peak)
        res["components"] = run_components(dev, b, r, max_hits, float(np.mean(votes)), hbm_peak)
    for c in ctxs:
        c.close()
    if not args.no_extras and world == 1:
        res["serving_peaks_only"] = run_serving(args.serving_seconds, rates=(10000, 50000), peaks_only=True,
                                                per_event=False)
        res["serving"] = run_serving(args.serving_seconds)
        res["batched"] = run_batched()
    if not args.no_cpu_baseline and world == 1:
        res["cpu_baseline"] = cpu_baseline(budget_s=10.0)
    return res


# ---------------------------------------------------------------------------
# The step's components against their own rooflines: the two-kernel path
# (privatised fill, then the standalone streaming scan) against HBM, and the
# paper's naive fill (one global atomic per vote) against measured L2 atomics
# ---------------------------------------------------------------------------
def run_components(dev, b, r, max_hits, mean_votes, hbm_peak, steps=200):
    import torch
    from paper_1507_03074_gb300 import ht

    st = torch.cuda.Stream()
    out = torch.empty(65536 * 8, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    cells_bytes = b.n_cells * 4

    def profile(tuning, naive):
        with ht.Context(b, r, threshold=THRESHOLD, max_hits=max_hits) as ctx:
            ctx.set_tuning(**tuning)
            for k in range(10):
                ctx.fill(*dev[k % N_POOL], naive=naive, stream=st)
                ctx.find_maxima(capacity=65536, out=out, count=cnt, stream=st)
            st.synchronize()
            ctx.profile(True)
            for k in range(steps):
                ctx.fill(*dev[k % N_POOL], naive=naive, stream=st)
                ctx.find_maxima(capacity=65536, out=out, count=cnt, stream=st)
            p = ctx.profile_read()
            ctx.profile(False)
        return {kn: t / n * 1e3 for kn, (n, t) in p.items() if n}

    def naive_alone(reps=4 * N_POOL):
        # the naive fill with the L2 holding only clean lines when it starts,
        # as under ncu's cache flush: an empty fill clears M_H, a 512 MiB read
        # writes back the dirty lines the clear left, then the event is
        # accumulated into the zeroed matrix (no clear of its own)
        flush = torch.empty(128 << 20, dtype=torch.float32, device="cuda")
        empty = torch.empty(0, dtype=torch.float32, device="cuda")
        total_ms = 0.0
        with ht.Context(b, r, threshold=THRESHOLD, max_hits=max_hits) as ctx:
            for k in range(reps + 2):
                ctx.fill(empty, empty, empty, naive=True, stream=st)
                with torch.cuda.stream(st):
                    flush.sum()
                ctx.profile(True)
                ctx.fill(*dev[k % N_POOL], naive=True, accumulate=True, stream=st)
                n, t = ctx.profile_read()["k_fill_naive"]
                ctx.profile(False)
                if k >= 2:
                    total_ms += t / n
        return total_ms / reps * 1e3

    def scan_alone(reps=4 * N_POOL):
        # the standalone scan with the L2 holding only clean lines when it
        # starts: a 512 MiB read between the fill and the scan writes back the
        # rows of M_H the fill left dirty (as ncu's cache flush does)
        flush = torch.empty(128 << 20, dtype=torch.float32, device="cuda")
        with ht.Context(b, r, threshold=THRESHOLD, max_hits=max_hits) as ctx:
            ctx.set_tuning(fill_fused_scan=2)
            ctx.profile(True)
            for k in range(reps + 2):
                ctx.fill(*dev[k % N_POOL], stream=st)
                with torch.cuda.stream(st):
                    flush.sum()
                ctx.find_maxima(capacity=65536, out=out, count=cnt, stream=st)
            p = ctx.profile_read()
            ctx.profile(False)
        n, t = p["k_scan"]
        return t / n * 1e3

    two = profile({"fill_fused_scan": 2}, False)
    naive = profile({"fill_fused_scan": 2}, True)
    alone_us = naive_alone()
    scan_alone_us = scan_alone()
    l2_res = ht.measure_atomics(32 << 20)
    l2_hbm = ht.measure_atomics(256 << 20)
    fill_us, scan_us = two.get("k_fill_priv"), two.get("k_scan")
    nv_us = naive.get("k_fill_naive")
    return {
        "fill_priv": {"avg_us": round(fill_us, 2), "gbs_written": round(cells_bytes / fill_us / 1e3, 1),
                      "frac_of_hbm": round(cells_bytes / fill_us / 1e3 / hbm_peak, 4)},
        "scan_stream": {"avg_us": round(scan_us, 2), "gbs_read": round(cells_bytes / scan_us / 1e3, 1),
                        "frac_of_hbm": round(cells_bytes / scan_us / 1e3 / hbm_peak, 4),
                        "alone": {"avg_us": round(scan_alone_us, 2),
                                  "gbs_read": round(cells_bytes / scan_alone_us / 1e3, 1),
                                  "frac_of_hbm": round(cells_bytes / scan_alone_us / 1e3 / hbm_peak, 4),
                                  "l2_before": "clean (a 512 MiB read wrote back the fill's dirty lines)"}},
        "fill_naive": {"avg_us": round(nv_us, 2), "clear_us": round(naive.get("k_clear", 0.0), 2),
                       "gvotes_per_s": round(mean_votes / nv_us / 1e3, 3),
                       "frac_of_l2_atomics_32mib": round(mean_votes / nv_us * 1e6 / l2_res, 4),
                       "frac_of_l2_atomics_256mib": round(mean_votes / nv_us * 1e6 / l2_hbm, 4),
                       "alone": {"avg_us": round(alone_us, 2), "gvotes_per_s": round(mean_votes / alone_us / 1e3, 3),
                                 "frac_of_l2_atomics_32mib": round(mean_votes / alone_us * 1e6 / l2_res, 4),
                                 "l2_before": "clean (a 512 MiB read wrote back the clear's dirty lines)"}},
        "l2_atomics": {"gupdates_per_s_32mib": round(l2_res / 1e9, 2), "gupdates_per_s_256mib": round(l2_hbm / 1e9, 2)},
    }


# ---------------------------------------------------------------------------
# High-occupancy upgrade-like events: 50 000 hits, M_H 8x32x2048x2048 u32 (4 GiB)
# ---------------------------------------------------------------------------
def run_upgrade(hbm_peak, n_events=4, steps=20):
    import torch
    from paper_1507_03074_gb300 import ht

    b, r = ht.Binning(*synth.UPGRADE_BINNING), ht.Ranges()
    evs = [synth.upgrade_event(i) for i in range(n_events)]
    st = torch.cuda.Stream()
    out = torch.empty(65536 * 8, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    with ht.Context(b, r, threshold=THRESHOLD, max_hits=max(e.n_hits for e in evs)) as ctx:
        dev = [tuple(torch.from_numpy(a).cuda() for a in (e.x, e.y, e.z)) for e in evs]

        def step(k):
            ctx.fill(*dev[k % n_events], stream=st)
            ctx.find_maxima(capacity=65536, out=out, count=cnt, stream=st)

        for k in range(3):
            step(k)
        st.synchronize()
        a, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            a.record(st)
            for k in range(steps):
                step(k)
            e_.record(st)
        st.synchronize()
        ms = a.elapsed_time(e_) / steps
        ctx.profile(True)
        for k in range(4):
            step(k)
        prof = ctx.profile_read()
        ctx.profile(False)
        # two events in flight: a second context (another 4 GiB M_H) on its own
        # stream, the events alternating between them
        with ht.Context(b, r, threshold=THRESHOLD, max_hits=max(e.n_hits for e in evs)) as ctx2:
            ctx2.set_tuning(**ctx.get_tuning())
            ctxs, sts = (ctx, ctx2), (st, torch.cuda.Stream())
            outs = (out, torch.empty_like(out))
            cnts = (cnt, torch.empty_like(cnt))

            def step2(k):
                c = k % 2
                ctxs[c].fill(*dev[k % n_events], stream=sts[c])
                ctxs[c].find_maxima(capacity=65536, out=outs[c], count=cnts[c], stream=sts[c])

            ms2 = timed_in_flight(sts, step2, steps, 4)
    kern = {kn: t / n * 1e3 for kn, (n, t) in prof.items() if n}
    fill_us = kern.get("k_fill_tma", kern.get("k_fill_scan"))
    cells_bytes = b.n_cells * 4
    return {"workload": "50 000 hits, M_H 8x32x2048x2048 u32 (4 GiB)",
            "events_per_s": round(1e3 / ms, 2), "ms_per_event": round(ms, 4),
            "kernels_us": {kn: round(v, 1) for kn, v in kern.items()},
            "fill_gbs": round(cells_bytes / fill_us / 1e3, 1) if fill_us else None,
            "fill_frac_of_hbm": round(cells_bytes / fill_us / 1e3 / hbm_peak, 4) if fill_us else None,
            "in_flight": {"contexts": 2, "events_per_s": round(1e3 / ms2, 2), "ms_per_event": round(ms2, 4),
                          "m_h_gbs": round(cells_bytes / ms2 / 1e6, 1),
                          "frac_of_hbm": round(cells_bytes / ms2 / 1e6 / hbm_peak, 4)}}


# ---------------------------------------------------------------------------
# Phi sectors (Sec. 4): four sector contexts on their own streams, merged
# ---------------------------------------------------------------------------
def run_sectors(dev, b, r, max_hits, K, W, peaks_ref, n_sectors=4):
    import torch
    from paper_1507_03074_gb300 import ht

    st = torch.cuda.Stream()
    cap = 1 << 16
    out = torch.empty(cap * 8, dtype=torch.int32, device="cuda")
    cnt = torch.empty(1, dtype=torch.int32, device="cuda")
    with ht.Sectors(b, r, threshold=THRESHOLD, n_sectors=n_sectors, max_hits=max_hits) as sec:
        def step(k):
            sec.fill(*dev[k % N_POOL], stream=st)
            sec.find_maxima(capacity=cap, out=out, count=cnt, stream=st)

        same = True
        for k in range(N_POOL):
            step(k)
            st.synchronize()
            same = same and int(cnt.item()) == peaks_ref[k]
        for k in range(W):
            step(k)
        st.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            ev0.record(st)
            for k in range(K):
                step(k)
            ev1.record(st)
        st.synchronize()
        ms = ev0.elapsed_time(ev1) / K
    return {"n_sectors": n_sectors, "events_per_s": round(1e3 / ms, 1), "ms_per_step": round(ms, 4),
            "same_peak_counts": bool(same)}


# ---------------------------------------------------------------------------
# The 4-D (80-neighbour) maxima rule: the 2-D pipeline plus the k_peaks4d filter
# ---------------------------------------------------------------------------
def timed_in_flight(sts, step, K, W):
    """Milliseconds per step of K steps (after W) issued by step(k) onto the
    streams sts, between two CUDA events on a stream that forks to and joins
    all of them."""
    import torch

    for k in range(W):
        step(k)
    torch.cuda.synchronize()
    main = torch.cuda.Stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(main)
    for s in sts:
        s.wait_stream(main)
    for k in range(K):
        step(k)
    for s in sts:
        main.wait_stream(s)
    ev1.record(main)
    main.synchronize()
    return ev0.elapsed_time(ev1) / K


def pick_in_flight(ctxs, sts, step, tuning, n=600):
    """The faster, over n in-flight steps, of the single-event launch shape and
    the same shape with one fill CTA per SM (two events' fills then share each
    SM), the binning launches left to the library's choice for each shape;
    leaves the contexts at the choice and returns it as they report it."""
    cands = [dict(tuning, bin_cluster=0), dict(tuning, fill_blocks_per_sm=1, bin_cluster=0)]
    best, best_ms = cands[0], None
    for t in cands:
        for c in ctxs:
            c.set_tuning(**t)
        ms = timed_in_flight(sts, step, n, len(ctxs))
        if best_ms is None or ms < best_ms:
            best, best_ms = t, ms
    for c in ctxs:
        c.set_tuning(**best)
    return ctxs[0].get_tuning()


def run_maxima4d(ctxs, dev, outs, cnts, cap, sts, K, W):
    C = len(ctxs)

    def run_on(c, k):
        ctxs[c].fill(*dev[k % N_POOL], stream=sts[c])
        ctxs[c].find_maxima(capacity=cap, out=outs[c], count=cnts[c], stream=sts[c], four_d=True)

    def step(k):
        run_on(k % C, k)

    ctx, st = ctxs[0], sts[0]
    n4 = []
    for k in range(N_POOL):
        ctx.fill(*dev[k], stream=st)
        ctx.find_maxima(capacity=cap, out=outs[0], count=cnts[0], stream=st, four_d=True)
        st.synchronize()
        n4.append(int(cnts[0].item()))
    tun = ctx.get_tuning()
    tun_fl = pick_in_flight(ctxs, sts, step, tun)
    ms = timed_in_flight(sts, step, K, W)
    for c in ctxs:
        c.set_tuning(**tun)
    ms1 = timed_in_flight(sts[:1], lambda k: run_on(0, k), K, W)
    ctx.profile(True)
    for k in range(max(1, K // 4)):
        run_on(0, k)
    prof = ctx.profile_read()
    ctx.profile(False)
    return {"events_per_s": round(1e3 / ms, 1), "one_context_events_per_s": round(1e3 / ms1, 1),
            "in_flight_blocks_per_sm": tun_fl.get("fill_blocks_per_sm"), "peaks_per_event": float(np.mean(n4)),
            "kernels_us": {kn: round(t / n * 1e3, 2) for kn, (n, t) in prof.items() if n}}


# ---------------------------------------------------------------------------
# Track read-out of the pool events' peaks against the generator's truth
# ---------------------------------------------------------------------------
def run_readout(ctx, events, b, r):
    from paper_1507_03074_gb300 import ht, readout

    per = []
    for e in events:
        ctx.fill(e.x, e.y, e.z)
        pk, _ = ctx.find_maxima(capacity=1 << 16)
        per.append(readout.match(ht.track_params(b, r, pk, synth.B_FIELD_T), e, b, r))
    return readout.summarise(per)


# ---------------------------------------------------------------------------
# Peaks-only fills (M_H not written), the same resident events
# ---------------------------------------------------------------------------
def run_peaks_only(ctxs, dev, outs, cnts, cap, sts, K, W, peaks_ref):
    C = len(ctxs)

    def run_on(c, k):
        ctxs[c].fill(*dev[k % N_POOL], peaks_only=True, stream=sts[c])
        ctxs[c].find_maxima(capacity=cap, out=outs[c], count=cnts[c], stream=sts[c])

    def step(k):
        run_on(k % C, k)

    ctx, st = ctxs[0], sts[0]
    same = True
    for k in range(N_POOL):          # the peak counts of the plain path
        ctx.fill(*dev[k], peaks_only=True, stream=st)
        ctx.find_maxima(capacity=cap, out=outs[0], count=cnts[0], stream=st)
        st.synchronize()
        same = same and int(cnts[0].item()) == peaks_ref[k]
    tun = ctx.get_tuning()
    tun_fl = pick_in_flight(ctxs, sts, step, tun)
    ms = timed_in_flight(sts, step, K, W)
    for c in ctxs:
        c.set_tuning(**tun)
    ms1 = timed_in_flight(sts[:1], lambda k: run_on(0, k), K, W)
    ctx.profile(True)
    for k in range(max(1, K // 4)):
        run_on(0, k)
    prof = ctx.profile_read()
    ctx.profile(False)
    return {"events_per_s": round(1e3 / ms, 1), "one_context_events_per_s": round(1e3 / ms1, 1),
            "in_flight_blocks_per_sm": tun_fl.get("fill_blocks_per_sm"), "same_peak_counts": bool(same),
            "kernels_us": {kn: round(t / n * 1e3, 2) for kn, (n, t) in prof.items() if n}}


# ---------------------------------------------------------------------------
# Batched vs per-event (100 uneven events) and the serving stream
# ---------------------------------------------------------------------------

def _pct(v, q):
    return round(float(np.percentile(v, q)), 4)


def run_batched(n_events=100, reps=5):
    """100 independent events, hit counts uniform in 500..5000 (seeds 1000+i),
    binning 4x16x1024x1024, threshold 10: one batch launch sequence (graph
    replay) against the same events one per launch sequence."""
    import torch
    from paper_1507_03074_gb300 import ht
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    evs = synth.batch_events(n_events, seed0=1000)
    x, y, z, off = ht.Batch.concat([(e.x, e.y, e.z) for e in evs])
    # the hits in page-locked host memory, where the end-to-end runs copy
    # them from; every event is a view of them
    pinned = [torch.empty(v.size, dtype=torch.float32, pin_memory=True) for v in (x, y, z)]
    for t, v in zip(pinned, (x, y, z)):
        t.numpy()[:] = v
    x, y, z = (t.numpy() for t in pinned)
    host = [tuple(v[off[e]:off[e + 1]] for v in (x, y, z)) for e in range(n_events)]
    n_hits = int(off[-1])
    st = torch.cuda.Stream()
    res = {"workload": f"{n_events} events, hits U(500..5000), 4x16x1024x1024; e2e inputs in page-locked host memory"}
    # per event, through a context
    with ht.Context(b, r, threshold=THRESHOLD, max_hits=max(e.n_hits for e in evs)) as ctx:
        M = torch.empty(b.n_cells, dtype=torch.int32, device="cuda")
        votes = 0
        dev = [tuple(torch.from_numpy(a).cuda() for a in ev) for ev in host]
        out = torch.empty(4096 * 8, dtype=torch.int32, device="cuda")
        cnt = torch.empty(1, dtype=torch.int32, device="cuda")
        for d in dev:
            ctx.fill(*d, stream=st)
            ctx.matrix_into(M, stream=st)
            st.synchronize()
            votes += int(M.to(torch.int64).sum().item())
        del M
        for ev in host[:10]:
            ctx.fill(*ev)
            ctx.find_maxima(capacity=4096)
        lat = []
        t0 = time.perf_counter()
        for ev in host:
            ts = time.perf_counter()
            ctx.fill(*ev)
            ctx.find_maxima(capacity=4096)
            lat.append((time.perf_counter() - ts) * 1e3)
        t_host = time.perf_counter() - t0
        a, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for d in dev[:10]:
            ctx.fill(*d, stream=st)
            ctx.find_maxima(capacity=4096, out=out, count=cnt, stream=st)
        a.record(st)
        for d in dev:
            ctx.fill(*d, stream=st)
            ctx.find_maxima(capacity=4096, out=out, count=cnt, stream=st)
        e_.record(st)
        st.synchronize()
        t_dev = a.elapsed_time(e_) / 1e3
    res["per_event"] = {"e2e": round(n_events / t_host, 1), "device": round(n_events / t_dev, 1),
                        "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99)}
    # the same per-event calls with events in flight: 8 contexts, each on its
    # own stream, the events round-robin
    C = 8
    ctxs = [ht.Context(b, r, threshold=THRESHOLD, max_hits=max(e.n_hits for e in evs)) for _ in range(C)]
    sts = [torch.cuda.Stream() for _ in range(C)]
    outs = [torch.empty(4096 * 8, dtype=torch.int32, device="cuda") for _ in range(C)]
    cnts = [torch.empty(1, dtype=torch.int32, device="cuda") for _ in range(C)]

    def step(k):
        c = k % C
        ctxs[c].fill(*dev[k % n_events], stream=sts[c])
        ctxs[c].find_maxima(capacity=4096, out=outs[c], count=cnts[c], stream=sts[c])

    tun_fl = pick_in_flight(ctxs, sts, step, ctxs[0].get_tuning(), n=200)
    ms_fl = timed_in_flight(sts, step, n_events * reps, 2 * C)
    slot = 1024
    res_pk = torch.zeros((n_events, slot * 8), dtype=torch.int32, pin_memory=True)
    res_n = torch.zeros(n_events, dtype=torch.int32, pin_memory=True)
    t_fl = []
    for _ in range(reps):
        for c in ctxs:
            c.sync()
        t0 = time.perf_counter()
        for k, ev in enumerate(host):
            c = ctxs[k % C]
            c.fill(*ev)
            c.find_maxima(capacity=slot, out=res_pk[k], count=res_n[k:k + 1])
        for c in ctxs:
            c.sync()
        t_fl.append(time.perf_counter() - t0)
    counts_fl = res_n.numpy().copy()
    for c in ctxs:
        c.close()
    res["per_event_in_flight"] = {"e2e": round(n_events / float(np.median(t_fl)), 1),
                                  "device": round(1e3 / ms_fl, 1), "contexts": C,
                                  "blocks_per_sm": tun_fl.get("fill_blocks_per_sm"),
                                  "all_100_ms": round(float(np.median(t_fl)) * 1e3, 3)}
    # one batch
    with ht.Batch(b, r, threshold=THRESHOLD, max_events=n_events, max_hits=n_hits + 64, capacity=1 << 17) as B:
        for _ in range(2):
            B.run(x, y, z, off)
        tuning, _ = B.autotune(reps=2)
        for _ in range(2):
            B.run(x, y, z, off)
        lat_b = []
        for _ in range(reps):
            ts = time.perf_counter()
            pk, counts = B.run(x, y, z, off)
            lat_b.append((time.perf_counter() - ts) * 1e3)
        dx, dy, dz = (torch.from_numpy(v).cuda() for v in (x, y, z))
        doff = torch.from_numpy(off.astype(np.int32)).cuda()
        bout = torch.empty((1 << 17) * 8, dtype=torch.int32, device="cuda")
        bcnt = torch.empty(n_events, dtype=torch.int32, device="cuda")
        for _ in range(2):
            B.run_device(dx, dy, dz, doff, n_hits, bout, bcnt, stream=st)
        a.record(st)
        for _ in range(reps):
            B.run_device(dx, dy, dz, doff, n_hits, bout, bcnt, stream=st)
        e_.record(st)
        st.synchronize()
        t_bdev = a.elapsed_time(e_) / 1e3 / reps
        # the same batch with peaks-only fills (the matrices not written)
        pk_po, counts_po = B.run(x, y, z, off, peaks_only=True)
        same_po = bool(np.array_equal(counts_po, counts))
        lat_po = []
        for _ in range(reps):
            ts = time.perf_counter()
            B.run(x, y, z, off, peaks_only=True)
            lat_po.append((time.perf_counter() - ts) * 1e3)
        for _ in range(2):
            B.run_device(dx, dy, dz, doff, n_hits, bout, bcnt, stream=st, peaks_only=True)
        a.record(st)
        for _ in range(reps):
            B.run_device(dx, dy, dz, doff, n_hits, bout, bcnt, stream=st, peaks_only=True)
        e_.record(st)
        st.synchronize()
        t_podev = a.elapsed_time(e_) / 1e3 / reps
        B.profile(True)
        B.run(x, y, z, off)
        prof = B.profile_read()
        B.profile(False)
    t_b = float(np.median(lat_b)) / 1e3
    res["batch"] = {"e2e": round(n_events / t_b, 1), "device": round(n_events / t_bdev, 1),
                    "gvotes_per_s": round(votes / t_bdev / 1e9, 3), "p50_ms": _pct(lat_b, 50),
                    "p99_ms": _pct(lat_b, 99), "tuning": tuning,
                    "kernels_us": {k: round(ms / n * 1e3, 1) for k, (n, ms) in prof.items() if n}}
    res["batch_peaks_only"] = {"e2e": round(n_events / (float(np.median(lat_po)) / 1e3), 1),
                               "device": round(n_events / t_podev, 1), "same_counts": same_po}
    res["per_event_in_flight"]["same_counts"] = bool(np.array_equal(counts_fl, counts))
    res["unit"] = "events/s (e2e: host buffers, copies included; device: inputs resident)"
    return res


def run_serving(seconds=1.5, rates=(1000, 10000, 50000), pool_per_kind=48, warmup_s=1.0, peaks_only=False,
                per_event=True, fill_blocks_per_sm=0):
    """Poisson arrivals at each rate for `seconds`; hit counts lognormal
    (median 3000, sigma 1, clipped 200..50000); 90% binning 4x16x1024x1024,
    10% 8x32x2048x2048; threshold 10.  Requests reuse a pool of seeded events
    with the stream's first hit counts.  Latency is the server's own
    submit-to-ready time; the sustained rate counts completions over the
    time from the first submit to the last completion.  Each rate runs 1 s of
    its own stream (another seed) first, unmeasured."""
    import ctypes
    import queue
    import threading
    from paper_1507_03074_gb300 import ht
    bins = {False: ht.Binning(*synth.PAPER_BINNING), True: ht.Binning(*synth.UPGRADE_BINNING)}
    r = ht.Ranges()
    _, n0, up0, _ = synth.serving_stream(1000.0, 4 * pool_per_kind, seed=3000)
    pools = {False: [], True: []}
    for k in range(len(n0)):
        kind = bool(up0[k])
        if len(pools[kind]) < (pool_per_kind if not kind else pool_per_kind // 4):
            t, nz = synth.split_hits(int(n0[k]))
            e = synth.make_event(t, nz, seed=3000 + k)
            pools[kind].append((e.x, e.y, e.z))
    L = ht.lib()
    sys.setswitchinterval(1e-4)          # let the polling thread run beside the arrival loop
    out = {"workload": "Poisson; hits lognormal(3000, 1) in 200..50000; 90% 4x16x1024^2 / 10% 8x32x2048^2",
           "rates": []}
    if fill_blocks_per_sm:
        out["fill_blocks_per_sm"] = fill_blocks_per_sm
    with ht.Server(peaks_only=peaks_only, fill_blocks_per_sm=fill_blocks_per_sm) as S:
        # warm-up: lanes of both binnings
        warm = [S.submit(bins[k], r, THRESHOLD, *pools[k][i]) for k in (False, True) for i in range(4)]
        for t in warm:
            S.poll(t, timeout_us=60_000_000)
        S.stats(reset=True)
        for rate in rates:
            n = max(1, int(rate * seconds))
            # 1 s of the same kind of stream first (not measured): the lanes and
            # captured graphs the rate needs are made before the timed arrivals
            warm_n = min(max(1, int(rate * warmup_s)), 10000)
            w_arr, _, w_up, _ = synth.serving_stream(float(rate), warm_n, seed=3002)
            w_t = []
            t0 = time.perf_counter()
            for i in range(warm_n):
                while time.perf_counter() - t0 < w_arr[i]:
                    pass
                kind = bool(w_up[i])
                try:
                    w_t.append(S.submit(bins[kind], r, THRESHOLD, *pools[kind][i % len(pools[kind])]))
                except ht.HTError:
                    pass
            for t in w_t:
                S.poll(t, timeout_us=60_000_000)
            S.stats(reset=True)
            arr, _, up, _ = synth.serving_stream(float(rate), n, seed=3001)
            tickets = queue.Queue()
            done_t = [0.0]

            def poller():
                buf = np.zeros(4096, ht.PEAK_DTYPE)
                nf = ctypes.c_uint32()
                while True:
                    t = tickets.get()
                    if t is None:
                        break
                    L.ht_poll(S._h, t, buf.ctypes.data_as(ctypes.c_void_p), 4096, ctypes.byref(nf), 60_000_000)
                    done_t[0] = time.perf_counter()

            th = threading.Thread(target=poller)
            th.start()
            busy = 0
            t0 = time.perf_counter()
            for i in range(n):
                while time.perf_counter() - t0 < arr[i]:
                    pass
                kind = bool(up[i])
                ev = pools[kind][i % len(pools[kind])]
                try:
                    tickets.put(S.submit(bins[kind], r, THRESHOLD, *ev))
                except ht.HTError:
                    busy += 1
            t_sub = time.perf_counter() - t0
            tickets.put(None)
            th.join()
            span = done_t[0] - t0
            st = S.stats(reset=True)
            out["rates"].append({
                "offered": rate, "sustained": round((n - busy) / span, 1), "refused_busy": busy,
                "p50_ms": round(st["p50_us"] / 1e3, 4), "p99_ms": round(st["p99_us"] / 1e3, 4),
                "max_ms": round(st["max_us"] / 1e3, 4), "mean_batch": round(st["mean_batch"], 2),
                "lanes": st["lanes"]})
    if not per_event:
        return out
    # the plain per-event path on the same streams: one context per binning,
    # each arrival filled and scanned on its own (blocking), in arrival order;
    # latency = completion - arrival (queueing included)
    out["per_event_path"] = []
    max_hits = max(len(ev[0]) for k in pools for ev in pools[k])
    with ht.Context(bins[False], r, threshold=THRESHOLD, max_hits=max_hits) as c0, \
            ht.Context(bins[True], r, threshold=THRESHOLD, max_hits=max_hits) as c1:
        ctxs = {False: c0, True: c1}
        for k in (False, True):
            for ev in pools[k][:3]:
                ctxs[k].fill(*ev)
                ctxs[k].find_maxima(capacity=4096)
        for rate in rates:
            n = min(max(1, int(rate * seconds)), 3000)
            arr, _, up, _ = synth.serving_stream(float(rate), n, seed=3001)
            lat = []
            t0 = time.perf_counter()
            for i in range(n):
                while time.perf_counter() - t0 < arr[i]:
                    pass
                kind = bool(up[i])
                ev = pools[kind][i % len(pools[kind])]
                ctxs[kind].fill(*ev)
                ctxs[kind].find_maxima(capacity=4096)
                lat.append((time.perf_counter() - t0 - arr[i]) * 1e3)
            span = time.perf_counter() - t0
            out["per_event_path"].append({
                "offered": rate, "requests": n, "sustained": round(n / span, 1),
                "p50_ms": _pct(lat, 50), "p99_ms": _pct(lat, 99), "max_ms": round(max(lat), 4)})
    return out


def _oracle_event(ob, orr, e):
    import oracle
    M, votes = oracle.fill(ob, orr, e.x, e.y, e.z)
    pk, n = oracle.find_maxima(ob, orr, M, THRESHOLD)
    return votes, n


def _oracle_worker(job):
    """One host process of the all-cores baseline: whole events until the
    budget has run out; returns (events done, seconds)."""
    wid, budget_s = job
    import oracle
    ob, orr = oracle.Binning(*synth.PAPER_BINNING), oracle.Ranges()
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        _oracle_event(ob, orr, synth.paper_event(seed=6000 + 1000 * wid + n))
        n += 1
    return n, time.perf_counter() - t0


def cpu_baseline(budget_s=10.0):
    """The oracle as it stands, single-threaded, on whole paper-scale events
    until budget_s of CPU work has run; then one oracle process per host core
    (a spawned pool: this process has used the GPU), each on its own events,
    for the same budget."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    import oracle
    ob, orr = oracle.Binning(*synth.PAPER_BINNING), oracle.Ranges()
    n, t0 = 0, time.perf_counter()
    while True:
        e = synth.paper_event(seed=5000 + n)
        _oracle_event(ob, orr, e)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    res = {"value": round(n / dt, 4), "unit": "events/s", "cores": 1, "kind": "oracle",
           "sample": f"{n} whole paper-scale events (fill + maxima), single thread, {dt:.1f} s"}
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    if cores > 1:
        t0 = time.perf_counter()
        pool = ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn"))
        try:
            futs = [pool.submit(_oracle_worker, (w, budget_s)) for w in range(cores)]
            done = [f.result(timeout=3 * budget_s + 120) for f in futs]
        except Exception as ex:   # a worker that could not start or finish: no all-cores number
            pool.shutdown(wait=False, cancel_futures=True)
            res["all_cores"] = {"unavailable": f"{type(ex).__name__}: {ex}"}
            return res
        pool.shutdown()
        wall = time.perf_counter() - t0
        n_all = sum(d[0] for d in done)
        span = max(d[1] for d in done)
        res["all_cores"] = {"value": round(n_all / span, 4), "unit": "events/s", "cores": cores, "kind": "oracle",
                            "sample": f"{n_all} whole paper-scale events over {cores} processes (one per core, "
                                      f"independent events), {span:.1f} s each, {wall:.1f} s with start-up"}
    return res


# ---------------------------------------------------------------------------
# Reference arm: the CPU oracle, bounded samples per step
# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    """The reference arm: the CPU oracle as it stands, single-threaded, on
    whole paper-scale events (fill + maxima, the program cpu_baseline times).
    A step of our arm is events_per_step events; here each step is a bounded
    sample of that step (whole events until the step's time share has run),
    so that --steps K --warmup W ends within a few minutes."""
    import oracle
    if rank != 0:
        return None
    ob, orr = oracle.Binning(*synth.PAPER_BINNING), oracle.Ranges()
    E = max(1, args.events_per_step)
    n_ev = [0]

    def one_event():
        _oracle_event(ob, orr, synth.paper_event(seed=5000 + n_ev[0]))
        n_ev[0] += 1

    t = time.perf_counter()
    one_event()
    t_event = max(time.perf_counter() - t, 1e-4)
    budget_per_step = min(2.0, 150.0 / max(1, args.steps + args.warmup))
    per = int(min(E, max(1, round(budget_per_step / t_event))))
    for _ in range(args.warmup):
        for _ in range(per):
            one_event()
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        for _ in range(per):
            one_event()
            done += 1
    dt = time.perf_counter() - t0
    value = done / dt
    return {"metric": METRIC, "value": round(value, 4), "unit": "events/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3 / args.steps * E / per, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "impl": "reference",
            "dtype": "f32", "data": "synthetic (seeded helix events; the paper's dataset is not available)",
            "config": bench_config(E),
            "cpu_baseline": {"value": round(value, 4), "unit": "events/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per} of the {E} whole paper-scale events (fill + maxima) of each step, "
                                       f"{done} events in {dt:.1f} s; ms_per_step scaled to {E} events"},
            "e2e": {"value": round(value, 4), "unit": "events/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world = dist_init(args.gpus)
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
