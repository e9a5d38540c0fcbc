"""Host-side parts of bench.py on CPU: its flags and the CPU baseline (the
oracle single-threaded and as one spawned process per core)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_flags():
    import bench
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
        assert (a.gpus, a.contexts, a.impl, a.peaks_only, a.components_only) == (1, 8, "ours", False, False)
        sys.argv = ["bench.py", "--contexts", "3", "--peaks-only", "--steps", "7", "--warmup", "3"]
        a = bench.parse()
        assert (a.contexts, a.peaks_only, a.steps, a.warmup) == (3, True, 7, 3)
    finally:
        sys.argv = argv
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--naive", "--peaks-only"],
                       capture_output=True, text=True, cwd=ROOT, timeout=120)
    assert r.returncode != 0 and "exclude each other" in r.stderr


def test_cpu_baseline_single_and_all_cores():
    import bench
    res = bench.cpu_baseline(budget_s=0.3)
    assert res["kind"] == "oracle" and res["cores"] == 1 and res["value"] > 0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    if cores > 1:
        ac = res["all_cores"]
        assert "unavailable" not in ac, ac
        assert ac["cores"] == cores and ac["value"] > res["value"]


def test_pick_in_flight_keeps_the_faster_shape(monkeypatch):
    import bench

    class FakeCtx:
        def __init__(self):
            self.t = None

        def set_tuning(self, **t):
            self.t = dict(t)

        def get_tuning(self):
            # the library resolves bin_cluster 0: two launches when the fill
            # is held below its CTAs per SM, one cluster launch otherwise
            t = dict(self.t)
            if t.get("bin_cluster", 0) == 0:
                t["bin_cluster"] = 2 if t["fill_blocks_per_sm"] == 1 else 1
            return t

    ctxs = [FakeCtx() for _ in range(4)]
    base = {"fill_rows": 32, "fill_blocks_per_sm": 2}
    for one_cta_faster in (True, False):
        def fake_timed(sts, step, n, w):
            bps = ctxs[0].t["fill_blocks_per_sm"]
            assert all(c.t == ctxs[0].t for c in ctxs)      # every context runs the candidate
            return (40.0 if bps == 1 else 50.0) if one_cta_faster else (60.0 if bps == 1 else 50.0)
        monkeypatch.setattr(bench, "timed_in_flight", fake_timed)
        best = bench.pick_in_flight(ctxs, [None] * 4, lambda k: None, base)
        assert best["fill_blocks_per_sm"] == (1 if one_cta_faster else 2)
        assert all(c.get_tuning() == best for c in ctxs)   # the contexts stay at the choice
        assert all(c.t["bin_cluster"] == 0 for c in ctxs)   # binning left to the library per shape
        assert best["bin_cluster"] == (2 if one_cta_faster else 1)
        assert best["fill_rows"] == 32


def test_kernel_source_hash_ignores_comments_only():
    """The hash that keys the committed DRAM traffic figure follows the
    kernels' code: comment and blank-line edits keep it, a code edit changes
    it, and the figure is reported only for the kernels it was taken on."""
    import bench

    code = "__global__ void k(int *p)\n{\n    p[0] = 1;   // one\n}\n"
    same = "// header\n/* block\n   comment */\n__global__ void k(int *p)\n{\n\n    p[0] = 1;\n}\n"
    other = "__global__ void k(int *p)\n{\n    p[0] = 2;\n}\n"
    assert bench.strip_comments(code) == bench.strip_comments(same)
    assert bench.strip_comments(code) != bench.strip_comments(other)
    import json
    import os
    with open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")) as f:
        d = json.load(f)
    want = d["kernels"]["k_fill_tma"]["dram_bytes_per_launch"] \
        if d["kernel_source_hash"] == bench.kernel_source_hash() else None   # a stale figure reads as null
    assert bench.profiled_traffic("k_fill_tma") == want
