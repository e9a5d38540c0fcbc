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
