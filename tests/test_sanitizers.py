"""Host code under AddressSanitizer and UndefinedBehaviorSanitizer.

Two drivers under tests/sanitize/ are compiled with gcc/g++ and
``-fsanitize=address,undefined -fno-sanitize-recover=all``: one calls every
entry point of the C oracle on small, empty and degenerate inputs, the other
the library's host-only code (argument validation, the angle edges, the B-bin
thresholds of Eq. 6, the track read-out of Eq. 4-5) on valid and invalid
arguments.  A report from either sanitizer, or a wrong status, fails the test.
No GPU is used: the CUDA sources are not part of these builds.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-O1", "-g", "-ffp-contract=off", "-fsanitize=address,undefined", "-fno-sanitize-recover=all"]
CSRC = os.path.join(ROOT, "paper_1507_03074_gb300", "csrc")


def _build_and_run(tmp_path, compiler, std, sources, includes, libs=()):
    if shutil.which(compiler) is None:
        pytest.skip(f"{compiler} not found")
    exe = str(tmp_path / "driver")
    cmd = [compiler, std, *SAN, *[f"-I{d}" for d in includes], *sources, "-o", exe, *libs]
    b = subprocess.run(cmd, capture_output=True, text=True)
    if b.returncode != 0 and ("asan" in b.stderr.lower() or "ubsan" in b.stderr.lower()):
        pytest.skip("sanitizer runtime not available: " + b.stderr.strip().splitlines()[-1])
    assert b.returncode == 0, b.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert "runtime error" not in r.stderr, r.stderr
    assert "AddressSanitizer" not in r.stderr, r.stderr
    assert "LeakSanitizer" not in r.stderr, r.stderr
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), (r.stdout, r.stderr)


def test_oracle_under_sanitizers(tmp_path):
    _build_and_run(tmp_path, "gcc", "-std=c11", [os.path.join(ROOT, "tests", "sanitize", "oracle_driver.c")],
                   [os.path.join(ROOT, "oracle")], ["-lm"])


def test_host_runtime_under_sanitizers(tmp_path):
    _build_and_run(tmp_path, "g++", "-std=c++17",
                   [os.path.join(ROOT, "tests", "sanitize", "host_driver.cpp"),
                    os.path.join(CSRC, "ht_geom.cpp"), os.path.join(CSRC, "ht_readout.cpp")],
                   [os.path.join(ROOT, "include"), CSRC])
