"""CPU-side checks of the CUDA library: it loads, exports every function
include/ht.h declares, and its host-only logic (argument validation, edge
tables) agrees with the oracle.  No device calls."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_1507_03074_gb300 import ht, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_03074_gb300 import build
    build.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ht.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ht_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert "ht_create" in names and "ht_find_maxima" in names
    L = ctypes.CDLL(ht.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("bins", [synth.TINY_BINNING, synth.PAPER_BINNING, synth.UPGRADE_BINNING,
                                  (7, 9, 4, 4), (1, 1, 8, 8), (3, 1024, 8, 8)])
@pytest.mark.parametrize("rng", [dict(), dict(theta_min=0.3, theta_max=2.9, phi_min=-1.0, phi_max=2.5),
                                 dict(theta_min=float(np.float32(np.pi / 4)), phi_min=0.0)])
def test_edges_match_oracle(bins, rng):
    et, ep = ht.compute_edges(ht.Binning(*bins), ht.Ranges(**rng))
    ot, op = oracle.edges(oracle.Binning(*bins), oracle.Ranges(**rng))
    assert et.tobytes() == ot.tobytes()
    assert ep.tobytes() == op.tobytes()


@pytest.mark.parametrize("bins,rng,thr", [
    ((0, 4, 8, 8), {}, 1), ((4, 0, 8, 8), {}, 1), ((2, 2, 0, 8), {}, 1), ((2, 2, 8, 70000), {}, 1),
    ((1025, 1, 8, 8), {}, 1), ((128, 128, 8, 8), {}, 1), ((8, 32, 4096, 4096), {}, 1),
    ((2, 4, 64, 64), {}, 0), ((2, 4, 64, 64), dict(a_min=5.0, a_max=5.0), 1),
    ((2, 4, 64, 64), dict(theta_max=4.0), 1), ((2, 4, 64, 64), dict(phi_min=-4.0), 1),
    ((2, 4, 64, 64), dict(b_max=float("nan")), 1)])
def test_validation_rejects(bins, rng, thr):
    assert ht.validate(ht.Binning(*bins), ht.Ranges(**rng), thr) == ht.HT_E_INVAL
    assert ht.last_error()


def test_validation_accepts_configs():
    for bins in (synth.TINY_BINNING, synth.PAPER_BINNING, synth.UPGRADE_BINNING):
        assert ht.validate(ht.Binning(*bins), ht.Ranges(), 10) == ht.HT_OK


def test_create_rejects_before_touching_device():
    h = ctypes.c_void_p()
    b, r = ht.Binning(0, 4, 8, 8).c(), ht.Ranges().c()
    rc = ht.lib().ht_create(ctypes.byref(b), ctypes.byref(r), 5, 100, ctypes.byref(h))
    assert rc == ht.HT_E_INVAL and not h.value
