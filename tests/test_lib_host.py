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


def _bin_by_division(B, b_min, db, nb):
    # the documented FP32 rule, evaluated with numpy float32 operations
    t = (B - np.float32(b_min)) / np.float32(db)
    out = np.full(B.shape, -1, np.int64)
    ok = (t >= 0) & (t < np.float32(nb))
    out[ok] = t[ok].astype(np.int64)
    return out


@pytest.mark.parametrize("nb,rng", [(64, dict()), (1024, dict()), (2048, dict()), (29, dict(b_min=-900.0, b_max=2100.0)),
                                    (1000, dict(b_min=-1234.5, b_max=987.25)), (7, dict(b_min=0.125, b_max=0.5))])
def test_b_thresholds_equal_division(nb, rng):
    b, r = ht.Binning(1, 1, 4, nb), ht.Ranges(**rng)
    beta = ht.compute_b_thresholds(b, r)
    assert np.all(np.diff(beta) > 0)
    db = np.float32((np.float32(r.b_max) - np.float32(r.b_min)) / np.float32(nb))
    g = np.random.default_rng(nb)
    span = r.b_max - r.b_min
    B = g.uniform(r.b_min - 0.1 * span, r.b_max + 0.1 * span, 200000).astype(np.float32)
    # every threshold and its float neighbours, plus the range ends
    near = np.concatenate([beta, np.nextafter(beta, np.float32(-np.inf)), np.nextafter(beta, np.float32(np.inf)),
                           np.float32([r.b_min, r.b_max, np.nan, np.inf, -np.inf])])
    B = np.concatenate([B, near.astype(np.float32)])
    want = _bin_by_division(B, r.b_min, db, nb)
    inr = (B >= beta[0]) & (B < beta[nb])
    got = np.where(inr, np.searchsorted(beta, B, side="right") - 1, -1)
    assert np.array_equal(np.where(want >= 0, want, -1), got)


def test_binding_pointer_marshalling():
    """The binding hands the C ABI the address of the caller's own data when
    it already is a C-contiguous array of the right dtype (writable or not,
    empty included), and a converted copy otherwise; tensors are checked for
    dtype and contiguity."""
    import torch
    from paper_1507_03074_gb300 import ht
    x = np.arange(7, dtype=np.float32)
    ro = x.copy()
    ro.setflags(write=False)
    for a in (x, ro, np.zeros(0, np.float32)):
        p, mem, keep = ht._ptr_and_mem(a, np.float32)
        assert keep is a and mem == ht.HT_MEM_HOST
        assert p.value == (a.ctypes.data or None)
    for a in (x.astype(np.float64), x[::2], list(range(4))):
        p, mem, keep = ht._ptr_and_mem(a, np.float32)
        assert keep.dtype == np.float32 and keep.flags.c_contiguous and p.value == keep.ctypes.data
        assert np.array_equal(keep, np.asarray(a, dtype=np.float32))
    t = torch.arange(5, dtype=torch.float32)
    p, mem, keep = ht._ptr_and_mem(t, np.float32)
    assert p.value == t.data_ptr() and mem == ht.HT_MEM_HOST and keep is t
    assert ht._ptr_and_mem(torch.zeros(3, dtype=torch.uint8), np.uint32)[1] == ht.HT_MEM_HOST
    with pytest.raises(TypeError):
        ht._ptr_and_mem(torch.zeros(3, dtype=torch.int64), np.float32)
    with pytest.raises(ValueError):
        ht._ptr_and_mem(torch.zeros(4, 4)[:, 0], np.float32)
