"""ht_find_maxima_noalloc: the maxima scan with the library's static scratch.

Its peaks and counts must equal those of ht_find_maxima (through a context)
and those of the CPU oracle (Sec. 2: threshold plus local maxima of the
(A, B) neighbourhood) on the same matrices, on consecutive calls that share
the static scratch.  A call whose peaks overflow the scratch reports
HT_E_NOMEM, and the next call still gives the right answer.  Collected last
(file name) so that it also runs after every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1507_03074_gb300 import synth


def _lib():
    from paper_1507_03074_gb300 import build
    build.build()
    from paper_1507_03074_gb300 import ht
    return ht


def test_noalloc_rejects_sizes_beyond_its_scratch():
    # validated on the host before any CUDA call: runs without a GPU
    ht = _lib()
    L = ht.lib()
    b, r = ht.Binning(*synth.PAPER_BINNING).c(), ht.Ranges().c()
    fake = ctypes.c_void_p(256)        # never dereferenced: the call returns first
    for n_events in (0, 4097):
        s = L.ht_find_maxima_noalloc(ctypes.byref(b), ctypes.byref(r), 10, fake, n_events, fake, 16, fake, None)
        assert s == ht.HT_E_INVAL
        assert "4096" in ht.last_error()
    s = L.ht_find_maxima_noalloc(ctypes.byref(b), ctypes.byref(r), 10, None, 1, fake, 16, fake, None)
    assert s == ht.HT_E_INVAL
    s = L.ht_find_maxima_noalloc(ctypes.byref(b), ctypes.byref(r), 0, fake, 1, fake, 16, fake, None)
    assert s == ht.HT_E_INVAL


def _context_result(ht, b, r, T, x, y, z, capacity):
    """M_H on the device and the peaks of the existing entry point."""
    import torch
    with ht.Context(b, r, threshold=T, max_hits=max(len(x), 1)) as ctx:
        ctx.fill(x, y, z)
        pk, n = ctx.find_maxima(capacity=capacity)
        M = torch.empty(b.n_cells, dtype=torch.int32, device="cuda")
        ctx.matrix_into(M)
        torch.cuda.synchronize()
    return M, pk, n


def _noalloc(ht, b, r, T, M, n_events, capacity):
    import torch
    out = torch.zeros(n_events * capacity * 8, dtype=torch.int32, device="cuda")
    counts = torch.full((n_events,), -1, dtype=torch.int32, device="cuda")
    ht.find_maxima_noalloc(b, r, T, M, n_events, out, capacity, counts)
    pk = out.cpu().numpy().view(ht.PEAK_DTYPE).reshape(n_events, capacity)
    return pk, counts.cpu().numpy().astype(np.int64)


def _same(got, want):
    assert len(got) == len(want)
    for f in want.dtype.names:
        assert np.array_equal(got[f], want[f]), f


def _oracle_peaks(b, r, T, M):
    """The oracle's peak list of a device matrix (copied to the host)."""
    ob = oracle.Binning(b.n_theta, b.n_phi, b.n_a, b.n_b, b.win_theta, b.win_phi)
    Mh = M.cpu().numpy().view(np.uint32).reshape(b.shape())
    return oracle.find_maxima(ob, oracle.Ranges(**r.__dict__), Mh, T)


def _same_as_oracle(got, want):
    assert len(got) == len(want)
    for f in ("itheta", "iphi", "ia", "ib", "votes", "a_c", "b_c"):
        assert np.array_equal(got[f], want[f]), f


@pytest.mark.gpu
def test_noalloc_matches_find_maxima():
    import torch
    ht = _lib()
    torch.cuda.init()
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    cap = 1 << 12
    evA, evB = synth.paper_event(seed=31), synth.paper_event(seed=32, n_tracks=150, n_noise=40)
    MA, pkA, nA = _context_result(ht, b, r, 10, evA.x, evA.y, evA.z, cap)
    MB, pkB, nB = _context_result(ht, b, r, 10, evB.x, evB.y, evB.z, cap)
    assert nA > 0 and nB > 0 and nA != nB
    refA, n_refA = _oracle_peaks(b, r, 10, MA)
    refB, n_refB = _oracle_peaks(b, r, 10, MB)
    assert (n_refA, n_refB) == (nA, nB)

    # two calls in a row on different matrices (the second sees the first's scratch)
    for M, pk, n in ((MA, pkA, nA), (MB, pkB, nB), (MA, pkA, nA)):
        got, cnt = _noalloc(ht, b, r, 10, M, 1, cap)
        assert cnt[0] == n
        _same(got[0, :n], pk)
        _same_as_oracle(got[0, :n], refA if M is MA else refB)

    # both matrices in one call: per-event lists and counts
    MAB = torch.cat([MA, MB])
    got, cnt = _noalloc(ht, b, r, 10, MAB, 2, cap)
    assert list(cnt) == [nA, nB]
    _same(got[0, :nA], pkA)
    want_b = pkB.copy()
    want_b["event"] = 1
    _same(got[1, :nB], want_b)

    # truncation: the count keeps the total, out holds the first `capacity`
    got, cnt = _noalloc(ht, b, r, 10, MA, 1, 16)
    assert cnt[0] == nA
    _same(got[0], pkA[:16])


@pytest.mark.gpu
def test_noalloc_ragged_binning_direct_scan():
    # n_b not a multiple of 4: the direct-load scan variant
    ht = _lib()
    b = ht.Binning(3, 5, 37, 29)
    r = ht.Ranges(a_min=-1500.0, a_max=1700.0, b_min=-900.0, b_max=2100.0)
    rng = np.random.default_rng(3)
    rad, ph = rng.uniform(20.0, 1100.0, 700), rng.uniform(-np.pi, np.pi, 700)
    x, y = (rad * np.cos(ph)).astype(np.float32), (rad * np.sin(ph)).astype(np.float32)
    z = rng.uniform(-2500, 2500, 700).astype(np.float32)
    for T in (2, 3):
        M, pk, n = _context_result(ht, b, r, T, x, y, z, 1 << 14)
        got, cnt = _noalloc(ht, b, r, T, M, 1, 1 << 14)
        assert cnt[0] == n
        _same(got[0, :n], pk)
        ref, n_ref = _oracle_peaks(b, r, T, M)
        assert n_ref == n
        _same_as_oracle(got[0, :n], ref)


@pytest.mark.gpu
def test_noalloc_scratch_overflow_then_recovers():
    """524,288 isolated peaks (value T on every other row and column of a
    1 x 1 x 2048 x 1024 matrix) exceed the 262,144 entries of the static
    scratch: HT_E_NOMEM; the following call on an ordinary matrix, which
    reuses the same array, equals the oracle."""
    import torch
    ht = _lib()
    torch.cuda.init()
    T = 3
    b, r = ht.Binning(1, 1, 2048, 1024), ht.Ranges()
    Mh = np.zeros((2048, 1024), np.uint32)
    Mh[0::2, 0::2] = T
    M = torch.from_numpy(Mh.view(np.int32).ravel().copy()).cuda()
    cap = 16
    out = torch.zeros(cap * 8, dtype=torch.int32, device="cuda")
    counts = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ht.HTError) as err:
        ht.find_maxima_noalloc(b, r, T, M, 1, out, cap, counts)
    assert err.value.status == ht.HT_E_NOMEM
    assert "262144" in ht.last_error()

    # the next call shares the array, whose counters it clears first
    rng = np.random.default_rng(7)
    Mr = rng.choice(np.arange(4, dtype=np.uint32), size=(2048, 1024), p=[0.5, 0.3, 0.15, 0.05])
    Md = torch.from_numpy(Mr.view(np.int32).ravel().copy()).cuda()
    ref, n_ref = _oracle_peaks(b, r, T, Md)
    got, cnt = _noalloc(ht, b, r, T, Md, 1, n_ref + 8)
    assert cnt[0] == n_ref
    _same_as_oracle(got[0, :n_ref], ref)
