"""Batches (ht_batch_*): every event's M_H and peaks equal the oracle's and
the single-event context's, whatever the batch around it; graph replays,
changing event counts, device-side inputs, truncation and the autotuner."""
import numpy as np
import pytest

import oracle
from paper_1507_03074_gb300 import synth

pytestmark = pytest.mark.gpu

PEAK_FIELDS = ("itheta", "iphi", "ia", "ib", "votes", "a_c", "b_c")


@pytest.fixture(scope="module")
def ht():
    import torch
    from paper_1507_03074_gb300 import build
    build.build()
    from paper_1507_03074_gb300 import ht as _ht
    torch.cuda.init()
    return _ht


def _ob(b):
    return oracle.Binning(b.n_theta, b.n_phi, b.n_a, b.n_b, b.win_theta, b.win_phi)


def _orr(r):
    return oracle.Ranges(**r.__dict__)


def _oracle_event(b, r, T, ev):
    M, _ = oracle.fill(_ob(b), _orr(r), ev[0], ev[1], ev[2])
    pk, n = oracle.find_maxima(_ob(b), _orr(r), M, T)
    return M, pk, n


def _split(pk, counts):
    off = np.concatenate([[0], np.cumsum(counts, dtype=np.int64)]).astype(np.int64)
    return [pk[off[e]:off[e + 1]] for e in range(len(counts))]


def _check_events(events, pk, counts, refs, ev_ids=None):
    parts = _split(pk, counts)
    for e, (M_ref, pk_ref, n_ref) in enumerate(refs):
        assert counts[e] == n_ref, e
        got = parts[e]
        for f in PEAK_FIELDS:
            assert np.array_equal(got[f], pk_ref[f]), (e, f)
        assert np.all(got["event"] == e)


@pytest.fixture(scope="module")
def uneven():
    # 6 events, 40 .. 5000 hits (one tiny), paper-scale binning
    evs = [(e.x, e.y, e.z) for e in synth.batch_events(5, seed0=1000, lo=500, hi=5000)]
    t = synth.make_event(3, 4, seed=77)
    evs.insert(2, (t.x, t.y, t.z))
    b = oracle.Binning(*synth.PAPER_BINNING)
    refs = []
    for ev in evs:
        M, _ = oracle.fill(b, oracle.Ranges(), *ev)
        pk, n = oracle.find_maxima(b, oracle.Ranges(), M, 10)
        refs.append((M, pk, n))
    return evs, refs


def test_batch_matches_oracle_and_replays(ht, uneven):
    evs, refs = uneven
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    with ht.Batch(b, r, threshold=10, max_events=8, max_hits=40000, capacity=1 << 16) as B:
        x, y, z, off = ht.Batch.concat(evs)
        for rep in range(3):                       # direct + capture, then graph replays
            pk, counts = B.run(x, y, z, off)
            _check_events(evs, pk, counts, refs)
        for e in (0, 2, len(evs) - 1):
            assert np.array_equal(B.matrix(e), refs[e][0])
        # a different set with the same event count replays the same graph
        rev = evs[::-1]
        x2, y2, z2, off2 = ht.Batch.concat(rev)
        pk, counts = B.run(x2, y2, z2, off2)
        _check_events(rev, pk, counts, refs[::-1])
        # fewer events, then back
        pk, counts = B.run(*ht.Batch.concat(evs[:3]))
        _check_events(evs[:3], pk, counts, refs[:3])
        pk, counts = B.run(x, y, z, off)
        _check_events(evs, pk, counts, refs)


@pytest.mark.parametrize("bin_cluster", [1, 2])
def test_batch_binning_launches(ht, uneven, bin_cluster):
    """Batches of at most 16384 hits: binning and unit lists in one
    thread-block-cluster launch (1, whose CTAs also find each hit's event by
    its offsets) or in two launches (2) -- the same peaks and matrices."""
    evs, refs = uneven
    keep, n = [], 0
    for i, ev in enumerate(evs):
        if n + len(ev[0]) <= 16383:                # room for the one-hit event below
            keep.append(i)
            n += len(ev[0])
    assert len(keep) >= 3 and len(keep) + 2 <= 8
    sub, subr = [evs[i] for i in keep], [refs[i] for i in keep]
    # an empty first event and a one-hit last one: the edges of the search
    # that finds each hit's event by the offsets
    empty = tuple(np.zeros(0, np.float32) for _ in range(3))
    one = tuple(a[:1].copy() for a in sub[0])
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    sub = [empty] + sub + [one]
    subr = [_oracle_event(b, r, 10, empty)] + subr + [_oracle_event(b, r, 10, one)]
    with ht.Batch(b, r, threshold=10, max_events=8, max_hits=16384, capacity=1 << 16) as B:
        B.set_tuning(bin_cluster=bin_cluster)
        assert B.get_tuning()["bin_cluster"] == bin_cluster
        for rep in range(3):                       # direct + capture, then a graph replay
            pk, counts = B.run(*ht.Batch.concat(sub))
            _check_events(sub, pk, counts, subr)
        for e in range(len(sub)):
            assert np.array_equal(B.matrix(e), subr[e][0])
        pk, counts = B.run(*ht.Batch.concat(sub[::-1]))
        _check_events(sub[::-1], pk, counts, subr[::-1])


def test_batch_peaks_only(ht, uneven):
    """HT_PEAKS_ONLY runs: the same peaks, the matrices left as the last
    normal run wrote them; normal and peaks-only runs alternate on their own
    captured graphs, with host and device memory."""
    import torch
    evs, refs = uneven
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    x, y, z, off = ht.Batch.concat(evs)
    with ht.Batch(b, r, threshold=10, max_events=8, max_hits=40000, capacity=1 << 16) as B:
        pk, counts = B.run(x, y, z, off)                      # normal: writes the matrices
        _check_events(evs, pk, counts, refs)
        rev = evs[::-1]
        for _ in range(3):                                     # peaks-only, then graph replays
            pk, counts = B.run(*ht.Batch.concat(rev), peaks_only=True)
            _check_events(rev, pk, counts, refs[::-1])
        assert np.array_equal(B.matrix(0), refs[0][0])         # still the normal run's matrix
        pk, counts = B.run(*ht.Batch.concat(evs[:3]), peaks_only=True)
        _check_events(evs[:3], pk, counts, refs[:3])
        pk, counts = B.run(x, y, z, off)                       # normal again
        _check_events(evs, pk, counts, refs)
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        doff = torch.from_numpy(off.astype(np.int32)).cuda()
        out = torch.zeros((1 << 16) * 8, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(len(evs), dtype=torch.int32, device="cuda")
        B.run_device(dx, dy, dz, doff, int(off[-1]), out, cnt, peaks_only=True)
        B.sync()
        total = sum(n for _, _, n in refs)
        _check_events(evs, out.cpu().numpy().view(ht.PEAK_DTYPE)[:total], cnt.cpu().numpy().astype(np.uint32),
                      refs)


def test_batch_page_locked_inputs(ht, uneven):
    """Hits in page-locked host memory go to the device without the staging
    copy: the same peaks and matrices, and the arrays may be overwritten as
    soon as the call returns."""
    import torch
    evs, refs = uneven
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    x, y, z, off = ht.Batch.concat(evs)
    pinned = [torch.empty(v.size, dtype=torch.float32, pin_memory=True) for v in (x, y, z)]
    for t, v in zip(pinned, (x, y, z)):
        t.numpy()[:] = v
    px, py, pz = (t.numpy() for t in pinned)
    with ht.Batch(b, r, threshold=10, max_events=8, max_hits=40000, capacity=1 << 16) as B:
        for _ in range(2):
            pk, counts = B.run(px, py, pz, off)
            _check_events(evs, pk, counts, refs)
            for t in pinned:
                t.numpy()[:] = np.nan            # reused at once: the run has its copy
            pk2, counts2 = B.run(px, py, pz, off)
            assert counts2.sum() == 0            # all-NaN hits are dropped
            for t, v in zip(pinned, (x, y, z)):
                t.numpy()[:] = v
        assert np.array_equal(B.matrix(1), np.zeros_like(refs[1][0]))
        pk, counts = B.run(px, py, pz, off)
        _check_events(evs, pk, counts, refs)
        for e in range(len(evs)):
            assert np.array_equal(B.matrix(e), refs[e][0]), e


def test_batch_naive_fill(ht, uneven):
    """HT_FILL_NAIVE runs (the paper's fill, its blocks walking the unit
    lists of every event of the batch): the oracle's matrices and peaks;
    naive and fused runs alternate on their own captured graphs, with host
    and device memory."""
    import torch
    evs, refs = uneven
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    x, y, z, off = ht.Batch.concat(evs)
    with ht.Batch(b, r, threshold=10, max_events=8, max_hits=40000, capacity=1 << 16) as B:
        for _ in range(3):                                     # direct, capture, replay
            pk, counts = B.run(x, y, z, off, naive=True)
            _check_events(evs, pk, counts, refs)
        for e in range(len(evs)):
            assert np.array_equal(B.matrix(e), refs[e][0]), e
        rev = evs[::-1]
        pk, counts = B.run(*ht.Batch.concat(rev))              # fused, then naive again
        _check_events(rev, pk, counts, refs[::-1])
        pk, counts = B.run(*ht.Batch.concat(rev), naive=True)
        _check_events(rev, pk, counts, refs[::-1])
        assert np.array_equal(B.matrix(1), refs[-2][0])
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        doff = torch.from_numpy(off.astype(np.int32)).cuda()
        out = torch.zeros((1 << 16) * 8, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(len(evs), dtype=torch.int32, device="cuda")
        B.run_device(dx, dy, dz, doff, int(off[-1]), out, cnt, naive=True)
        B.sync()
        total = sum(n for _, _, n in refs)
        _check_events(evs, out.cpu().numpy().view(ht.PEAK_DTYPE)[:total], cnt.cpu().numpy().astype(np.uint32),
                      refs)
        with pytest.raises(ht.HTError):
            B.run(x, y, z, off, naive=True, peaks_only=True)


def test_event_alone_equals_event_in_batch(ht, uneven):
    evs, refs = uneven
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    with ht.Context(b, r, threshold=10, max_hits=6000) as ctx:
        ctx.fill(*evs[1])
        alone, n_alone = ctx.find_maxima(capacity=1 << 14)
        M_alone = ctx.matrix()
    with ht.Batch(b, r, threshold=10, max_events=8, max_hits=40000, capacity=1 << 16) as B:
        pk, counts = B.run(*ht.Batch.concat(evs))
        mine = _split(pk, counts)[1]
        assert counts[1] == n_alone
        for f in PEAK_FIELDS:
            assert np.array_equal(mine[f], alone[f])
        assert np.array_equal(B.matrix(1), M_alone)


def test_batch_device_mode_and_truncation(ht, uneven):
    import torch
    evs, refs = uneven
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    x, y, z, off = ht.Batch.concat(evs)
    total = sum(n for _, _, n in refs)
    with ht.Batch(b, r, threshold=10, max_events=8, max_hits=40000, capacity=1 << 16) as B:
        dx, dy, dz = (torch.from_numpy(a).cuda() for a in (x, y, z))
        doff = torch.from_numpy(off.astype(np.int32)).cuda()
        out = torch.zeros((1 << 16) * 8, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(len(evs), dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        for _ in range(2):
            B.run_device(dx, dy, dz, doff, int(off[-1]), out, cnt, stream=s)
            B.sync(stream=s)
            counts = cnt.cpu().numpy().astype(np.uint32)
            pk = out.cpu().numpy().view(ht.PEAK_DTYPE)[:total]
            _check_events(evs, pk, counts, refs)
    # a batch with room for fewer peaks than the events hold
    with ht.Batch(b, r, threshold=10, max_events=8, max_hits=40000, capacity=100) as B:
        pk, counts, status = B.run_raw(x, y, z, off)
        assert status == ht.HT_TRUNCATED and int(counts.sum()) == total and len(pk) == 100
        full = np.concatenate([p for _, p, _ in refs])
        for f in PEAK_FIELDS:
            assert np.array_equal(pk[f], full[:100][f])


def test_batch_ragged_binning_and_autotune(ht):
    # n_b not a multiple of 4 (direct scan) and several strips per slice
    b = ht.Binning(3, 5, 37, 29)
    r = ht.Ranges(a_min=-1500.0, a_max=1700.0, b_min=-900.0, b_max=2100.0)
    rng = np.random.default_rng(5)
    evs = []
    for n in (700, 50, 0, 1200):
        rad, ph = rng.uniform(20.0, 1100.0, n), rng.uniform(-np.pi, np.pi, n)
        evs.append(((rad * np.cos(ph)).astype(np.float32), (rad * np.sin(ph)).astype(np.float32),
                    rng.uniform(-2500, 2500, n).astype(np.float32)))
    refs = [_oracle_event(b, r, 2, ev) for ev in evs]
    with ht.Batch(b, r, threshold=2, max_events=4, max_hits=4000, capacity=1 << 16) as B:
        x, y, z, off = ht.Batch.concat(evs)
        pk, counts = B.run(x, y, z, off)
        _check_events(evs, pk, counts, refs)
        chosen, us = B.autotune(reps=2)
        assert us > 0
        for _ in range(2):
            pk, counts = B.run(x, y, z, off)
            _check_events(evs, pk, counts, refs)
        for e in range(len(evs)):
            assert np.array_equal(B.matrix(e), refs[e][0])


def test_batch_windows_every_fill(ht):
    """Admission windows (a hit votes in up to 3 x 3 slices) on a batch of
    uneven events, one of them empty: the fused fill, the paper's fill and the
    peaks-only fill all give the oracle's peaks, and the two that write M_H
    its matrices."""
    b = ht.Binning(4, 16, 128, 128, 1, 1)
    r = ht.Ranges()
    evs = []
    for k, (nt, nn) in enumerate(((60, 10), (0, 0), (140, 30), (25, 5))):
        e = synth.paper_event(seed=300 + k, n_tracks=nt, n_noise=nn) if nt else None
        evs.append((e.x, e.y, e.z) if e is not None else tuple(np.zeros(0, np.float32) for _ in range(3)))
    refs = [_oracle_event(b, r, 5, ev) for ev in evs]
    x, y, z, off = ht.Batch.concat(evs)
    with ht.Batch(b, r, threshold=5, max_events=4, max_hits=8000, capacity=1 << 16) as B:
        for kw in (dict(), dict(naive=True), dict(peaks_only=True), dict()):
            pk, counts = B.run(x, y, z, off, **kw)
            _check_events(evs, pk, counts, refs)
            if not kw.get("peaks_only"):
                for e in range(len(evs)):
                    assert np.array_equal(B.matrix(e), refs[e][0]), (kw, e)


def test_batch_rejects_bad_arguments(ht):
    b, r = ht.Binning(*synth.TINY_BINNING), ht.Ranges()
    ev = synth.tiny_event()
    with ht.Batch(b, r, threshold=8, max_events=2, max_hits=1000, capacity=64) as B:
        x, y, z, off = ht.Batch.concat([(ev.x, ev.y, ev.z)] * 3)
        with pytest.raises(ht.HTError):
            B.run(x, y, z, off)                    # 3 events > max_events
        x, y, z, off = ht.Batch.concat([(ev.x, ev.y, ev.z)] * 2)
        bad = off.copy()
        bad[1] = bad[2] + 1                        # decreasing offsets
        with pytest.raises(ht.HTError):
            B.run(x, y, z, bad)
        pk, counts = B.run(x, y, z, off)           # still usable
        assert counts[0] == counts[1]


def test_batch_cluster_binning_at_its_unit_limit(ht):
    """53 events of 64 (theta, phi) slices fill the one-launch binning's 40 KB
    of counts exactly (3 words per (event, slice) unit and 1 per event, with
    every CTA finding its hits' events by the offsets); 54 events exceed it
    and take the two-launch binning.  Both give the oracle's matrices and
    peaks, event by event."""
    bins = (4, 16, 64, 64)
    b, r = ht.Binning(*bins), ht.Ranges()
    ob, orr = oracle.Binning(*bins), oracle.Ranges()
    evs = [(e.x, e.y, e.z) for e in (synth.make_event(20, 20, seed=3000 + k) for k in range(54))]
    assert sum(len(e[0]) for e in evs) <= 16384
    refs = []
    for ev in evs:
        M, _ = oracle.fill(ob, orr, *ev)
        pk, n = oracle.find_maxima(ob, orr, M, 4)
        refs.append((M, pk, n))
    with ht.Batch(b, r, threshold=4, max_events=54, max_hits=16384, capacity=1 << 16) as B:
        B.set_tuning(bin_cluster=1)
        for n_ev, cluster in ((53, True), (54, False), (53, True)):
            B.profile(True)                        # direct launches, counted per kernel
            pk, counts = B.run(*ht.Batch.concat(evs[:n_ev]))
            prof = B.profile_read()
            B.profile(False)
            assert (prof["k_bin_cluster"][0] > 0) == cluster and (prof["k_bin"][0] > 0) != cluster, prof
            _check_events(evs[:n_ev], pk, counts, refs[:n_ev])
            for e in (0, n_ev // 2, n_ev - 1):
                assert np.array_equal(B.matrix(e), refs[e][0])
        pk, counts = B.run(*ht.Batch.concat(evs[:53]))   # captured graph of the cluster binning
        _check_events(evs[:53], pk, counts, refs[:53])
