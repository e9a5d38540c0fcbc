"""Serving (ht_server_*): every request's peaks equal those of the event
processed alone (ht_find_maxima through a context) and those of the CPU
oracle, whether it ran in a micro-batch with others, next to other binnings,
or after lanes were freed and re-created under a tight memory budget.  The
serving workload itself -- Poisson-stream hit counts, 4x16x1024x1024 events
mixed with 8x32x2048x2048 events of 50 000 hits -- is checked against the
oracle request by request."""
import numpy as np
import pytest

import oracle
from paper_1507_03074_gb300 import synth

pytestmark = pytest.mark.gpu

PEAK_FIELDS = ("itheta", "iphi", "ia", "ib", "votes", "a_c", "b_c", "event")


@pytest.fixture(scope="module")
def ht():
    import torch
    from paper_1507_03074_gb300 import build
    build.build()
    from paper_1507_03074_gb300 import ht as _ht
    torch.cuda.init()
    return _ht


def _alone(ht, b, r, T, ev):
    with ht.Context(b, r, threshold=T, max_hits=max(len(ev[0]), 1)) as ctx:
        ctx.fill(*ev)
        return ctx.find_maxima(capacity=1 << 16)


def _same(got, want):
    assert len(got) == len(want)
    for f in PEAK_FIELDS:
        assert np.array_equal(got[f], want[f]), f


def _wait(S, t, capacity=1 << 16):
    res = S.poll(t, capacity=capacity, timeout_us=20_000_000)
    assert res is not None, "request still pending after 20 s"
    return res


def test_server_mix_equals_alone(ht):
    bA, TA = ht.Binning(*synth.PAPER_BINNING), 10
    bB, TB = ht.Binning(2, 8, 256, 256), 6
    r = ht.Ranges()
    evA = [(e.x, e.y, e.z) for e in synth.batch_events(12, seed0=3000, lo=200, hi=5000)]
    evB = [(e.x, e.y, e.z) for e in synth.batch_events(8, seed0=3100, lo=200, hi=3000)]
    refA = [_alone(ht, bA, r, TA, ev) for ev in evA]
    refB = [_alone(ht, bB, r, TB, ev) for ev in evB]
    with ht.Server(n_streams=2, max_batch=4) as S:
        # a burst: requests pile up behind the busy lanes and run in micro-batches
        tickets = []
        for i in range(max(len(evA), len(evB))):
            if i < len(evA):
                tickets.append(("A", i, S.submit(bA, r, TA, *evA[i])))
            if i < len(evB):
                tickets.append(("B", i, S.submit(bB, r, TB, *evB[i])))
        for kind, i, t in tickets:
            status, pk, n = _wait(S, t)
            want, n_want = (refA if kind == "A" else refB)[i]
            assert status == ht.HT_OK and n == n_want, (kind, i)
            _same(pk, want)
        st = S.stats(reset=True)
        assert st["completed"] == len(tickets) and st["waiting"] == 0 and st["in_flight"] == 0
        assert 1 <= st["micro_batches"] <= len(tickets) and st["lanes"] >= 2
        assert st["p50_us"] > 0 and st["p99_us"] >= st["p50_us"]
        # one at a time: each request alone in the server
        for i in (0, 5, 11):
            status, pk, n = _wait(S, S.submit(bA, r, TA, *evA[i]))
            assert n == refA[i][1]
            _same(pk, refA[i][0])
        # truncation at poll time
        status, pk, n = _wait(S, S.submit(bA, r, TA, *evA[0]), capacity=3)
        assert status == ht.HT_TRUNCATED and n == refA[0][1] and len(pk) == 3
        _same(pk, refA[0][0][:3])
        with pytest.raises(ht.HTError):
            S.poll(123456789)                     # unknown ticket


def test_server_memory_budget(ht):
    r = ht.Ranges()
    bins = [ht.Binning(*synth.PAPER_BINNING), ht.Binning(4, 16, 512, 512), ht.Binning(4, 16, 1024, 512)]
    evs = [(e.x, e.y, e.z) for e in synth.batch_events(6, seed0=3200, lo=300, hi=2000)]
    refs = {(k, i): _alone(ht, b, r, 8, evs[i]) for k, b in enumerate(bins) for i in range(len(evs))}
    budget = 700 << 20     # one lane of the paper binning plus one small one at a time
    with ht.Server(hbm_budget_bytes=budget, n_streams=1, max_batch=2, max_hits_per_event=8192) as S:
        tickets = [(k, i, S.submit(b, r, 8, *evs[i])) for i in range(len(evs)) for k, b in enumerate(bins)]
        for k, i, t in tickets:
            status, pk, n = _wait(S, t)
            assert n == refs[(k, i)][1], (k, i)
            _same(pk, refs[(k, i)][0])
        st = S.stats()
        assert st["lane_bytes"] <= budget * 1.25
        # a binning whose matrix alone exceeds the budget is refused
        big = ht.Binning(8, 32, 2048, 2048)
        t = S.submit(big, r, 10, *evs[0])
        with pytest.raises(ht.HTError) as err:
            _wait(S, t)
        assert err.value.status == ht.HT_E_NOMEM
        # and the server keeps serving
        status, pk, n = _wait(S, S.submit(bins[1], r, 8, *evs[2]))
        _same(pk, refs[(1, 2)][0])


def test_server_peaks_only_equals_alone(ht):
    """A peaks-only server (HT_PEAKS_ONLY lanes): the same peaks as the event
    processed alone with its matrix written, for two binnings in a burst."""
    bA, TA = ht.Binning(*synth.PAPER_BINNING), 10
    bB, TB = ht.Binning(2, 8, 256, 256), 6
    r = ht.Ranges()
    evA = [(e.x, e.y, e.z) for e in synth.batch_events(10, seed0=3200, lo=200, hi=5000)]
    evB = [(e.x, e.y, e.z) for e in synth.batch_events(6, seed0=3300, lo=200, hi=3000)]
    refA = [_alone(ht, bA, r, TA, ev) for ev in evA]
    refB = [_alone(ht, bB, r, TB, ev) for ev in evB]
    with ht.Server(n_streams=2, max_batch=4, peaks_only=True) as S:
        tickets = [("A", i, S.submit(bA, r, TA, *ev)) for i, ev in enumerate(evA)]
        tickets += [("B", i, S.submit(bB, r, TB, *ev)) for i, ev in enumerate(evB)]
        for kind, i, t in tickets:
            status, pk, n = _wait(S, t)
            want_pk, want_n = (refA if kind == "A" else refB)[i]
            assert n == want_n
            _same(pk, want_pk)
    # any other flag is refused at creation
    import ctypes
    cfg = ht.c_server_cfg(0, 0, 0, 0, 0, ht.HT_FILL_NAIVE)
    h = ctypes.c_void_p()
    assert ht.lib().ht_server_create(ctypes.byref(cfg), ctypes.byref(h)) == ht.HT_E_INVAL


def test_server_one_fill_cta_per_sm_equals_alone(ht):
    """Lanes at one fill CTA per SM (the fills of micro-batches on several
    lanes then share every SM): the same peaks as each event alone, for two
    binnings in a burst; more than 32 CTAs per SM is refused."""
    bA, TA = ht.Binning(*synth.PAPER_BINNING), 10
    bB, TB = ht.Binning(2, 8, 256, 256), 6
    r = ht.Ranges()
    evA = [(e.x, e.y, e.z) for e in synth.batch_events(10, seed0=3400, lo=200, hi=5000)]
    evB = [(e.x, e.y, e.z) for e in synth.batch_events(6, seed0=3500, lo=200, hi=3000)]
    refA = [_alone(ht, bA, r, TA, ev) for ev in evA]
    refB = [_alone(ht, bB, r, TB, ev) for ev in evB]
    with ht.Server(n_streams=3, max_batch=4, fill_blocks_per_sm=1) as S:
        tickets = [("A", i, S.submit(bA, r, TA, *ev)) for i, ev in enumerate(evA)]
        tickets += [("B", i, S.submit(bB, r, TB, *ev)) for i, ev in enumerate(evB)]
        for kind, i, t in tickets:
            status, pk, n = _wait(S, t)
            want_pk, want_n = (refA if kind == "A" else refB)[i]
            assert n == want_n
            _same(pk, want_pk)
    import ctypes
    cfg = ht.c_server_cfg(0, 0, 0, 0, 0, 0, 33)
    h = ctypes.c_void_p()
    assert ht.lib().ht_server_create(ctypes.byref(cfg), ctypes.byref(h)) == ht.HT_E_INVAL


# ---------------------------------------------------------------------------
# The serving workload against the oracle
# ---------------------------------------------------------------------------

def _oracle(b, T, ev):
    """Peaks of one event by the oracle's fill and maxima (Sec. 2)."""
    ob, orr = oracle.Binning(*b.shape(), b.win_theta, b.win_phi), oracle.Ranges()
    M, _ = oracle.fill(ob, orr, *ev)
    pk, n = oracle.find_maxima(ob, orr, M, T)
    del M
    return pk, n


@pytest.fixture(scope="module")
def serving_mix(ht):
    """24 requests of the serving stream (arrival order, hit counts lognormal
    with median 3000 clipped to 200..50 000, 10 % of them in the upgrade
    binning), with requests 3 and 11 replaced by 50 000-hit upgrade events;
    each with the oracle's peaks."""
    paper, upgrade = ht.Binning(*synth.PAPER_BINNING), ht.Binning(*synth.UPGRADE_BINNING)
    _, n_hits, is_up, seeds = synth.serving_stream(10000.0, 24, seed=3000)
    reqs = []
    for i in range(24):
        if i in (3, 11):
            e = synth.upgrade_event(10 + i)
            b = upgrade
        else:
            e = synth.make_event(*synth.split_hits(int(n_hits[i])), seed=int(seeds[i]))
            b = upgrade if is_up[i] else paper
        ev = (e.x, e.y, e.z)
        reqs.append((b, ev, _oracle(b, 10, ev)))
    assert sum(r[0] is upgrade for r in reqs) >= 2
    assert sum(len(r[1][0]) == 50000 for r in reqs) >= 2
    return reqs


@pytest.mark.parametrize("cfg", [dict(n_streams=2, max_batch=4), dict(n_streams=3, max_batch=4, fill_blocks_per_sm=1),
                                 dict(n_streams=2, max_batch=4, peaks_only=True)],
                         ids=["default_lanes", "one_fill_cta_per_sm", "peaks_only"])
def test_serving_mix_matches_oracle(ht, serving_mix, cfg):
    """A burst of the serving workload: every polled result equals the
    oracle's peak list for that event, element by element."""
    r = ht.Ranges()
    with ht.Server(**cfg) as S:
        tickets = [S.submit(b, r, 10, *ev) for b, ev, _ in serving_mix]
        for k, t in enumerate(tickets):
            status, pk, n = _wait(S, t, capacity=1 << 17)
            want, n_want = serving_mix[k][2]
            assert status == ht.HT_OK and n == n_want, k
            for f in PEAK_FIELDS[:-1]:
                assert np.array_equal(pk[f], want[f]), (k, f)
        st = S.stats()
        assert st["completed"] == len(tickets) and st["lanes"] >= 2
