"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Vote matrices and peak lists must be bit-exact (integer votes; FP32 vote
arithmetic fixed by the ABI, so bins agree exactly).  Shapes span several
fill tiles and scan stages with ragged tails (n_a not a multiple of the
strip, n_b not a multiple of 4), both fill kernels, host and device inputs,
windows, partial ranges, u32 counter tiles, and the paper-scale and
upgrade-scale binnings at full size.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1507_03074_gb300 import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
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


def assert_peaks_equal(got, want):
    assert len(got) == len(want)
    for f in PEAK_FIELDS:
        assert np.array_equal(got[f], want[f]), f


def random_hits(n, seed, rmax=1100.0):
    rng = np.random.default_rng(seed)
    rad = rng.uniform(20.0, rmax, n)
    ph = rng.uniform(-np.pi, np.pi, n)
    x = (rad * np.cos(ph)).astype(np.float32)
    y = (rad * np.sin(ph)).astype(np.float32)
    z = rng.uniform(-2500, 2500, n).astype(np.float32)
    return x, y, z


def degenerate_hits():
    """A small event plus the hits the method's arithmetic has to drop or
    bin on an edge: y = 0 (2y = 0: B is +-inf or NaN), x = 0, the origin
    (rho = 0), signed zeros, both diagonals and the axes (pseudo-angles on
    phi edges), z = 0 and z = +-rho (theta edges), NaN and inf
    coordinates, x^2 + y^2 overflowing, subnormal coordinates."""
    ev = synth.paper_event(seed=7, n_tracks=100, n_noise=20)
    nan, inf = np.float32(np.nan), np.float32(np.inf)
    pts = []
    for rr in (30.0, 100.0, 527.5, 1000.0):
        for (a, bb) in ((rr, 0.0), (-rr, 0.0), (0.0, rr), (0.0, -rr), (rr, rr), (-rr, rr), (-rr, -rr), (rr, -rr),
                        (-0.0, rr), (rr, -0.0), (0.0, -0.0)):
            rho = float(np.hypot(a, bb))
            for zz in (0.0, rho, -rho, 0.5 * rr, -2.0 * rr):
                pts.append((a, bb, zz))
    pts += [(nan, 10.0, 0.0), (10.0, nan, 0.0), (10.0, 10.0, nan), (inf, 10.0, 0.0), (10.0, -inf, 5.0),
            (10.0, 10.0, inf), (1e30, 1e30, 0.0), (-1e30, 3.0, 1.0), (1e-40, 1e-40, 0.0), (-1e-40, 7.0, 1e-40)]
    d = np.array(pts, dtype=np.float32)
    x = np.concatenate([ev.x, d[:, 0]]).astype(np.float32)
    y = np.concatenate([ev.y, d[:, 1]]).astype(np.float32)
    z = np.concatenate([ev.z, d[:, 2]]).astype(np.float32)
    perm = np.random.default_rng(11).permutation(x.size)
    return x[perm], y[perm], z[perm]


def run_gpu(ht, b, r, T, x, y, z, naive=False, device=True, capacity=1 << 20, max_hits=None, tuning=None):
    import torch
    with ht.Context(b, r, threshold=T, max_hits=max_hits or max(len(x), 1)) as ctx:
        if tuning:
            ctx.set_tuning(**tuning)
        if device:
            ctx.fill(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(z).cuda(),
                     naive=naive)
        else:
            ctx.fill(x, y, z, naive=naive)
        pk, n = ctx.find_maxima(capacity=capacity)
        M = ctx.matrix()
        launches = ctx.launches
    return M, pk, n, launches


def event_cases():
    ev = synth.tiny_event()
    yield "tiny", synth.TINY_BINNING, {}, 8, (ev.x, ev.y, ev.z)
    ev = synth.paper_event(seed=1)
    yield "paper", synth.PAPER_BINNING, {}, 10, (ev.x, ev.y, ev.z)
    yield "ragged_nb", (3, 5, 37, 29), dict(a_min=-1500.0, a_max=1700.0, b_min=-900.0, b_max=2100.0), \
        2, random_hits(700, 3)
    ev = synth.paper_event(seed=5, n_tracks=150, n_noise=50)
    yield "ragged_na", (4, 8, 100, 96), {}, 4, (ev.x, ev.y, ev.z)
    yield "windows", (4, 16, 128, 128, 1, 1), {}, 5, (ev.x, ev.y, ev.z)
    yield "partial_ranges", (3, 6, 80, 64, 1, 2), dict(theta_min=0.4, theta_max=2.6, phi_min=-2.0,
                                                       phi_max=1.5), 3, (ev.x, ev.y, ev.z)
    yield "wide_b", (2, 2, 40, 2048), {}, 3, (ev.x, ev.y, ev.z)
    # thousands of hits per slice: the fill selects them in several chunks
    yield "dense_slices", (1, 2, 70, 128), {}, 6, random_hits(5000, 4, rmax=900.0)
    # axes, diagonals, zeros, NaN / inf / overflowing / subnormal coordinates
    yield "degenerate_hits", (4, 16, 256, 256), {}, 3, degenerate_hits()


CASES = list(event_cases())


@pytest.mark.parametrize("naive", [False, True], ids=["priv", "naive"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fill_and_maxima_match_oracle(ht, case, naive):
    name, bins, rng, T, (x, y, z) = case
    b, r = ht.Binning(*bins), ht.Ranges(**rng)
    M_ref, votes = oracle.fill(_ob(b), _orr(r), x, y, z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
    M, pk, n, _ = run_gpu(ht, b, r, T, x, y, z, naive=naive, device=(name != "tiny"))
    assert int(M.sum(dtype=np.uint64)) == votes
    assert np.array_equal(M, M_ref)
    assert n == n_ref
    assert_peaks_equal(pk, pk_ref)
    assert np.all(pk["event"] == 0)


@pytest.mark.parametrize("bin_cluster", [1, 2], ids=["cluster", "two_launches"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_binning_launches_match_oracle(ht, case, bin_cluster):
    """Both binnings -- one thread-block-cluster launch (k_bin_cluster, which
    also splits the bulk-copy-tile fill's work) or k_bin + k_scatter -- on
    every geometry: windows, partial ranges, ragged shapes, dense slices and
    degenerate coordinates, each with the default fill of its shape, twice
    in a row on one context."""
    name, bins, rng, T, (x, y, z) = case
    b, r = ht.Binning(*bins), ht.Ranges(**rng)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), x, y, z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
    with ht.Context(b, r, threshold=T, max_hits=max(len(x), 1)) as ctx:
        ctx.set_tuning(bin_cluster=bin_cluster)
        assert ctx.get_tuning()["bin_cluster"] == bin_cluster
        for _ in range(2):
            ctx.fill(x, y, z)
            pk, n = ctx.find_maxima(capacity=1 << 20)
            assert n == n_ref
            assert_peaks_equal(pk, pk_ref)
        assert np.array_equal(ctx.matrix(), M_ref)


@pytest.mark.parametrize("mode", [4, 5], ids=["staging", "tiles"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_bulk_store_fill_matches_oracle(ht, case, mode):
    """The fused fills whose passes leave by bulk async copies -- through
    shared-memory staging (fill_fused_scan=4) or as whole u32 tiles
    (fill_fused_scan=5): bit-exact M_H and peaks, or a refusal when n_b is
    not a multiple of 4."""
    name, bins, rng, T, (x, y, z) = case
    b, r = ht.Binning(*bins), ht.Ranges(**rng)
    M_ref, votes = oracle.fill(_ob(b), _orr(r), x, y, z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
    with ht.Context(b, r, threshold=T, max_hits=max(len(x), 1)) as ctx:
        if b.n_b % 4:
            with pytest.raises(ht.HTError):
                ctx.set_tuning(fill_fused_scan=mode)
            return
        ctx.set_tuning(fill_fused_scan=mode)
        assert ctx.get_tuning()["fill_fused_scan"] == mode
        for _ in range(2):
            ctx.fill(x, y, z)
            pk, n = ctx.find_maxima(capacity=1 << 20)
            assert n == n_ref
            assert_peaks_equal(pk, pk_ref)
        assert np.array_equal(ctx.matrix(), M_ref)


U32_TUNINGS = [None, dict(fill_fused_scan=2), dict(fill_fused_scan=1, fill_rows=2, fill_threads=256),
               dict(fill_fused_scan=1, fill_rows=4, fill_threads=256), dict(fill_fused_scan=3, fill_rows=2),
               dict(fill_fused_scan=3, fill_rows=8), dict(fill_fused_scan=4), dict(fill_fused_scan=4, fill_rows=4),
               dict(fill_fused_scan=5), dict(fill_fused_scan=5, fill_rows=2, fill_threads=256),
               dict(fill_fused_scan=5, fill_rows=64, fill_threads=1024), dict(fill_fused_scan=5, fill_vote_agg=1),
               dict(fill_fused_scan=5, fill_vote_agg=1, fill_rows=2, fill_threads=256)]


@pytest.mark.parametrize("tuning", U32_TUNINGS, ids=[str(t) for t in U32_TUNINGS])
def test_u32_counter_tiles(ht, tuning):
    # > 65535 hits in one slice: the fill switches that slice to u32 counters
    # (half the rows per pass; one row per pass with 2-row strips).  T = 3
    # lists more cells per pass than the fused fill's candidate lists hold.
    b, r = ht.Binning(1, 1, 64, 96), ht.Ranges()
    x, y, z = random_hits(70000, 9, rmax=400.0)
    # half the hits on one circle so that cells exceed 16 bits
    x[:35000], y[:35000] = np.float32(300.0), np.float32(250.0)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), x, y, z)
    assert M_ref.max() >= 35000
    for T in (50, 3):
        pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
        M, pk, n, _ = run_gpu(ht, b, r, T, x, y, z, tuning=tuning)
        assert np.array_equal(M, M_ref)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)


def test_empty_event_clears_in_place(ht):
    import torch
    b, r = ht.Binning(*synth.TINY_BINNING), ht.Ranges()
    ev = synth.tiny_event()
    with ht.Context(b, r, threshold=8, max_hits=256) as ctx:
        ctx.fill(ev.x, ev.y, ev.z)
        assert ctx.matrix().sum() > 0
        e = torch.empty(0, dtype=torch.float32, device="cuda")
        for naive in (False, True):
            ctx.fill(ev.x, ev.y, ev.z, naive=not naive)
            ctx.fill(e, e, e, naive=naive)
            assert ctx.matrix().sum() == 0
            pk, n = ctx.find_maxima(capacity=16)
            assert n == 0 and len(pk) == 0


def test_permutation_and_accumulate(ht):
    b, r = ht.Binning(4, 16, 256, 256), ht.Ranges()
    ev = synth.paper_event(seed=8, n_tracks=200, n_noise=60)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), ev.x, ev.y, ev.z)
    perm = np.random.default_rng(1).permutation(ev.n_hits)
    with ht.Context(b, r, threshold=6, max_hits=ev.n_hits) as ctx:
        ctx.fill(ev.x[perm], ev.y[perm], ev.z[perm])
        assert np.array_equal(ctx.matrix(), M_ref)
        for naive in (False, True):
            k = ev.n_hits // 3
            ctx.fill(ev.x[:k], ev.y[:k], ev.z[:k], naive=naive)
            ctx.fill(ev.x[k:], ev.y[k:], ev.z[k:], accumulate=True, naive=naive)
            assert np.array_equal(ctx.matrix(), M_ref)
        with pytest.raises(ht.HTError):
            ctx.fill(ev.x, ev.y, ev.z, accumulate=True)      # beyond max_hits


def test_truncation_and_repeat(ht):
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    ev = synth.paper_event(seed=1)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), ev.x, ev.y, ev.z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, 10)
    assert n_ref > 5
    with ht.Context(b, r, threshold=10, max_hits=ev.n_hits) as ctx:
        ctx.fill(ev.x, ev.y, ev.z)
        for cap in (5, 0, n_ref, n_ref + 7):
            pk, n = ctx.find_maxima(capacity=cap)
            assert n == n_ref
            assert_peaks_equal(pk, pk_ref[:cap])


def test_device_mode_on_torch_stream(ht):
    import torch
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    ev = synth.paper_event(seed=2)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), ev.x, ev.y, ev.z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, 10)
    s = torch.cuda.Stream()
    cap = 4096
    with ht.Context(b, r, threshold=10, max_hits=8192) as ctx, torch.cuda.stream(s):
        x, y, z = (torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z))
        out = torch.zeros(cap * 8, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        Md = torch.zeros(b.n_cells, dtype=torch.int32, device="cuda")
        ctx.fill(x, y, z, stream=s)
        ctx.find_maxima(capacity=cap, out=out, count=cnt, stream=s)
        ctx.matrix_into(Md, stream=s)
        s.synchronize()
        ctx.sync()
    assert int(cnt.item()) == n_ref
    got = out.cpu().numpy().view(ht.PEAK_DTYPE)[:n_ref]
    assert_peaks_equal(got, pk_ref)
    assert np.array_equal(Md.cpu().numpy().view(np.uint32).reshape(b.shape()), M_ref)


@pytest.mark.parametrize("tuning", [None, dict(fill_blocks_per_sm=1)], ids=["default", "one_fill_cta_per_sm"])
def test_contexts_in_flight(ht, tuning):
    # Several contexts on their own streams, events issued round-robin with no
    # waits in between (the bench's events in flight): every event's peaks and
    # the last M_H of every context equal the oracle's; odd rounds take the
    # peaks-only fill.  Ragged binning, a few thousand hits per event.
    import torch
    b = ht.Binning(3, 6, 200, 136)
    r = ht.Ranges(a_min=-1800.0, a_max=1600.0, b_min=-1700.0, b_max=1900.0)
    T, C, n_ev, cap = 5, 4, 12, 8192
    evs = [random_hits(2000 + 150 * k, 700 + k) for k in range(n_ev)]
    refs = []
    for x, y, z in evs:
        M_ref, _ = oracle.fill(_ob(b), _orr(r), x, y, z)
        refs.append((M_ref,) + tuple(oracle.find_maxima(_ob(b), _orr(r), M_ref, T)))
    ctxs = [ht.Context(b, r, threshold=T, max_hits=4096) for _ in range(C)]
    sts = [torch.cuda.Stream() for _ in range(C)]
    try:
        for c in ctxs:
            if tuning:
                c.set_tuning(**tuning)
        dev = [tuple(torch.from_numpy(a).cuda() for a in e) for e in evs]
        outs = [torch.zeros(cap * 8, dtype=torch.int32, device="cuda") for _ in range(n_ev)]
        cnts = torch.zeros(n_ev, dtype=torch.int32, device="cuda")
        Ms = [torch.zeros(b.n_cells, dtype=torch.int32, device="cuda") for _ in range(C)]
        torch.cuda.synchronize()
        for k in range(n_ev):
            c = k % C
            po = (k // C) % 2 == 1 and k < n_ev - C   # the last round writes M_H
            ctxs[c].fill(*dev[k], peaks_only=po, stream=sts[c])
            ctxs[c].find_maxima(capacity=cap, out=outs[k], count=cnts[k:k + 1], stream=sts[c])
        for c in range(C):
            ctxs[c].matrix_into(Ms[c], stream=sts[c])
        torch.cuda.synchronize()
        for c in ctxs:
            c.sync()
        got_n = cnts.cpu().numpy()
        for k in range(n_ev):
            _, pk_ref, n_ref = refs[k]
            assert int(got_n[k]) == n_ref, k
            assert_peaks_equal(outs[k].cpu().numpy().view(ht.PEAK_DTYPE)[:n_ref], pk_ref)
        for c in range(C):
            k = n_ev - C + c
            assert np.array_equal(Ms[c].cpu().numpy().view(np.uint32).reshape(b.shape()), refs[k][0]), c
    finally:
        for c in ctxs:
            c.close()


# ---------------------------------------------------------------------------
# The scan alone on hand-built and random matrices
# ---------------------------------------------------------------------------

with open(os.path.join(HERE, "golden", "maxima_cases.json")) as _f:
    GOLD = json.load(_f)


@pytest.mark.parametrize("nb", [6, 8], ids=["nb6_scalar_scan", "nb8_bulk_scan"])
def test_golden_maxima_on_gpu(ht, nb):
    nt, np_, na, nb0 = GOLD["binning"]
    b = ht.Binning(nt, np_, na, nb)
    # a context's threshold is fixed: one context per case
    for case in GOLD["cases"]:
        M = np.zeros(b.shape(), np.uint32)
        for t, p, i, j, v in case["cells"]:
            M[t, p, i, j] = v
        with ht.Context(b, ht.Ranges(), threshold=case["threshold"], max_hits=16) as ctx:
            ctx.set_matrix(M)
            pk, n = ctx.find_maxima(capacity=64)
        got = [[int(q[f]) for f in ("itheta", "iphi", "ia", "ib", "votes")] for q in pk]
        assert got == case["expected"], case["name"]


@pytest.mark.parametrize("shape,vmax,seed", [
    ((2, 3, 300, 64), 4, 0), ((2, 3, 97, 50), 3, 1), ((1, 1, 4096, 1024), 3, 2),
    ((1, 2, 333, 2048), 5, 3), ((3, 1, 50, 7), 3, 4)])
def test_random_matrix_scan(ht, shape, vmax, seed):
    rng = np.random.default_rng(seed)
    M = rng.integers(0, vmax, shape).astype(np.uint32)
    b = ht.Binning(*shape)
    for T in (1, vmax - 1):
        ref, n_ref = oracle.find_maxima(_ob(b), oracle.Ranges(), M, T)
        with ht.Context(b, ht.Ranges(), threshold=T, max_hits=1) as ctx:
            ctx.set_matrix(M)
            pk, n = ctx.find_maxima(capacity=n_ref + 10)
            pk2, n2 = ctx.find_maxima(capacity=n_ref + 10)      # counters reset between scans
        assert n == n_ref == n2
        assert_peaks_equal(pk, ref)
        assert_peaks_equal(pk2, ref)


# ---------------------------------------------------------------------------
# Full-size upgrade binning (8 x 32 x 2048 x 2048, a 4 GiB matrix)
# ---------------------------------------------------------------------------

def test_upgrade_full_size_complete(ht):
    """One 50 000-hit upgrade event: the whole 4 GiB M_H (all 256 slices,
    compared slice group by slice group on the host) and the whole peak list
    equal the oracle's fill and maxima (Sec. 2, binning scaled up)."""
    import torch
    b, r = ht.Binning(*synth.UPGRADE_BINNING), ht.Ranges()
    ev = synth.upgrade_event(0)
    ob, orr = _ob(b), _orr(r)
    M_ref, votes_ref = oracle.fill(ob, orr, ev.x, ev.y, ev.z)
    pk_ref, n_ref = oracle.find_maxima(ob, orr, M_ref, 10)
    assert votes_ref > 50_000_000 and n_ref > 1000
    with ht.Context(b, r, threshold=10, max_hits=ev.n_hits) as ctx:
        ctx.fill(*(torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z)))
        Md = torch.empty(b.n_cells, dtype=torch.int32, device="cuda")
        ctx.matrix_into(Md)
        ctx.sync()
        pk, n = ctx.find_maxima(capacity=n_ref + 16)
    Md = Md.view(b.n_slices, b.n_a * b.n_b)
    Mr = M_ref.reshape(b.n_slices, b.n_a * b.n_b)
    group = 16                                  # 256 MiB per host copy
    for s0 in range(0, b.n_slices, group):
        got = Md[s0:s0 + group].cpu().numpy().view(np.uint32)
        if not np.array_equal(got, Mr[s0:s0 + group]):
            bad = np.argwhere(got != Mr[s0:s0 + group])[0]
            pytest.fail(f"M_H differs first at slice {s0 + bad[0]}, cell {bad[1]}")
    del Md
    assert n == n_ref
    assert_peaks_equal(pk, pk_ref)


def test_first_fill_right_after_create_on_a_priority_stream(ht):
    """The first fill of a new context, issued at once on a high-priority
    stream of its own: it must not overlap the zeroing of the context's
    buffers (4 GiB M_H, counters, bookkeeping), which creation finishes
    before it returns.  Peaks equal the oracle's."""
    import torch
    b, r = ht.Binning(*synth.UPGRADE_BINNING), ht.Ranges()
    ev = synth.upgrade_event(10)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), ev.x, ev.y, ev.z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, 10)
    del M_ref
    d = [torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z)]
    lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") else (0, -5)
    st = torch.cuda.Stream(priority=min(lo, hi))
    torch.cuda.synchronize()
    for _ in range(2):
        with ht.Context(b, r, threshold=10, max_hits=ev.n_hits) as ctx:
            ctx.fill(*d, stream=st)
            out = torch.empty((n_ref + 16) * 8, dtype=torch.int32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
            ctx.find_maxima(capacity=n_ref + 16, out=out, count=cnt, stream=st)
            st.synchronize()
            assert int(cnt.item()) == n_ref
            pk = out.cpu().numpy().view(ht.PEAK_DTYPE)[:n_ref]
        assert_peaks_equal(pk, pk_ref)


def test_upgrade_full_size_sampled(ht):
    """A second upgrade event: the vote total over all slices and six whole
    slices (the busiest among them) with their peaks."""
    import torch
    b, r = ht.Binning(*synth.UPGRADE_BINNING), ht.Ranges()
    ev = synth.upgrade_event(1)
    ob, orr = _ob(b), _orr(r)
    _, votes_ref = oracle.fill_slices(ob, orr, ev.x, ev.y, ev.z, np.arange(256), count_only=True)
    sl, _ = oracle.admit(ob, orr, ev.x, ev.y, ev.z)
    counts = np.bincount(sl[:, 0][sl[:, 0] >= 0], minlength=256)
    busiest = int(np.argmax(counts))
    sample = sorted({0, 17, 100, 131, 255, busiest})
    Msel, _ = oracle.fill_slices(ob, orr, ev.x, ev.y, ev.z, sample)
    with ht.Context(b, r, threshold=10, max_hits=ev.n_hits) as ctx:
        ctx.fill(*(torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z)))
        Md = torch.empty(b.n_cells, dtype=torch.int32, device="cuda")
        ctx.matrix_into(Md)
        ctx.sync()
        pk, n = ctx.find_maxima(capacity=1 << 20)
    assert int(Md.to(torch.int64).sum().item()) == votes_ref
    Md = Md.view(256, b.n_a * b.n_b)
    for k, s in enumerate(sample):
        got = Md[s].cpu().numpy().view(np.uint32).reshape(b.n_a, b.n_b)
        assert np.array_equal(got, Msel[k]), s
        one = oracle.Binning(1, 1, b.n_a, b.n_b)
        ref, _ = oracle.find_maxima(one, orr, Msel[k], 10)
        mine = pk[(pk["itheta"] * b.n_phi + pk["iphi"]) == s]
        for f in ("ia", "ib", "votes", "a_c", "b_c"):
            assert np.array_equal(mine[f], ref[f]), (s, f)
    # ordering of the whole list: ascending linear index
    lin = ((pk["itheta"].astype(np.int64) * b.n_phi + pk["iphi"]) * b.n_a + pk["ia"]) * b.n_b + pk["ib"]
    assert np.all(np.diff(lin) > 0)


# ---------------------------------------------------------------------------
# Launch shapes never change results
# ---------------------------------------------------------------------------

TUNINGS = [
    dict(), dict(scan_kind=1), dict(scan_kind=2), dict(scan_kind=3),
    dict(scan_kind=1, scan_slots=2, scan_stage_bytes=16384),
    dict(scan_kind=1, scan_slots=8, scan_stage_bytes=24576),
    dict(fill_rows=8, fill_threads=256), dict(fill_rows=64, fill_threads=1024, fill_hits_staged=4096),
    dict(fill_rows=16, fill_blocks_per_sm=1, scan_blocks_per_sm=1, scan_kind=2),
    dict(fill_fused_scan=2, scan_kind=2), dict(fill_fused_scan=2, scan_kind=1),
    dict(fill_fused_scan=1, fill_rows=4, fill_threads=256), dict(fill_fused_scan=3, fill_rows=16),
    dict(fill_fused_scan=3, fill_rows=32, fill_hits_staged=1024),
    dict(fill_fused_scan=4), dict(fill_fused_scan=4, fill_rows=16), dict(fill_fused_scan=4, fill_rows=8, fill_threads=512),
    dict(fill_fused_scan=4, fill_hits_staged=64),
    dict(fill_fused_scan=5), dict(fill_fused_scan=5, fill_rows=16, fill_threads=1024),
    dict(fill_fused_scan=5, fill_rows=4, fill_threads=256), dict(fill_fused_scan=5, fill_hits_staged=64),
    dict(fill_fused_scan=5, fill_rows=2, fill_blocks_per_sm=1), dict(fill_fused_scan=5, fill_rows=8, fill_threads=1024),
    dict(fill_vote_agg=1), dict(fill_fused_scan=5, fill_vote_agg=1, fill_rows=4, fill_threads=256),
    dict(fill_blocks_per_sm=1), dict(bin_cluster=2), dict(bin_cluster=1, fill_blocks_per_sm=1),
    dict(bin_cluster=1, fill_fused_scan=2), dict(bin_cluster=1, fill_fused_scan=4),
]


@pytest.fixture(scope="module")
def paper_ref():
    ev = synth.paper_event(seed=11)
    b = oracle.Binning(*synth.PAPER_BINNING)
    M, _ = oracle.fill(b, oracle.Ranges(), ev.x, ev.y, ev.z)
    pk, n = oracle.find_maxima(b, oracle.Ranges(), M, 10)
    return ev, M, pk, n


@pytest.mark.parametrize("tuning", TUNINGS, ids=[",".join(f"{k}={v}" for k, v in t.items()) or "auto"
                                                 for t in TUNINGS])
def test_tuning_sweep(ht, paper_ref, tuning):
    ev, M_ref, pk_ref, n_ref = paper_ref
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    with ht.Context(b, r, threshold=10, max_hits=ev.n_hits) as ctx:
        ctx.set_tuning(**tuning)
        got = ctx.get_tuning()
        for k, v in tuning.items():
            if k in ("scan_kind", "fill_rows", "fill_threads", "scan_slots", "fill_fused_scan", "fill_vote_agg",
                     "bin_cluster"):
                assert got[k] == v, (k, got)
        ctx.fill(ev.x, ev.y, ev.z)
        pk, n = ctx.find_maxima(capacity=1 << 16)
        assert np.array_equal(ctx.matrix(), M_ref)
    assert n == n_ref
    assert_peaks_equal(pk, pk_ref)


def test_bin_cluster_auto(ht, paper_ref):
    """bin_cluster 0 resolves to one cluster launch for the bulk-copy-tile
    fill at its occupancy and to two launches when fill_blocks_per_sm holds
    the fill below it; either way the peaks are the oracle's."""
    ev, M_ref, pk_ref, n_ref = paper_ref
    with ht.Context(ht.Binning(*synth.PAPER_BINNING), ht.Ranges(), threshold=10, max_hits=ev.n_hits) as ctx:
        assert ctx.get_tuning()["bin_cluster"] == 1
        for tun, want in ((dict(fill_blocks_per_sm=1), 2), (dict(fill_blocks_per_sm=1, bin_cluster=1), 1),
                          (dict(bin_cluster=2), 2), (dict(fill_fused_scan=2), 2)):
            ctx.set_tuning(**tun)
            assert ctx.get_tuning()["bin_cluster"] == want, tun
            ctx.fill(ev.x, ev.y, ev.z)
            pk, n = ctx.find_maxima(capacity=1 << 16)
            assert n == n_ref
            assert_peaks_equal(pk, pk_ref)


def test_bad_tuning_rejected(ht):
    with ht.Context(ht.Binning(*synth.TINY_BINNING), ht.Ranges(), threshold=8, max_hits=256) as ctx:
        for bad in (dict(fill_threads=300), dict(fill_rows=12), dict(scan_kind=9), dict(fill_vote_agg=2),
                    dict(bin_cluster=3)):
            with pytest.raises(ht.HTError):
                ctx.set_tuning(**bad)
        ev = synth.tiny_event()
        ctx.fill(ev.x, ev.y, ev.z)           # still usable with the previous shapes
        assert ctx.find_maxima(capacity=64)[1] > 0


# ---------------------------------------------------------------------------
# The fused fill + maxima path: seams between strips and between CTAs
# ---------------------------------------------------------------------------

FUSED_TUNINGS = [dict(fill_fused_scan=2), dict(fill_fused_scan=1), dict(fill_fused_scan=1, fill_rows=4,
                 fill_threads=256), dict(fill_fused_scan=1, fill_rows=64, fill_threads=1024),
                 dict(fill_fused_scan=1, fill_rows=8, fill_blocks_per_sm=1), dict(fill_fused_scan=3),
                 dict(fill_fused_scan=3, fill_rows=4), dict(fill_fused_scan=3, fill_rows=64),
                 dict(fill_fused_scan=4), dict(fill_fused_scan=4, fill_rows=4),
                 dict(fill_fused_scan=5), dict(fill_fused_scan=5, fill_rows=4), dict(fill_fused_scan=5, fill_rows=16),
                 dict(fill_fused_scan=5, fill_rows=2, fill_threads=256), dict(fill_fused_scan=5, fill_vote_agg=1)]


def _track(A, B, theta, branch):
    import math
    Rr = math.hypot(A, B)
    psi = math.atan2(B, A)
    xs, ys, zs = [], [], []
    for rad in synth.LAYER_RADII:
        ph = psi + branch * math.acos(rad / (2 * Rr))
        xs.append(rad * math.cos(ph)); ys.append(rad * math.sin(ph)); zs.append(rad / math.tan(theta))
    return np.float32(xs), np.float32(ys), np.float32(zs)


@pytest.mark.parametrize("tuning", FUSED_TUNINGS, ids=[str(t) for t in FUSED_TUNINGS])
def test_peaks_on_seams(ht, tuning):
    # tracks whose peaks sit on rows around strip boundaries (rows 3, 4, 7, 8,
    # 31, 32, 63 of a 64-row slice) plus background hits, binning 2x4x64x64
    b, r = ht.Binning(2, 4, 64, 64), ht.Ranges()
    xs, ys, zs = [], [], []
    import math
    for ia, ib, branch in [(40, 29, 1), (31, 29, 1), (32, 29, 1), (3, 40, -1), (4, 41, -1), (7, 45, -1),
                           (8, 46, -1), (63, 52, 1), (20, 45, -1)]:
        A = -2000 + (ia + 0.5) * 62.5
        B = -2000 + (ib + 0.5) * 62.5
        if 2 * math.hypot(A, B) < 1000:
            continue
        x, y, z = _track(A, B, 1.5 * math.pi / 2, branch)
        xs.append(x); ys.append(y); zs.append(z)
    x, y, z = (np.concatenate(v) for v in (xs, ys, zs))
    bx, by, bz = random_hits(300, 21)
    x, y, z = np.concatenate([x, bx]), np.concatenate([y, by]), np.concatenate([z, bz])
    for T in (3, 8, 12):
        M_ref, _ = oracle.fill(_ob(b), _orr(r), x, y, z)
        pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
        with ht.Context(b, r, threshold=T, max_hits=x.size) as ctx:
            ctx.set_tuning(**tuning)
            ctx.fill(x, y, z)
            pk, n = ctx.find_maxima(capacity=4096)
            assert np.array_equal(ctx.matrix(), M_ref)
        assert n == n_ref, (T, n, n_ref)
        assert_peaks_equal(pk, pk_ref)


@pytest.mark.parametrize("tuning", FUSED_TUNINGS[1:4] + FUSED_TUNINGS[5:7] + FUSED_TUNINGS[8:],
                         ids=[str(t) for t in FUSED_TUNINGS[1:4] + FUSED_TUNINGS[5:7] + FUSED_TUNINGS[8:]])
def test_fused_candidate_overflow(ht, paper_ref, tuning):
    # low thresholds on the paper-scale event: some passes list more cells
    # >= T than the fused fill's candidate lists hold (whole-row fallback,
    # also for the pending row of the next pass), others fewer
    ev, M_ref = paper_ref[0], paper_ref[1]
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    for T in (3, 5, 7):
        pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
        with ht.Context(b, r, threshold=T, max_hits=6000) as ctx:
            ctx.set_tuning(**tuning)
            ctx.fill(ev.x, ev.y, ev.z)
            pk, n = ctx.find_maxima(capacity=1 << 20)
        assert n == n_ref, (T, n, n_ref)
        assert_peaks_equal(pk, pk_ref)


@pytest.mark.parametrize("tuning", FUSED_TUNINGS[1:3] + FUSED_TUNINGS[5:6] + FUSED_TUNINGS[8:9],
                         ids=[str(t) for t in FUSED_TUNINGS[1:3] + FUSED_TUNINGS[5:6] + FUSED_TUNINGS[8:9]])
def test_fused_state_sequences(ht, paper_ref, tuning):
    ev, M_ref, pk_ref, n_ref = paper_ref
    ev2 = synth.paper_event(seed=12)
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    M2, _ = oracle.fill(_ob(b), _orr(r), ev2.x, ev2.y, ev2.z)
    pk2, n2 = oracle.find_maxima(_ob(b), _orr(r), M2, 10)
    with ht.Context(b, r, threshold=10, max_hits=6000) as ctx:
        ctx.set_tuning(**tuning)
        # a fused fill consumed twice: the second call rescans M_H
        ctx.fill(ev.x, ev.y, ev.z)
        for _ in range(2):
            pk, n = ctx.find_maxima(capacity=1 << 16)
            assert n == n_ref
            assert_peaks_equal(pk, pk_ref)
        # two fills in a row: only the second counts
        ctx.fill(ev.x, ev.y, ev.z)
        ctx.fill(ev2.x, ev2.y, ev2.z)
        pk, n = ctx.find_maxima(capacity=1 << 16)
        assert n == n2
        assert_peaks_equal(pk, pk2)
        # an unconsumed fused fill, then a matrix set by hand
        ctx.fill(ev.x, ev.y, ev.z)
        ctx.set_matrix(M2)
        pk, n = ctx.find_maxima(capacity=1 << 16)
        assert n == n2
        assert_peaks_equal(pk, pk2)
        # naive and accumulating fills fall back to the standalone scan
        ctx.fill(ev.x, ev.y, ev.z)
        ctx.fill(ev.x[:10], ev.y[:10], ev.z[:10], naive=True)
        ctx.fill(ev.x[10:], ev.y[10:], ev.z[10:], accumulate=True)
        pk, n = ctx.find_maxima(capacity=1 << 16)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)


def test_autotune_keeps_results(ht, paper_ref):
    ev, M_ref, pk_ref, n_ref = paper_ref
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    with ht.Context(b, r, threshold=10, max_hits=6000) as ctx:
        with pytest.raises(ht.HTError):
            ctx.autotune()                        # nothing filled yet
        ctx.fill(ev.x, ev.y, ev.z)
        chosen, us = ctx.autotune(reps=3)
        assert us > 0 and chosen["fill_fused_scan"] in (1, 2, 3, 4, 5)
        assert np.array_equal(ctx.matrix(), M_ref)
        pk, n = ctx.find_maxima(capacity=1 << 16)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)
        # later fills run with the chosen shapes
        ctx.fill(ev.x[::-1].copy(), ev.y[::-1].copy(), ev.z[::-1].copy())
        pk, n = ctx.find_maxima(capacity=1 << 16)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)
        ctx.fill(ev.x[:100], ev.y[:100], ev.z[:100], accumulate=True)
        with pytest.raises(ht.HTError):
            ctx.autotune()                        # last fill accumulated


# ---------------------------------------------------------------------------
# Peaks-only fills: M_H never written, the same peaks
# ---------------------------------------------------------------------------

PEAKS_ONLY_TUNINGS = [dict(), dict(fill_rows=4, fill_threads=256), dict(fill_rows=2, fill_threads=256),
                      dict(fill_rows=64, fill_threads=1024)]


@pytest.mark.parametrize("tuning", PEAKS_ONLY_TUNINGS, ids=[str(t) for t in PEAKS_ONLY_TUNINGS])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_peaks_only_matches_oracle(ht, case, tuning):
    name, bins, rng, T, (x, y, z) = case
    b, r = ht.Binning(*bins), ht.Ranges(**rng)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), x, y, z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
    with ht.Context(b, r, threshold=T, max_hits=max(len(x), 1)) as ctx:
        ctx.set_tuning(**tuning)
        ctx.set_matrix(np.full(b.shape(), 7, np.uint32))      # a marker M_H must keep
        ctx.fill(x, y, z, peaks_only=True)
        pk, n = ctx.find_maxima(capacity=1 << 20)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)
        assert np.all(ctx.matrix() == 7)
        # a normal fill afterwards writes M_H again
        ctx.fill(x, y, z)
        assert np.array_equal(ctx.matrix(), M_ref)


@pytest.mark.parametrize("T", [1, 2, 1 << 20])
def test_threshold_edges_both_fills(ht, T):
    """T = 1 (every voted cell a candidate), T = 2 and a threshold no cell
    reaches: the fused fill and the peaks-only fill both give the oracle's
    peaks.  T = 0 is rejected by the context."""
    name, bins, rng, _, (x, y, z) = CASES[2]
    assert name == "ragged_nb"
    b, r = ht.Binning(*bins), ht.Ranges(**rng)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), x, y, z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
    for po in (False, True):
        with ht.Context(b, r, threshold=T, max_hits=max(len(x), 1)) as ctx:
            ctx.fill(x, y, z, peaks_only=po)
            pk, n = ctx.find_maxima(capacity=1 << 20)
        assert n == n_ref, (po, n, n_ref)
        assert_peaks_equal(pk, pk_ref)
    if T == 1:
        with pytest.raises(ht.HTError):
            ht.Context(b, r, threshold=0, max_hits=16)


def test_peaks_only_low_threshold_and_u32(ht, paper_ref):
    ev, M_ref = paper_ref[0], paper_ref[1]
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    for T in (3, 5):          # passes with more cells >= T than the lists hold
        pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
        with ht.Context(b, r, threshold=T, max_hits=6000) as ctx:
            ctx.fill(ev.x, ev.y, ev.z, peaks_only=True)
            pk, n = ctx.find_maxima(capacity=1 << 20)
        assert n == n_ref, (T, n, n_ref)
        assert_peaks_equal(pk, pk_ref)
    b = ht.Binning(1, 1, 64, 96)    # u32 tiles (half-height passes)
    x, y, z = random_hits(70000, 9, rmax=400.0)
    x[:35000], y[:35000] = np.float32(300.0), np.float32(250.0)
    M2, _ = oracle.fill(_ob(b), _orr(r), x, y, z)
    for tun in (dict(), dict(fill_rows=2, fill_threads=256)):
        pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M2, 3)
        with ht.Context(b, r, threshold=3, max_hits=x.size) as ctx:
            ctx.set_tuning(**tun)
            ctx.fill(x, y, z, peaks_only=True)
            pk, n = ctx.find_maxima(capacity=1 << 20)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)
    with ht.Context(b, r, threshold=3, max_hits=x.size) as ctx:
        with pytest.raises(ht.HTError):
            ctx.fill(x, y, z, peaks_only=True, accumulate=True)


def test_bounded_wait_gives_up_and_context_survives(ht):
    """A device wait that nothing ends (ht_check_wait_timeout) gives up
    after its limit, is reported as HT_E_TIMEOUT, and the context goes on
    working: the next fill and scan are still bit-exact."""
    import time
    ev = synth.tiny_event()
    b = ht.Binning(*synth.TINY_BINNING)
    M_ref, _ = oracle.fill(_ob(b), _orr(ht.Ranges()), ev.x, ev.y, ev.z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(ht.Ranges()), M_ref, 8)
    with ht.Context(b, ht.Ranges(), threshold=8, max_hits=1024) as ctx:
        t0 = time.perf_counter()
        st = ctx.check_wait_timeout(50)
        dt = time.perf_counter() - t0
        assert st == ht.HT_E_TIMEOUT and "wait" in ht.last_error()
        assert dt < 5.0
        assert ctx.check_wait_timeout(0) == ht.HT_E_INVAL
        ctx.fill(ev.x, ev.y, ev.z)
        pk, n = ctx.find_maxima(capacity=1024)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)
        assert np.array_equal(ctx.matrix(), M_ref)


def test_measure_atomics(ht):
    """The L2-atomic roofline helper: a positive rate, an L2-resident
    footprint no slower than one 8x larger, bad sizes refused."""
    small = ht.measure_atomics(32 << 20, 16)
    big = ht.measure_atomics(256 << 20, 16)
    assert small > 1e9 and big > 1e8
    assert small > 0.5 * big
    for fp, per in ((3 << 20, 16), (1024, 16), (32 << 20, 0), (32 << 20, 5000)):
        with pytest.raises(ht.HTError):
            ht.measure_atomics(fp, per)


def test_last_admitted_counts_the_oracle_admissions(ht):
    """ht_last_admitted: the admitted (hit, slice) records of the last fill
    equal the oracle's admission count (windows included)."""
    for name, bins, rng, T, (x, y, z) in (CASES[1], CASES[4]):
        b, r = ht.Binning(*bins), ht.Ranges(**rng)
        _, cnt = oracle.admit(_ob(b), _orr(r), x, y, z)
        with ht.Context(b, r, threshold=T, max_hits=max(len(x), 1)) as ctx:
            assert ctx.last_admitted() == 0
            ctx.fill(x, y, z)
            assert ctx.last_admitted() == int(np.asarray(cnt).sum()), name
