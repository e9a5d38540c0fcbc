"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself:
closed-form edge values, exact rational arithmetic, an independent atan2
route to the slice, an analytic vote count, a constructed noiseless track,
and exact invariants.  Paper: arXiv 1507.03074, Sec. 2 (method, binning)
and Sec. 3 (per-A evaluation of B).
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
from oracle import Binning, Ranges
from paper_1507_03074_gb300 import synth
from tests import exact

R = Ranges()
TINY = Binning(*synth.TINY_BINNING)
PAPER = Binning(*synth.PAPER_BINNING)
UPGRADE = Binning(*synth.UPGRADE_BINNING)


# ---------------------------------------------------------------------------
# Edge tables: closed forms of the pseudo-angle at the uniform angle edges
# ---------------------------------------------------------------------------

def test_edges_closed_form():
    # theta = k*pi/4 -> k/2 exactly; phi = -pi + k*pi/2 -> k exactly
    et, ep = oracle.edges(Binning(4, 4, 8, 8), R)
    assert et.tolist() == [0.0, 0.5, 1.0, 1.5, 2.0]
    assert ep.tolist() == [0.0, 1.0, 2.0, 3.0, 4.0]
    # 16 phi bins: phi = -pi + k*pi/8.  Odd k: diamond angle of a direction at
    # pi/8 inside a quadrant is tan(pi/8)/(1+tan(pi/8)) = 1 - 1/sqrt(2).
    _, ep = oracle.edges(PAPER, R)
    q = 1.0 - 1.0 / math.sqrt(2.0)
    for k in range(17):
        want = (k // 2) * 0.5 + (q if k % 2 else 0.0)
        if k % 4 == 3:
            want = (k // 4) + (1.0 - q)       # 3*pi/8 into the quadrant: 1 - (1 - 1/sqrt2)
        assert ep[k] == np.float32(want), (k, ep[k], want)
    # 8 theta bins (upgrade binning): theta = pi/8 -> 1 - 1/sqrt(2)
    et, _ = oracle.edges(UPGRADE, R)
    assert et[1] == np.float32(q) and et[2] == np.float32(0.5) and et[4] == np.float32(1.0)
    assert et[3] == np.float32(1.0 - q) and et[5] == np.float32(1.0 + q)


def test_edges_partial_range_monotone():
    r = Ranges(theta_min=0.3, theta_max=2.9, phi_min=-1.0, phi_max=2.5)
    et, ep = oracle.edges(Binning(7, 9, 4, 4), r)
    assert np.all(np.diff(et) > 0) and np.all(np.diff(ep) > 0)
    # theta 0.3 rad: rho/(z+rho) = sin/(cos+sin)
    assert abs(et[0] - math.sin(0.3) / (math.cos(0.3) + math.sin(0.3))) < 1e-7


# ---------------------------------------------------------------------------
# Slice admission: pseudo-angle bins == atan2 bins away from edges
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("binning", [TINY, PAPER, UPGRADE])
def test_slice_matches_atan2(binning):
    ev = synth.paper_event(seed=7)
    rng = np.random.default_rng(5)
    # add hits exactly on bin edges and on the axes
    ang = np.concatenate([np.arange(binning.n_phi + 1) * (2 * np.pi / binning.n_phi) - np.pi,
                          rng.uniform(-np.pi, np.pi, 200)])
    ex = (300 * np.cos(ang)).astype(np.float32)
    ey = (300 * np.sin(ang)).astype(np.float32)
    ez = rng.uniform(-3000, 3000, ang.size).astype(np.float32)
    x = np.concatenate([ev.x, ex]); y = np.concatenate([ev.y, ey]); z = np.concatenate([ev.z, ez])
    sl, cnt = oracle.admit(binning, R, x, y, z)
    assert np.all(cnt == 1)
    bad = 0
    for h in range(x.size):
        it, ip, near = exact.slice_by_atan2(x[h], y[h], z[h], binning.n_theta, binning.n_phi)
        if near:
            continue
        if sl[h, 0] != it * binning.n_phi + ip:
            bad += 1
    assert bad == 0


def test_admission_windows_and_drops():
    b = Binning(4, 8, 16, 16, win_theta=1, win_phi=1)
    # hit in theta bin 0 (near +z), phi bin 0 (just above -pi): theta window clips, phi wraps
    x, y, z = np.float32([-100.0]), np.float32([-1.0]), np.float32([1000.0])
    sl, cnt = oracle.admit(b, R, x, y, z)
    assert cnt[0] == 2 * 3
    got = sorted(sl[0, :cnt[0]].tolist())
    assert got == sorted([t * 8 + p for t in (0, 1) for p in (7, 0, 1)])
    # window wider than the axis -> every phi bin once
    b2 = Binning(2, 4, 8, 8, win_theta=0, win_phi=3)
    sl, cnt = oracle.admit(b2, R, np.float32([50.0]), np.float32([10.0]), np.float32([0.0]))
    assert cnt[0] == 4 and sorted(sl[0, :4].tolist()) == [4, 5, 6, 7]
    # rho == 0 and NaN hits are dropped; a partial phi range drops hits outside it
    sl, cnt = oracle.admit(TINY, R, np.float32([0.0, np.nan]), np.float32([0.0, 1.0]),
                           np.float32([5.0, 1.0]))
    assert cnt.tolist() == [0, 0]
    rp = Ranges(phi_min=0.0, phi_max=1.0)
    sl, cnt = oracle.admit(Binning(2, 4, 8, 8), rp, np.float32([1.0, -1.0]), np.float32([1.0, 0.1]),
                           np.float32([0.0, 0.0]))
    assert cnt.tolist() == [1, 0]


def test_admission_at_the_limits():
    """Non-finite and extreme coordinates follow the pseudo-angle formulas:
    z = +inf gives rho / (z + rho) = 0, the polar angle's limit (the hit
    votes exactly as at any large finite z in theta bin 0); z = -inf gives
    inf / inf = NaN and drops the hit, as x^2 + y^2 overflowing to inf
    (rho = inf: NaN pseudo-angles) and subnormal x, y (x^2 + y^2 underflows
    to 0: rho = 0) do."""
    b = Binning(4, 16, 64, 64)
    x = np.float32([300.0, 300.0, 300.0, 1e30, 1e-40, 300.0])
    y = np.float32([-200.0, -200.0, -200.0, 1e30, 1e-40, -200.0])
    z = np.float32([np.inf, 1e6, -np.inf, 0.0, 0.0, -1e6])
    sl, cnt = oracle.admit(b, R, x, y, z)
    assert cnt.tolist() == [1, 1, 0, 0, 0, 1]
    assert sl[0, 0] == sl[1, 0] and sl[0, 0] // b.n_phi == 0        # theta bin 0
    assert sl[5, 0] // b.n_phi == b.n_theta - 1                        # z = -1e6: the last theta bin
    M_inf, v_inf = oracle.fill(b, R, x[:1], y[:1], z[:1])
    M_big, v_big = oracle.fill(b, R, x[1:2], y[1:2], z[1:2])
    assert v_inf == v_big > 0 and np.array_equal(M_inf, M_big)
    _, v_drop = oracle.fill(b, R, x[2:5], y[2:5], z[2:5])
    assert v_drop == 0


# ---------------------------------------------------------------------------
# P-c: exact rational brute force of every (hit, A) vote on the tiny config
# ---------------------------------------------------------------------------

def _single_hit_votes(b, r, x, y, z):
    M, _ = oracle.fill(b, r, np.float32([x]), np.float32([y]), np.float32([z]))
    nz = np.argwhere(M)
    return {(int(s0) * b.n_phi + int(s1), int(i)): (int(j), int(M[s0, s1, i, j]))
            for s0, s1, i, j in nz}


def test_bruteforce_exact_tiny():
    ev = synth.tiny_event()
    b = TINY
    A = exact.a_centres_exact(b.n_a, R.a_min, R.a_max)
    db = (exact.frac(R.b_max) - exact.frac(R.b_min)) / b.n_b
    bmin = exact.frac(R.b_min)
    mismatches, flagged = 0, 0
    for h in range(ev.n_hits):
        x, y, z = ev.x[h], ev.y[h], ev.z[h]
        it, ip, near = exact.slice_by_atan2(x, y, z, b.n_theta, b.n_phi)
        assert not near
        s = it * b.n_phi + ip
        got = _single_hit_votes(b, R, x, y, z)
        for i in range(b.n_a):
            t = exact.t_exact(x, y, A[i], bmin, db)
            want = math.floor(t) if (t is not None and 0 <= t < b.n_b) else None
            have = got.get((s, i))
            have_j = have[0] if have else None
            if have:
                assert have[1] == 1
            if have_j != want:
                tol = exact.t_tolerance(x, y, A[i], R.b_min, db, t)
                assert exact.near_integer(t, tol), (h, i, have_j, want, float(t))
                flagged += 1
            mismatches += have_j != want
        # no vote outside the hit's slice
        assert all(k[0] == s for k in got)
    assert mismatches == flagged and mismatches <= 3


def test_bruteforce_exact_random_geometry():
    # odd ranges: non-power-of-two bins, asymmetric A/B windows
    b = Binning(3, 5, 37, 29)
    r = Ranges(a_min=-1500.0, a_max=1700.0, b_min=-900.0, b_max=2100.0)
    rng = np.random.default_rng(11)
    n = 40
    rad = rng.uniform(20, 1100, n)
    ph = rng.uniform(-np.pi, np.pi, n)
    x = (rad * np.cos(ph)).astype(np.float32)
    y = (rad * np.sin(ph)).astype(np.float32)
    z = rng.uniform(-2000, 2000, n).astype(np.float32)
    da = (exact.frac(r.a_max) - exact.frac(r.a_min)) / b.n_a
    # the oracle's A centres are exact here only if dA is; use its float values
    A = [exact.frac(np.float32(np.float32(r.a_min) + np.float32(np.float32(i + 0.5) * np.float32(da))))
         for i in range(b.n_a)]
    db_f = np.float32((np.float32(r.b_max) - np.float32(r.b_min)) / np.float32(b.n_b))
    db = exact.frac(db_f)
    bmin = exact.frac(r.b_min)
    flagged = 0
    for h in range(n):
        it, ip, near = exact.slice_by_atan2(x[h], y[h], z[h], b.n_theta, b.n_phi)
        if near:
            continue
        s = it * b.n_phi + ip
        got = _single_hit_votes(b, r, x[h], y[h], z[h])
        for i in range(b.n_a):
            t = exact.t_exact(x[h], y[h], A[i], bmin, db)
            want = math.floor(t) if (t is not None and 0 <= t < b.n_b) else None
            have = got.get((s, i))
            have_j = have[0] if have else None
            if have_j != want:
                tol = exact.t_tolerance(x[h], y[h], A[i], r.b_min, db, t)
                assert exact.near_integer(t, tol), (h, i, have_j, want, float(t))
                flagged += 1
    assert flagged <= 3


# ---------------------------------------------------------------------------
# P-b: the total vote count equals the analytic count of in-range pairs
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["tiny", "paper"])
def test_total_votes_analytic(which):
    if which == "tiny":
        ev, b = synth.tiny_event(), TINY
    else:
        ev, b = synth.paper_event(seed=1), PAPER
    M, votes = oracle.fill(b, R, ev.x, ev.y, ev.z)
    assert int(M.sum(dtype=np.uint64)) == votes
    _, cnt = oracle.admit(b, R, ev.x, ev.y, ev.z)
    analytic = 0
    for h in range(ev.n_hits):
        if cnt[h]:
            analytic += int(cnt[h]) * exact.analytic_votes_one_hit(
                ev.x[h], ev.y[h], b.n_a, R.a_min, R.a_max, R.b_min, R.b_max)
    # FP32 may move a vote across b_min / b_max only when B* is within rounding of it
    diff = votes - analytic
    assert abs(diff) <= 2, (votes, analytic)


def test_total_votes_boundary_cases():
    b = Binning(1, 1, 64, 64)
    r = Ranges(theta_min=0.0, theta_max=float(np.float32(np.pi)))
    # hits on the x axis (y -> B is independent of A), on the y axis, at y = 0
    # x = 0: B = y/2 for every A, so y = +-4000 puts B exactly on b_max (dropped,
    # half-open range) or b_min (kept, bin 0)
    for (x, y) in [(0.0, 500.0), (0.0, -700.0), (300.0, 0.0), (123.25, 1e-3), (-800.0, 45.5),
                   (0.0, 4000.0), (0.0, -4000.0), (0.0, 3999.0)]:
        _, v = oracle.fill(b, r, np.float32([x]), np.float32([y]), np.float32([0.0]))
        want = exact.analytic_votes_one_hit(x, y, b.n_a, r.a_min, r.a_max, r.b_min, r.b_max)
        assert v == want, (x, y, v, want)
    # B exactly on an interior edge b_min + k dB lands in bin k
    M, v = oracle.fill(b, r, np.float32([0.0]), np.float32([2 * (-2000.0 + 17 * 62.5)]),
                       np.float32([0.0]))
    assert v == 64 and np.all(M[0, 0, :, 17] == 1)


# ---------------------------------------------------------------------------
# P-a: a single noiseless track peaks at its true cell with one vote per layer
# ---------------------------------------------------------------------------

def _track_hits(A, B, theta, branch=+1):
    Rr = math.hypot(A, B)
    psi = math.atan2(B, A)
    xs, ys, zs = [], [], []
    for r in synth.LAYER_RADII:
        ph = psi + branch * math.acos(r / (2 * Rr))
        xs.append(r * math.cos(ph)); ys.append(r * math.sin(ph)); zs.append(r / math.tan(theta))
    return np.float32(xs), np.float32(ys), np.float32(zs)


def _true_cell_setup(b, ia, ib, branch):
    da = (R.a_max - R.a_min) / b.n_a
    db = (R.b_max - R.b_min) / b.n_b
    A = R.a_min + (ia + 0.5) * da
    B = R.b_min + (ib + 0.5) * db
    theta = 1.5 * math.pi / b.n_theta
    x, y, z = _track_hits(A, B, theta, branch)
    assert np.all(np.hypot(x, y) > 0)
    M, votes = oracle.fill(b, R, x, y, z)
    sl, cnt = oracle.admit(b, R, x, y, z)
    assert np.all(cnt == 1) and np.unique(sl[:, 0]).size == 1, "track must sit in one slice"
    it, ip = divmod(int(sl[0, 0]), b.n_phi)
    assert it == int(theta / (math.pi / b.n_theta))
    return M, it, ip, A, B


# parameters chosen so that all 12 hits share one (theta, phi) slice and the
# 12 hit lines B(A) cross steeply enough for a one-cell peak
@pytest.mark.parametrize("binning,ia,ib,branch", [
    (TINY, 40, 29, +1), (TINY, 20, 45, -1), (TINY, 25, 20, +1), (TINY, 44, 40, -1),
    (PAPER, 40, 30, -1), (PAPER, 40, 297, -1)])
def test_single_track_peak(binning, ia, ib, branch):
    b = binning
    M, it, ip, A, B = _true_cell_setup(b, ia, ib, branch)
    assert M[it, ip, ia, ib] == 12                 # one vote per layer
    assert M.max() == 12
    peaks, n = oracle.find_maxima(b, R, M, 12)
    assert n == 1
    p = peaks[0]
    assert (p["itheta"], p["iphi"], p["ia"], p["ib"], p["votes"]) == (it, ip, ia, ib, 12)
    assert p["a_c"] == np.float32(A) and p["b_c"] == np.float32(B)


@pytest.mark.parametrize("ia,ib,branch", [(40, 475, -1), (40, 653, -1), (40, 920, -1), (40, 564, +1)])
def test_single_stiff_track_ridge(ia, ib, branch):
    # a stiff track's hit lines are nearly parallel: the 12-vote region is a
    # ridge; the true cell holds 12 and the single peak lies on its ridge
    b = PAPER
    M, it, ip, _, _ = _true_cell_setup(b, ia, ib, branch)
    assert M[it, ip, ia, ib] == 12 and M.max() == 12
    S = M[it, ip]
    comp, todo = {(ia, ib)}, [(ia, ib)]
    while todo:
        i, j = todo.pop()
        for di in (-1, 0, 1):
            for dj in (-1, 0, 1):
                q = (i + di, j + dj)
                if 0 <= q[0] < b.n_a and 0 <= q[1] < b.n_b and q not in comp and S[q] == 12:
                    comp.add(q); todo.append(q)
    peaks, n = oracle.find_maxima(b, R, M, 12)
    assert all((int(p["ia"]), int(p["ib"])) in comp for p in peaks)
    assert n == 1
    # the tie rule puts it at the ridge's smallest linear index
    assert (int(peaks[0]["ia"]), int(peaks[0]["ib"])) == min(comp)


# ---------------------------------------------------------------------------
# P-d: FP32 vs FP64 B-bin rule: rare, one-bin moves, each within rounding
# ---------------------------------------------------------------------------

def test_fp32_vs_fp64_bins():
    ev = synth.paper_event(seed=1)
    st, diffs = oracle.bins_f32_vs_f64(PAPER, R, ev.x, ev.y, ev.z)
    assert st["candidates"] == 1024 * ev.n_hits          # every hit admitted once
    assert st["ndiff"] / st["candidates"] < 1e-4
    assert st["maxdist"] <= 1
    A = exact.a_centres_exact(PAPER.n_a, R.a_min, R.a_max)
    db = (exact.frac(R.b_max) - exact.frac(R.b_min)) / PAPER.n_b
    for h, i, b32, b64 in diffs:
        t = exact.t_exact(ev.x[h], ev.y[h], A[i], exact.frac(R.b_min), db)
        tol = exact.t_tolerance(ev.x[h], ev.y[h], A[i], R.b_min, db, t)
        assert exact.near_integer(t, tol), (h, i, b32, b64, float(t))


# ---------------------------------------------------------------------------
# P-e: invariants
# ---------------------------------------------------------------------------

def test_permutation_and_linearity():
    ev = synth.paper_event(seed=3, n_tracks=60, n_noise=40)
    b = Binning(4, 16, 128, 128)
    M1, v1 = oracle.fill(b, R, ev.x, ev.y, ev.z)
    perm = np.random.default_rng(0).permutation(ev.n_hits)
    M2, v2 = oracle.fill(b, R, ev.x[perm], ev.y[perm], ev.z[perm])
    assert v1 == v2 and np.array_equal(M1, M2)
    k = ev.n_hits // 3
    M3, _ = oracle.fill(b, R, ev.x[:k], ev.y[:k], ev.z[:k])
    M3, _ = oracle.fill(b, R, ev.x[k:], ev.y[k:], ev.z[k:], M=M3)
    assert np.array_equal(M1, M3)


def test_mirror_symmetry():
    # (x, y) -> (-x, -y): A -> -A, B -> -B, phi -> phi + pi.  With symmetric
    # A/B ranges the cell (t, p, i, j) maps to (t, p + n_phi/2, N_A-1-i, N_B-1-j)
    # except votes whose B* is within rounding of a bin edge.
    ev = synth.paper_event(seed=4, n_tracks=80, n_noise=20)
    b = Binning(4, 16, 256, 256)
    M, v = oracle.fill(b, R, ev.x, ev.y, ev.z)
    Mm, vm = oracle.fill(b, R, -ev.x, -ev.y, ev.z)
    Mmap = np.roll(Mm, -b.n_phi // 2, axis=1)[:, :, ::-1, ::-1]
    d = np.abs(M.astype(np.int64) - Mmap.astype(np.int64)).sum()
    assert d <= 1e-4 * v, (d, v)


def test_fill_slices_equals_full_fill():
    # the slice-restricted fill (used for sampled full-size checks) is the
    # pinned full fill restricted to those slices
    ev = synth.paper_event(seed=9, n_tracks=120, n_noise=30)
    b = Binning(4, 16, 64, 128, win_theta=1, win_phi=1)
    M, v = oracle.fill(b, R, ev.x, ev.y, ev.z)
    sel = [0, 5, 17, 63, 40]
    Ms, vs = oracle.fill_slices(b, R, ev.x, ev.y, ev.z, sel)
    flat = M.reshape(b.n_slices, b.n_a, b.n_b)
    for k, s in enumerate(sel):
        assert np.array_equal(Ms[k], flat[s])
    assert vs == int(flat[sel].sum())
    _, vall = oracle.fill_slices(b, R, ev.x, ev.y, ev.z, np.arange(b.n_slices), count_only=True)
    assert vall == v
