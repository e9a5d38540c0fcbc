"""P-f: the oracle's threshold + local-maxima rule against hand-written cases.

The expected lists in tests/golden/maxima_cases.json were written by hand from
the rule (arXiv 1507.03074 Sec. 2 and Sec. 3 with the tie reading stated in
the fixture); a direct restatement on numpy arrays cross-checks random
matrices with many ties.
"""
import json
import os

import numpy as np
import pytest

import oracle
from oracle import Binning, Ranges
from tests import exact

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "maxima_cases.json")) as f:
    GOLD = json.load(f)
B = Binning(*GOLD["binning"])
R = Ranges()


def _matrix(cells):
    M = np.zeros(B.shape(), np.uint32)
    for t, p, i, j, v in cells:
        M[t, p, i, j] = v
    return M


@pytest.mark.parametrize("case", GOLD["cases"], ids=[c["name"] for c in GOLD["cases"]])
def test_golden_case(case):
    M = _matrix(case["cells"])
    peaks, n = oracle.find_maxima(B, R, M, case["threshold"])
    got = [[int(p[f]) for f in ("itheta", "iphi", "ia", "ib", "votes")] for p in peaks]
    assert got == case["expected"]
    assert n == len(case["expected"])
    assert [list(t) for t in exact.maxima_bruteforce(M, case["threshold"])] == case["expected"]


def test_peak_centres():
    M = _matrix([[0, 1, 4, 0, 9]])
    peaks, _ = oracle.find_maxima(B, R, M, 1)
    da, db = 4000.0 / B.n_a, 4000.0 / B.n_b
    assert peaks[0]["a_c"] == np.float32(-2000 + 4.5 * da)
    assert peaks[0]["b_c"] == np.float32(-2000 + 0.5 * db)


def test_truncation_keeps_first_in_order():
    M = _matrix([[0, 0, 0, 0, 5], [0, 0, 2, 2, 5], [0, 0, 4, 4, 5], [0, 1, 0, 0, 5]])
    peaks, n = oracle.find_maxima(B, R, M, 1, cap=2)
    assert n == 4 and len(peaks) == 2
    assert [(int(p["iphi"]), int(p["ia"])) for p in peaks] == [(0, 0), (0, 2)]


@pytest.mark.parametrize("seed", range(6))
def test_random_ties_vs_restatement(seed):
    rng = np.random.default_rng(seed)
    b = Binning(2, 3, 9, 11)
    M = rng.integers(0, 4, b.shape()).astype(np.uint32)     # small range: many ties
    for T in (1, 2, 3):
        peaks, n = oracle.find_maxima(b, R, M, T)
        got = [tuple(int(p[f]) for f in ("itheta", "iphi", "ia", "ib", "votes")) for p in peaks]
        assert got == exact.maxima_bruteforce(M, T)
        # invariants of the rule: no two peaks are neighbours; every peak >= T
        cells = {(t, p, i, j) for t, p, i, j, _ in got}
        for t, p, i, j, v in got:
            assert v >= T
            for di in (-1, 0, 1):
                for dj in (-1, 0, 1):
                    if (di or dj):
                        assert (t, p, i + di, j + dj) not in cells


# ---------------------------------------------------------------------------
# The 4-D (80-neighbour) variant
# ---------------------------------------------------------------------------

with open(os.path.join(HERE, "golden", "maxima4d_cases.json")) as f:
    GOLD4 = json.load(f)
B4 = Binning(*GOLD4["binning"])


def _restated_4d(M, T):
    """The 4-D rule restated on whole arrays: for every offset d in
    {-1, 0, 1}^4 \\ {0}, the matrix shifted by d (absent cells = -1) must be
    < M where d precedes 0 in linear order and <= M elsewhere."""
    import itertools
    V = M.astype(np.int64)
    ok = V >= T
    P = np.pad(V, 1, constant_values=-1)
    sh = V.shape
    for d in itertools.product((-1, 0, 1), repeat=4):
        if d == (0, 0, 0, 0):
            continue
        W = P[tuple(slice(1 + k, 1 + k + n) for k, n in zip(d, sh))]
        ok &= (V > W) if d < (0, 0, 0, 0) else (V >= W)
    idx = np.argwhere(ok)
    return [(int(t), int(p), int(i), int(j), int(V[t, p, i, j])) for t, p, i, j in idx]


@pytest.mark.parametrize("case", GOLD4["cases"], ids=[c["name"] for c in GOLD4["cases"]])
def test_golden_case_4d(case):
    M = np.zeros(B4.shape(), np.uint32)
    for t, p, i, j, v in case["cells"]:
        M[t, p, i, j] = v
    peaks, n = oracle.find_maxima(B4, R, M, case["threshold"], dims=4)
    got = [[int(p[f]) for f in ("itheta", "iphi", "ia", "ib", "votes")] for p in peaks]
    assert got == case["expected"] and n == len(case["expected"])
    assert [list(t) for t in _restated_4d(M, case["threshold"])] == case["expected"]


@pytest.mark.parametrize("seed", range(4))
def test_random_ties_4d_vs_restatement(seed):
    rng = np.random.default_rng(100 + seed)
    b = Binning(3, 4, 7, 9)
    M = rng.integers(0, 4, b.shape()).astype(np.uint32)
    for T in (1, 2, 3):
        p4, n4 = oracle.find_maxima(b, R, M, T, dims=4)
        got = [tuple(int(p[f]) for f in ("itheta", "iphi", "ia", "ib", "votes")) for p in p4]
        assert got == _restated_4d(M, T) and n4 == len(got)
        # every 4-D peak is a 2-D peak (its 8 slice neighbours are among the 80)
        p2, _ = oracle.find_maxima(b, R, M, T)
        s2 = {tuple(int(p[f]) for f in ("itheta", "iphi", "ia", "ib")) for p in p2}
        assert all(g[:4] in s2 for g in got)
    # one slice: the 4-D rule is the 2-D rule
    b1 = Binning(1, 1, 7, 9)
    M1 = rng.integers(0, 4, b1.shape()).astype(np.uint32)
    a, na = oracle.find_maxima(b1, R, M1, 1, dims=4)
    c, nc = oracle.find_maxima(b1, R, M1, 1)
    assert na == nc and np.array_equal(a, c)
