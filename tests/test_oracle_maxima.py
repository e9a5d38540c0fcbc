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
