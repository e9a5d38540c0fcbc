"""The 4-D (80-neighbour) maxima rule on the GPU (HT_MAXIMA_4D) against the
oracle's 4-D rule: every parity case, the hand-written cases through
ht_set_matrix, random tie-heavy matrices, device memory and truncation."""
import json
import os

import numpy as np
import pytest

import oracle
from tests.test_gpu_parity import ht, _ob, _orr, assert_peaks_equal, CASES  # noqa: F401

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_4d_matches_oracle(ht, case):
    name, bins, rng, T, (x, y, z) = case
    b, r = ht.Binning(*bins), ht.Ranges(**rng)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), x, y, z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T, dims=4)
    p2_ref, n2_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, T)
    with ht.Context(b, r, threshold=T, max_hits=max(len(x), 1)) as ctx:
        ctx.fill(x, y, z)
        pk, n = ctx.find_maxima(capacity=1 << 20, four_d=True)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)
        # the 2-D rule on the same fill is unchanged
        pk2, n2 = ctx.find_maxima(capacity=1 << 20)
        assert n2 == n2_ref
        assert_peaks_equal(pk2, p2_ref)


def test_4d_golden_cases_through_set_matrix(ht):
    gold = json.load(open(os.path.join(HERE, "golden", "maxima4d_cases.json")))
    b, r = ht.Binning(*gold["binning"]), ht.Ranges()
    for case in gold["cases"]:
        M = np.zeros(b.shape(), np.uint32)
        for t, p, i, j, v in case["cells"]:
            M[t, p, i, j] = v
        with ht.Context(b, r, threshold=case["threshold"], max_hits=16) as ctx:
            ctx.set_matrix(M)
            pk, n = ctx.find_maxima(capacity=64, four_d=True)
        got = [[int(p[f]) for f in ("itheta", "iphi", "ia", "ib", "votes")] for p in pk]
        assert got == case["expected"], case["name"]


@pytest.mark.parametrize("seed", range(3))
def test_4d_random_ties(ht, seed):
    import torch
    g = np.random.default_rng(300 + seed)
    b, r = ht.Binning(3, 5, 40, 37), ht.Ranges()
    M = g.integers(0, 4, b.shape()).astype(np.uint32)
    for T in (1, 2, 3):
        pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M, T, dims=4)
        with ht.Context(b, r, threshold=T, max_hits=16) as ctx:
            ctx.set_matrix(M)
            pk, n = ctx.find_maxima(capacity=1 << 16, four_d=True)
            assert n == n_ref
            assert_peaks_equal(pk, pk_ref)
            # device memory, and capacities below the total
            out = torch.zeros(8 * 4096, dtype=torch.int32, device="cuda")
            cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
            ctx.find_maxima(capacity=4096, out=out, count=cnt, four_d=True)
            ctx.sync()
            assert int(cnt.item()) == n_ref
            k = min(n_ref, 4096)
            assert_peaks_equal(out.cpu().numpy().view(ht.PEAK_DTYPE)[:k], pk_ref[:k])
            for cap in (1, max(1, n_ref // 2)):
                pk, n = ctx.find_maxima(capacity=cap, four_d=True)
                assert n == n_ref and len(pk) == min(cap, n_ref)
                assert_peaks_equal(pk, pk_ref[:cap])


def test_4d_needs_the_matrix(ht):
    from paper_1507_03074_gb300 import synth
    ev = synth.tiny_event()
    b = ht.Binning(*synth.TINY_BINNING)
    with ht.Context(b, ht.Ranges(), threshold=8, max_hits=ev.n_hits) as ctx:
        ctx.fill(ev.x, ev.y, ev.z, peaks_only=True)
        with pytest.raises(ht.HTError):
            ctx.find_maxima(four_d=True)
        ctx.find_maxima()             # the 2-D rule still works after a peaks-only fill
        ctx.fill(ev.x, ev.y, ev.z)
        ctx.find_maxima(four_d=True)  # and 4-D again once M_H is written
