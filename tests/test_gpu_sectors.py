"""Phi sectors (Sec. 4): one context per sector, merged peaks.  Each
sector's matrix must equal its phi bins of the oracle's unsplit M_H and the
merged peak list must equal the oracle's unsplit list, for every sector
count, with host and device memory, peaks-only fills and truncation."""
import numpy as np
import pytest

import oracle
from paper_1507_03074_gb300 import synth
from tests.test_gpu_parity import ht, _ob, _orr, assert_peaks_equal, random_hits  # noqa: F401

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def paper11():
    ev = synth.paper_event(seed=11)
    b = oracle.Binning(*synth.PAPER_BINNING)
    M, _ = oracle.fill(b, oracle.Ranges(), ev.x, ev.y, ev.z)
    pk, n = oracle.find_maxima(b, oracle.Ranges(), M, 10)
    return ev, M, pk, n


@pytest.mark.parametrize("S", [1, 2, 4, 8, 16])
def test_sectors_equal_unsplit(ht, paper11, S):
    ev, M_ref, pk_ref, n_ref = paper11
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    m = b.n_phi // S
    with ht.Sectors(b, r, threshold=10, n_sectors=S, max_hits=ev.n_hits) as sec:
        sec.fill(ev.x, ev.y, ev.z)
        pk, n = sec.find_maxima(capacity=1 << 16)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)
        for k in (0, S - 1):
            assert np.array_equal(sec.matrix(k), M_ref[:, k * m:(k + 1) * m])
        # peaks-only fills through the sectors: the same peaks
        sec.fill(ev.x, ev.y, ev.z, peaks_only=True)
        pk, n = sec.find_maxima(capacity=1 << 16)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)


def test_sectors_device_memory_and_truncation(ht, paper11):
    import torch
    ev, M_ref, pk_ref, n_ref = paper11
    b, r = ht.Binning(*synth.PAPER_BINNING), ht.Ranges()
    with ht.Sectors(b, r, threshold=10, n_sectors=4, max_hits=ev.n_hits) as sec:
        st = torch.cuda.Stream()
        d = [torch.from_numpy(a).cuda() for a in (ev.x, ev.y, ev.z)]
        out = torch.zeros(4096 * 8, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        for _ in range(3):            # repeated runs on a caller stream
            sec.fill(*d, stream=st)
            sec.find_maxima(capacity=4096, out=out, count=cnt, stream=st)
        st.synchronize()
        assert int(cnt.item()) == n_ref
        got = out.cpu().numpy().view(ht.PEAK_DTYPE)[:n_ref]
        assert_peaks_equal(got, pk_ref)
        # capacities below the total: the unsplit list's first entries
        for cap in (1, 7, n_ref // 3, n_ref - 1):
            pk, n = sec.find_maxima(capacity=cap)
            assert n == n_ref and len(pk) == cap
            assert_peaks_equal(pk, pk_ref[:cap])
        pk, n = sec.find_maxima(capacity=0)
        assert n == n_ref and len(pk) == 0


def test_sectors_partial_range_and_accumulate(ht):
    # a partial phi range with 3 sectors of 2 bins; two accumulated fills
    b, r = ht.Binning(3, 6, 80, 64), ht.Ranges(theta_min=0.4, theta_max=2.6, phi_min=-2.0, phi_max=1.5)
    x, y, z = random_hits(6000, 17, rmax=900.0)
    M_ref, _ = oracle.fill(_ob(b), _orr(r), x, y, z)
    pk_ref, n_ref = oracle.find_maxima(_ob(b), _orr(r), M_ref, 3)
    with ht.Sectors(b, r, threshold=3, n_sectors=3, max_hits=x.size) as sec:
        sec.fill(x[:2500], y[:2500], z[:2500])
        sec.fill(x[2500:], y[2500:], z[2500:], accumulate=True)
        pk, n = sec.find_maxima(capacity=1 << 18)
        assert n == n_ref
        assert_peaks_equal(pk, pk_ref)
        for k in range(3):
            assert np.array_equal(sec.matrix(k), M_ref[:, 2 * k:2 * k + 2])


def test_sectors_reject_bad_arguments(ht):
    b = ht.Binning(4, 16, 64, 64)
    for S in (0, 3, 32):
        with pytest.raises(ht.HTError):
            ht.Sectors(b, n_sectors=S, max_hits=16)
    with pytest.raises(ht.HTError):
        ht.Sectors(ht.Binning(4, 16, 64, 64, 0, 1), n_sectors=4, max_hits=16)
    with ht.Sectors(ht.Binning(4, 16, 64, 64, 0, 1), n_sectors=1, max_hits=16) as sec:   # one sector: a window is fine
        sec.fill(np.zeros(0, np.float32), np.zeros(0, np.float32), np.zeros(0, np.float32))
        pk, n = sec.find_maxima()
        assert n == 0
    with ht.Sectors(b, n_sectors=4, max_hits=16) as sec:
        with pytest.raises(ht.HTError):
            sec.fill(*[np.zeros(17, np.float32)] * 3)
        with pytest.raises(ht.HTError):
            sec.matrix(4)
