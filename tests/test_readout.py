"""Track read-out of the peaks (Sec. 2, Fig. 1): rho = sqrt(A^2 + B^2),
varphi = tan^-1(B/A), p_T = 0.3 B rho; the oracle's FP64 read-out pinned to
closed forms and to a constructed track, the library's host read-out
(ht_track_params) against it, and the truth matching.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_1507_03074_gb300 import ht, readout, synth

from tests.test_oracle_pins import _true_cell_setup, PAPER, TINY, R


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1507_03074_gb300 import build
    build.build()


def _ob(b):
    return oracle.Binning(b.n_theta, b.n_phi, b.n_a, b.n_b, b.win_theta, b.win_phi)


def _orr(r):
    return oracle.Ranges(r.theta_min, r.theta_max, r.phi_min, r.phi_max, r.a_min, r.a_max, r.b_min, r.b_max)


def _peaks(**cols):
    n = len(next(iter(cols.values())))
    pk = np.zeros(n, ht.PEAK_DTYPE)
    for k, v in cols.items():
        pk[k] = v
    return pk


def test_closed_form_cell():
    # 100 mm cells whose centres are whole: cell (23, 16) is centred on
    # (A, B) = (300, -400): rho = 500 mm, p_T = 0.3 * 2 T * 0.5 m = 0.3 GeV,
    # varphi = -atan(4/3); theta bin 1 of 4 over [0, pi] is centred on 3 pi / 8
    b = oracle.Binning(4, 8, 40, 40)
    r = oracle.Ranges(a_min=-2050.0, a_max=1950.0, b_min=-2050.0, b_max=1950.0)
    pk = _peaks(itheta=[1], iphi=[7], ia=[23], ib=[16], votes=[12])
    t = oracle.track_params(b, r, pk, b_field_t=2.0)
    assert t["a"][0] == 300.0 and t["b"][0] == -400.0
    assert t["rho"][0] == 500.0
    assert t["pt"][0] == pytest.approx(0.3, rel=1e-15)
    assert t["varphi"][0] == pytest.approx(-math.atan(4.0 / 3.0), rel=1e-15)
    assert t["theta"][0] == pytest.approx(3 * math.pi / 8, rel=1e-15)
    assert t["eta"][0] == pytest.approx(-math.log(math.tan(3 * math.pi / 16)), rel=1e-14)
    # phi bin 7 of 8 over [-pi, pi] is centred on 7 pi / 8
    assert t["phi_c"][0] == pytest.approx(7 * math.pi / 8, rel=1e-15)
    # the four quadrants of varphi and a centre on the -A axis
    q = oracle.track_params(b, r, _peaks(itheta=[0] * 4, iphi=[0] * 4, ia=[23, 16, 16, 23], ib=[23, 23, 16, 16]),
                            2.0)
    assert np.allclose(q["varphi"], [math.atan2(300, 300), math.atan2(300, -400), math.atan2(-400, -400),
                                     math.atan2(-400, 300)], rtol=1e-15)
    # p_T scales with the field
    assert oracle.track_params(b, r, pk, 4.0)["pt"][0] == pytest.approx(0.6, rel=1e-15)


@pytest.mark.parametrize("binning,ia,ib,branch", [(TINY, 40, 29, +1), (PAPER, 40, 30, -1)])
def test_constructed_track_reads_out_its_circle(binning, ia, ib, branch):
    # a noiseless track built on the circle with centre (A, B) of cell
    # (ia, ib): the oracle's single peak reads out that very circle
    M, it, ip, A, B = _true_cell_setup(binning, ia, ib, branch)
    peaks, n = oracle.find_maxima(binning, R, M, 12)
    assert n == 1
    t = oracle.track_params(binning, R, peaks)
    assert t["rho"][0] == pytest.approx(math.hypot(A, B), rel=1e-15)
    assert t["varphi"][0] == pytest.approx(math.atan2(B, A), rel=1e-15)
    assert t["pt"][0] == pytest.approx(0.6 * math.hypot(A, B) / 1000.0, rel=1e-15)
    lo = R.theta_min + it * (R.theta_max - R.theta_min) / binning.n_theta
    assert lo <= t["theta"][0] < lo + (R.theta_max - R.theta_min) / binning.n_theta


def test_generator_pt_from_centre():
    # the generator's own relation: |centre| = R(p_T) = p_T / (0.3 * 2 T)
    ev = synth.make_event(50, 0, seed=11)
    rho = np.hypot(ev.tracks["a"], ev.tracks["b"])
    assert np.allclose(0.3 * synth.B_FIELD_T * rho / 1000.0, ev.tracks["pt"], rtol=1e-12)


@pytest.mark.parametrize("bins,rng", [((4, 16, 1024, 1024), {}), ((3, 5, 37, 29), dict(a_min=-1500.0, a_max=1700.0,
                                                                                      b_min=-900.0, b_max=2100.0)),
                                      ((8, 32, 2048, 2048), dict(theta_min=0.4, theta_max=2.6, phi_min=-2.0,
                                                                 phi_max=1.5))])
def test_library_readout_matches_oracle(bins, rng):
    b, r = ht.Binning(*bins), ht.Ranges(**rng)
    g = np.random.default_rng(5)
    n = 500
    pk = _peaks(itheta=g.integers(0, b.n_theta, n), iphi=g.integers(0, b.n_phi, n), ia=g.integers(0, b.n_a, n),
                ib=g.integers(0, b.n_b, n), votes=g.integers(1, 40, n), event=g.integers(0, 7, n))
    got = ht.track_params(b, r, pk, 2.0)
    ref = oracle.track_params(_ob(b), _orr(r), pk, 2.0)
    for k in ("a", "b", "rho", "varphi", "pt", "theta", "eta", "phi_c"):
        assert np.allclose(got[k], ref[k], rtol=1e-13, atol=1e-13), k
    assert np.array_equal(got["votes"], pk["votes"]) and np.array_equal(got["event"], pk["event"])


def test_library_readout_rejects_bad_input():
    b, r = ht.Binning(2, 4, 64, 64), ht.Ranges()
    ok = _peaks(itheta=[1], iphi=[3], ia=[63], ib=[0])
    assert ht.track_params(b, r, ok).size == 1
    assert ht.track_params(b, r, np.zeros(0, ht.PEAK_DTYPE)).size == 0
    for bad in (dict(itheta=[2]), dict(iphi=[4]), dict(ia=[64]), dict(ib=[64])):
        pk = ok.copy()
        for k, v in bad.items():
            pk[k] = v
        with pytest.raises(ht.HTError):
            ht.track_params(b, r, pk)
    for field in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(ht.HTError):
            ht.track_params(b, r, ok, field)


def test_truth_matching_on_oracle_peaks():
    # 40 noiseless tracks with centres in range (p_T 0.5-1 GeV, R < 1.7 m)
    # on 4 x 4 slices: the oracle's peaks, read out, find most findable
    # tracks with per-mille rho and varphi resolutions
    b, r = ht.Binning(4, 4, 512, 512), ht.Ranges()
    ev = synth.make_event(40, 0, seed=21, pt_range=(0.5, 1.0))
    M, _ = oracle.fill(_ob(b), _orr(r), ev.x, ev.y, ev.z)
    pk, n = oracle.find_maxima(_ob(b), _orr(r), M, 8)
    full = np.zeros(len(pk), ht.PEAK_DTYPE)
    for k in pk.dtype.names:
        full[k] = pk[k]
    tr = ht.track_params(b, r, full)
    res = readout.match(tr, ev, b, r, tol=1.5)
    tt = readout.true_tracks(ev, r)
    assert res["findable"] == int(tt["findable"].sum()) == 40
    assert res["peaks"] == n and 0.6 <= res["efficiency"] <= 1.0, res
    assert res["rho_rel_res"] < 0.01 and res["varphi_res"] < 0.005, res
    assert 0.0 <= res["fake_fraction"] <= 1.0 and 0.0 <= res["duplicate_fraction"] <= res["fake_fraction"] + 1.0
    s = readout.summarise([res, res])
    assert s["findable"] == 2 * res["findable"] and s["efficiency"] == res["efficiency"]
    # no peaks: nothing found, nothing fake
    none = readout.match(np.zeros(0, ht.TRACK_DTYPE), ev, b, r)
    assert none["found"] == 0 and none["efficiency"] == 0.0 and none["fake_fraction"] is None
