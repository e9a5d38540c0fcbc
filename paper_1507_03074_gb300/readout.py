"""Track read-out of the peaks and its efficiency against the generator's truth.

Sec. 2 turns every peak of M_H into a track: its circle centre (A, B) gives
the radius rho = sqrt(A^2 + B^2) and the azimuth varphi = tan^-1(B/A)
(Fig. 1 shows both, with their resolutions against a chi^2 fit).  The
parameters themselves come from the library (``ht.track_params``, FP64 on
the host); this module matches them to the synthetic events' true tracks
and summarises the efficiency, the fake and duplicate fractions and the
rho / varphi resolutions.  The chi^2 fit is not reproduced: there is no
dataset and no fitter.

A true track is *findable* when its centre lies in the A and B ranges and
its polar angle in the theta range.  A peak matches a true track when its
centre is within ``tol`` cells of the true centre in A and in B and its
theta bin is the track's or a neighbour of it.
"""
from __future__ import annotations

import numpy as np

from . import ht


def true_tracks(event, ranges: ht.Ranges):
    """The generator's tracks of an event: centre, radius, varphi, theta and
    whether the track is findable (dict of arrays)."""
    t = event.tracks
    a, b = np.asarray(t["a"], np.float64), np.asarray(t["b"], np.float64)
    theta = 2.0 * np.arctan(np.exp(-np.asarray(t["eta"], np.float64)))
    findable = ((a >= ranges.a_min) & (a < ranges.a_max) & (b >= ranges.b_min) & (b < ranges.b_max) &
                (theta >= ranges.theta_min) & (theta < ranges.theta_max))
    return dict(a=a, b=b, rho=np.hypot(a, b), varphi=np.arctan2(b, a), theta=theta, pt=np.asarray(t["pt"]),
                findable=findable)


def match(tracks, event, binning: ht.Binning, ranges: ht.Ranges, tol: float = 1.5) -> dict:
    """Match read-out tracks (``ht.TRACK_DTYPE``, one event) to the event's
    true tracks; returns counts, fractions and resolutions."""
    tt = true_tracks(event, ranges)
    da = (ranges.a_max - ranges.a_min) / binning.n_a
    db = (ranges.b_max - ranges.b_min) / binning.n_b
    dth = (ranges.theta_max - ranges.theta_min) / binning.n_theta
    idx = np.flatnonzero(tt["findable"])
    n_pk = len(tracks)
    owner = np.full(n_pk, -1, np.int64)      # the true track a peak is matched to
    best = {}
    if n_pk and idx.size:
        pa, pb, pth = tracks["a"], tracks["b"], tracks["theta"]
        for k in idx:
            near = ((np.abs(pa - tt["a"][k]) <= tol * da) & (np.abs(pb - tt["b"][k]) <= tol * db) &
                    (np.abs(pth - tt["theta"][k]) <= 1.5 * dth))
            cand = np.flatnonzero(near)
            if cand.size == 0:
                continue
            d = np.hypot((pa[cand] - tt["a"][k]) / da, (pb[cand] - tt["b"][k]) / db)
            best[k] = int(cand[np.argmin(d)])
            free = cand[owner[cand] < 0]
            owner[free] = k
    n_find = int(idx.size)
    n_found = len(best)
    matched_peaks = int(np.count_nonzero(owner >= 0))
    res = dict(findable=n_find, found=n_found, peaks=n_pk,
               efficiency=(n_found / n_find) if n_find else None,
               fake_fraction=((n_pk - matched_peaks) / n_pk) if n_pk else None,
               duplicate_fraction=((matched_peaks - n_found) / n_pk) if n_pk else None)
    if best:
        ks = np.array(list(best.keys()))
        ps = np.array([best[k] for k in ks])
        drho = (tracks["rho"][ps] - tt["rho"][ks]) / tt["rho"][ks]
        dphi = np.angle(np.exp(1j * (tracks["varphi"][ps] - tt["varphi"][ks])))
        res.update(rho_rel_res=float(np.std(drho)), rho_rel_bias=float(np.mean(drho)),
                   varphi_res=float(np.std(dphi)), varphi_bias=float(np.mean(dphi)))
    return res


def summarise(per_event) -> dict:
    """Totals over events of ``match`` results (efficiency and fractions
    recomputed from the summed counts; resolutions averaged)."""
    f = sum(r["findable"] for r in per_event)
    n = sum(r["found"] for r in per_event)
    p = sum(r["peaks"] for r in per_event)
    fake = sum(r["fake_fraction"] * r["peaks"] for r in per_event if r["peaks"])
    dup = sum(r["duplicate_fraction"] * r["peaks"] for r in per_event if r["peaks"])
    out = dict(events=len(per_event), findable=f, found=n, peaks=p, efficiency=(n / f) if f else None,
               fake_fraction=(fake / p) if p else None, duplicate_fraction=(dup / p) if p else None)
    for key in ("rho_rel_res", "varphi_res"):
        vals = [r[key] for r in per_event if key in r]
        out[key] = float(np.mean(vals)) if vals else None
    return out
