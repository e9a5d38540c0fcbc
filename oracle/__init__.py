"""CPU oracle for the Hough-Transform track finder (test infrastructure).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never calls it and shares no code with it.

The arithmetic of Steps 1 and 2 lives in ``ht_oracle.c`` (scalar C, compiled
with ``-O2 -ffp-contract=off`` so every float operation is one IEEE binary32
round-to-nearest operation in source order); this module compiles it, loads
it with ctypes and marshals numpy arrays.  The track read-out of the peaks
(``track_params``) is plain numpy in float64.

Paper passages followed (arXiv 1507.03074):
  * Sec. 2: circles x^2 + y^2 - 2Ax - 2By = 0 through hit and interaction
    point; the vote matrix M_H(A,B,theta,phi) is incremented by one; cells
    above a threshold that are local maxima are the tracks.
  * Sec. 2: binning 4 x 16 x 1024 x 1024.
  * Sec. 3: "for each A, the corresponding B is evaluated"; each maxima
    thread compares one element with its neighbours.
  * Sec. 2, Fig. 1: a peak's circle centre (A, B) gives the track's
    rho = sqrt(A^2 + B^2) and varphi = tan^-1(B/A).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ht_oracle.c")
_LIB = os.path.join(_HERE, "libht_oracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile ht_oracle.c into libht_oracle.so (gcc, no contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.ho_edges.argtypes = [P, P, P, P]
        lib.ho_edges.restype = ctypes.c_int
        lib.ho_admit_hits.argtypes = [P, P, P, P, P, ctypes.c_int64, P, P]
        lib.ho_admit_hits.restype = ctypes.c_int
        lib.ho_fill.argtypes = [P, P, P, P, P, ctypes.c_int64, P]
        lib.ho_fill.restype = ctypes.c_int64
        lib.ho_fill_slices.argtypes = [P, P, P, P, P, ctypes.c_int64, P, ctypes.c_int64, P]
        lib.ho_fill_slices.restype = ctypes.c_int64
        lib.ho_find_maxima.argtypes = [P, P, P, ctypes.c_uint32, P, P, ctypes.c_int64]
        lib.ho_find_maxima.restype = ctypes.c_int64
        lib.ho_find_maxima4d.argtypes = [P, P, P, ctypes.c_uint32, P, P, ctypes.c_int64]
        lib.ho_find_maxima4d.restype = ctypes.c_int64
        lib.ho_bins_f32_vs_f64.argtypes = [P, P, P, P, P, ctypes.c_int64, P, P, ctypes.c_int64]
        lib.ho_bins_f32_vs_f64.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass(frozen=True)
class Binning:
    """M_H[theta][phi][A][B] sizes (B fastest) and slice admission windows."""

    n_theta: int
    n_phi: int
    n_a: int
    n_b: int
    win_theta: int = 0
    win_phi: int = 0

    @property
    def n_slices(self) -> int:
        return self.n_theta * self.n_phi

    @property
    def n_cells(self) -> int:
        return self.n_theta * self.n_phi * self.n_a * self.n_b

    def shape(self):
        return (self.n_theta, self.n_phi, self.n_a, self.n_b)


@dataclass(frozen=True)
class Ranges:
    """Angle ranges (rad) and circle-centre ranges (mm)."""

    theta_min: float = 0.0
    theta_max: float = float(np.float32(np.pi))
    phi_min: float = float(np.float32(-np.pi))
    phi_max: float = float(np.float32(np.pi))
    a_min: float = -2000.0
    a_max: float = 2000.0
    b_min: float = -2000.0
    b_max: float = 2000.0


def _bins(b: Binning) -> np.ndarray:
    return np.array([b.n_theta, b.n_phi, b.n_a, b.n_b, b.win_theta, b.win_phi], dtype=np.uint32)


def _rng(r: Ranges) -> np.ndarray:
    return np.array([r.theta_min, r.theta_max, r.phi_min, r.phi_max,
                     r.a_min, r.a_max, r.b_min, r.b_max], dtype=np.float32)


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float32)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def edges(b: Binning, r: Ranges):
    """FP32 pseudo-angle edge tables (theta: n_theta+1, phi: n_phi+1)."""
    lib = _load()
    bb, rr = _bins(b), _rng(r)
    et = np.zeros(b.n_theta + 1, np.float32)
    ep = np.zeros(b.n_phi + 1, np.float32)
    if lib.ho_edges(_p(bb), _p(rr), _p(et), _p(ep)) != 0:
        raise ValueError("bad binning")
    return et, ep


def admit(b: Binning, r: Ranges, x, y, z):
    """Per-hit admitted slices: (slices[n, max_admit] with -1 padding, count[n])."""
    lib = _load()
    x, y, z = _f32(x), _f32(y), _f32(z)
    n = x.size
    nt = min(2 * b.win_theta + 1, b.n_theta)
    np_ = min(2 * b.win_phi + 1, b.n_phi)
    ma = nt * np_
    sl = np.zeros((n, ma), np.uint32)
    cnt = np.zeros(n, np.uint32)
    rc = lib.ho_admit_hits(_p(_bins(b)), _p(_rng(r)), _p(x), _p(y), _p(z), n, _p(sl), _p(cnt))
    assert rc == ma, (rc, ma)
    out = sl.astype(np.int64)
    out[sl == 0xFFFFFFFF] = -1
    return out, cnt


def fill(b: Binning, r: Ranges, x, y, z, M: np.ndarray | None = None):
    """Step 1: vote matrix (uint32, shape (n_theta, n_phi, n_a, n_b)).

    If ``M`` is given it is accumulated into (the linearity invariant).
    Returns (M, votes_cast)."""
    lib = _load()
    x, y, z = _f32(x), _f32(y), _f32(z)
    if M is None:
        M = np.zeros(b.shape(), np.uint32)
    assert M.dtype == np.uint32 and M.flags.c_contiguous and M.size == b.n_cells
    votes = lib.ho_fill(_p(_bins(b)), _p(_rng(r)), _p(x), _p(y), _p(z), x.size, _p(M))
    if votes < 0:
        raise ValueError("bad binning")
    return M, int(votes)


def fill_slices(b: Binning, r: Ranges, x, y, z, slices, count_only: bool = False):
    """Step 1 restricted to the given slice ids (itheta * n_phi + iphi).

    Returns (Msel[len(slices), n_a, n_b] or None, votes cast into those slices)."""
    lib = _load()
    x, y, z = _f32(x), _f32(y), _f32(z)
    sel = np.ascontiguousarray(slices, dtype=np.uint32)
    M = None if count_only else np.zeros((sel.size, b.n_a, b.n_b), np.uint32)
    votes = lib.ho_fill_slices(_p(_bins(b)), _p(_rng(r)), _p(x), _p(y), _p(z), x.size, _p(sel),
                               sel.size, None if M is None else _p(M))
    if votes < 0:
        raise ValueError("bad binning")
    return M, int(votes)


PEAK_DTYPE = np.dtype([("itheta", np.uint32), ("iphi", np.uint32), ("ia", np.uint32),
                       ("ib", np.uint32), ("votes", np.uint32), ("a_c", np.float32),
                       ("b_c", np.float32)])


def find_maxima(b: Binning, r: Ranges, M: np.ndarray, threshold: int, cap: int | None = None, dims: int = 2):
    """Step 2: peaks (structured array, ascending linear index) and total count.
    dims=2: the 8 (A, B) neighbours of the slice; dims=4: the up to 80
    neighbours in (theta, phi, A, B), phi not wrapping."""
    assert dims in (2, 4)
    lib = _load()
    M = np.ascontiguousarray(M, dtype=np.uint32)
    assert M.size == b.n_cells
    if cap is None:
        cap = max(1, M.size // 4 + 1)
        # a cheap exact bound: peaks are pairwise non-adjacent and hold >= T votes
        cap = int(min(cap, int(M.sum(dtype=np.uint64)) // max(1, threshold) + 1))
    ids = np.zeros((cap, 5), np.uint32)
    cen = np.zeros((cap, 2), np.float32)
    fn = lib.ho_find_maxima if dims == 2 else lib.ho_find_maxima4d
    n = fn(_p(_bins(b)), _p(_rng(r)), _p(M), threshold, _p(ids), _p(cen), cap)
    if n < 0:
        raise ValueError("bad binning")
    k = min(n, cap)
    out = np.zeros(k, PEAK_DTYPE)
    for f, col in zip(("itheta", "iphi", "ia", "ib", "votes"), range(5)):
        out[f] = ids[:k, col]
    out["a_c"] = cen[:k, 0]
    out["b_c"] = cen[:k, 1]
    return out, int(n)


def bins_f32_vs_f64(b: Binning, r: Ranges, x, y, z, diff_cap: int = 4096):
    """FP32 vs FP64 B-bin rule over every admitted (hit, slice, A) candidate.

    Returns (stats dict, diffs[k, 4] = (hit, ia, bin32, bin64))."""
    lib = _load()
    x, y, z = _f32(x), _f32(y), _f32(z)
    stats = np.zeros(5, np.int64)
    diffs = np.zeros((diff_cap, 4), np.int64)
    rc = lib.ho_bins_f32_vs_f64(_p(_bins(b)), _p(_rng(r)), _p(x), _p(y), _p(z), x.size,
                                _p(stats), _p(diffs), diff_cap)
    if rc != 0:
        raise ValueError("bad binning")
    st = dict(zip(("candidates", "votes32", "votes64", "ndiff", "maxdist"), map(int, stats)))
    return st, diffs[: min(st["ndiff"], diff_cap)]


def _snap_quarter(a: float) -> float:
    """An angle within 1e-6 of a multiple of pi/4 (in units of pi/4) is that multiple."""
    q = float(a) / (np.pi / 4.0)
    m = round(q)
    return m * (np.pi / 4.0) if abs(q - m) < 1e-6 else float(a)


def track_params(b: Binning, r: Ranges, peaks, b_field_t: float = 2.0) -> dict:
    """Track read-out of peaks in float64 (Sec. 2, Fig. 1).

    The peak's cell centre (A, B) -- a_min + (ia + 1/2) (a_max - a_min) / n_a,
    likewise for B -- is the circle centre: rho = sqrt(A^2 + B^2) is the
    radius and varphi = tan^-1(B/A), taken over four quadrants (atan2), the
    azimuth of the centre.  A unit charge in a solenoid of b_field_t tesla
    has p_T = 0.3 b_field_t rho (GeV, T, m).  theta / phi_c are the centres of
    the peak's polar / azimuth bins and eta = -ln tan(theta / 2).  Returns a
    dict of float64 arrays.
    """
    r = Ranges(*(float(np.float32(v)) for v in (r.theta_min, r.theta_max, r.phi_min, r.phi_max, r.a_min, r.a_max,
                                                  r.b_min, r.b_max)))   # the ranges are binary32 values
    ia = np.asarray(peaks["ia"], np.float64)
    ib = np.asarray(peaks["ib"], np.float64)
    it = np.asarray(peaks["itheta"], np.float64)
    ip = np.asarray(peaks["iphi"], np.float64)
    a = r.a_min + (ia + 0.5) * ((r.a_max - r.a_min) / b.n_a)
    bb = r.b_min + (ib + 0.5) * ((r.b_max - r.b_min) / b.n_b)
    t0, t1 = _snap_quarter(r.theta_min), _snap_quarter(r.theta_max)
    f0, f1 = _snap_quarter(r.phi_min), _snap_quarter(r.phi_max)
    theta = t0 + (it + 0.5) * ((t1 - t0) / b.n_theta)
    rho = np.sqrt(a * a + bb * bb)
    return dict(a=a, b=bb, rho=rho, varphi=np.arctan2(bb, a), pt=0.3 * b_field_t * rho / 1000.0, theta=theta,
                eta=-np.log(np.tan(0.5 * theta)), phi_c=f0 + (ip + 0.5) * ((f1 - f0) / b.n_phi))
