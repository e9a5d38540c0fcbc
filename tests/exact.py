"""Independent checkers that pin the oracle (exact rationals and double-precision angles).

None of this calls the oracle: it recomputes what the paper's definitions fix
(Sec. 2: the circle x^2 + y^2 - 2Ax - 2By = 0 through hit and interaction point,
one vote per (theta, phi, A) for the B it gives) in exact rational arithmetic on
the exact float32 inputs, so that an error anywhere in the oracle's FP32 path
(a dropped term, a wrong sign, a transposed operand, a wrong bin index) shows up
as a disagreement that rounding cannot explain.
"""
from __future__ import annotations

import math
from fractions import Fraction as F

import numpy as np

U = 2.0 ** -24          # unit roundoff of binary32


def frac(v) -> F:
    return F(float(np.float32(v)))


def a_centres_exact(n_a, a_min, a_max):
    """Exact bin centres a_min + (i + 1/2)(a_max - a_min)/N_A as rationals."""
    lo, hi = frac(a_min), frac(a_max)
    d = (hi - lo) / n_a
    return [lo + (F(2 * i + 1, 2)) * d for i in range(n_a)]


def t_exact(x, y, A, b_min, db):
    """Exact (B* - b_min) / dB with B* = (x^2 + y^2 - 2 A x) / (2 y); None if y == 0."""
    X, Y = frac(x), frac(y)
    if Y == 0:
        return None
    B = (X * X + Y * Y - 2 * A * X) / (2 * Y)
    return (B - b_min) / db


def t_tolerance(x, y, A, b_min, db, t):
    """A bound (with a 2x safety factor) on |t_fp32 - t_exact| for the FP32 op order
    r2 = x*x + y*y; num = r2 - (2A)*x; B = num / (2y); t = (B - b_min) / dB."""
    xf, yf, Af = abs(float(x)), abs(float(y)), abs(float(A))
    K = xf * xf + yf * yf
    e_num = 4 * U * (K + 2 * Af * xf) + 1.01 * U * abs(K - 2 * float(A) * float(x))
    Bv = abs(float(t)) * float(db) + abs(float(b_min))
    e_B = e_num / (2 * yf) + 2 * U * Bv
    e_t = (e_B + 2 * U * (Bv + abs(float(b_min)))) / float(db) + 2 * U * abs(float(t))
    return 2.0 * e_t + 1e-30


def near_integer(t: F, tol: float, ints=None) -> bool:
    """Is the rational t within tol of an integer (or of one of ``ints``)?"""
    if ints is None:
        k = round(t)
        return abs(float(t - k)) <= tol
    return any(abs(float(t - k)) <= tol for k in ints)


# ---------------------------------------------------------------------------
# Angles in double precision via atan2 (an independent route to the slice)
# ---------------------------------------------------------------------------

def slice_by_atan2(x, y, z, n_theta, n_phi, theta_rng=(0.0, math.pi), phi_rng=(-math.pi, math.pi),
                   edge_tol=1e-5):
    """(itheta, iphi, near_edge) from the polar angle atan2(rho, z) and the azimuth
    atan2(y, x) in double; near_edge flags hits within edge_tol rad of a bin edge."""
    x, y, z = float(x), float(y), float(z)
    rho = math.hypot(x, y)
    th = math.atan2(rho, z)
    ph = math.atan2(y, x)
    if ph >= math.pi:
        ph -= 2 * math.pi
    dth = (theta_rng[1] - theta_rng[0]) / n_theta
    dph = (phi_rng[1] - phi_rng[0]) / n_phi
    ft = (th - theta_rng[0]) / dth
    fp = (ph - phi_rng[0]) / dph
    it = min(max(int(math.floor(ft)), 0), n_theta - 1)
    ip = min(max(int(math.floor(fp)), 0), n_phi - 1)
    near = (abs(ft - round(ft)) * dth < edge_tol) or (abs(fp - round(fp)) * dph < edge_tol)
    return it, ip, near


# ---------------------------------------------------------------------------
# Analytic vote count of one hit (P-b)
# ---------------------------------------------------------------------------

def analytic_votes_one_hit(x, y, n_a, a_min, a_max, b_min, b_max):
    """Number of A bin centres A_i whose exact B*(A_i) lies in [b_min, b_max).

    B*(A) = (K - 2 A X) / (2 Y) is linear in A, so the admissible A form one
    interval; count the centres A_i = a_min + (i + 1/2) dA inside it in closed
    form (no loop over A)."""
    X, Y = frac(x), frac(y)
    lo, hi = frac(a_min), frac(a_max)
    dA = (hi - lo) / n_a
    bl, bh = frac(b_min), frac(b_max)
    if Y == 0:
        return 0
    K = X * X + Y * Y
    if X == 0:
        B = K / (2 * Y)
        return n_a if bl <= B < bh else 0
    # b_l <= (K - 2AX)/(2Y) < b_h  <=>  p_l <= K - 2AX < p_h   (for Y > 0; flipped for Y < 0)
    if Y > 0:
        p_l, p_h, incl_l, incl_h = 2 * Y * bl, 2 * Y * bh, True, False
    else:
        p_l, p_h, incl_l, incl_h = 2 * Y * bh, 2 * Y * bl, False, True
    # p_l (<= or <) K - 2AX (< or <=) p_h  ->  bounds on A
    # K - 2AX >= p_l  <=> A X <= (K - p_l)/2
    c_l, c_h = (K - p_l) / 2, (K - p_h) / 2      # A X <= c_l ; A X > c_h  (with the incl flags)
    if X > 0:
        A_hi, hi_incl = c_l / X, incl_l
        A_lo, lo_incl = c_h / X, incl_h
    else:
        A_lo, lo_incl = c_l / X, incl_l
        A_hi, hi_incl = c_h / X, incl_h
    # centres: i + 1/2 = (A - lo)/dA  ->  i in [ (A_lo - lo)/dA - 1/2 , (A_hi - lo)/dA - 1/2 ]
    u_lo = (A_lo - lo) / dA - F(1, 2)
    u_hi = (A_hi - lo) / dA - F(1, 2)
    i_lo = math.ceil(u_lo) if lo_incl else math.floor(u_lo) + 1
    i_hi = math.floor(u_hi) if hi_incl else math.ceil(u_hi) - 1
    i_lo = max(i_lo, 0)
    i_hi = min(i_hi, n_a - 1)
    return max(0, i_hi - i_lo + 1)


# ---------------------------------------------------------------------------
# The maxima rule, restated directly on a numpy array (cross-check for P-f)
# ---------------------------------------------------------------------------

def maxima_bruteforce(M: np.ndarray, threshold: int):
    """List of (itheta, iphi, ia, ib, votes) in ascending linear order."""
    nt, np_, na, nb = M.shape
    out = []
    for t in range(nt):
        for p in range(np_):
            S = M[t, p].astype(np.int64)
            for i in range(na):
                for j in range(nb):
                    v = S[i, j]
                    if v < threshold:
                        continue
                    ok = True
                    for di in (-1, 0, 1):
                        for dj in (-1, 0, 1):
                            if di == 0 and dj == 0:
                                continue
                            ii, jj = i + di, j + dj
                            if not (0 <= ii < na and 0 <= jj < nb):
                                continue
                            w = S[ii, jj]
                            earlier = (ii * nb + jj) < (i * nb + j)
                            if (earlier and not v > w) or (not earlier and not v >= w):
                                ok = False
                    if ok:
                        out.append((t, p, i, j, int(v)))
    return out
