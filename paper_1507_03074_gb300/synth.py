"""Seeded synthetic events for the Hough-Transform track finder.

This module only draws detector hits; it holds none of the Hough-Transform
arithmetic, so both the CUDA path and the CPU oracle take their inputs from
it.  It stands in for the paper's dataset (Sec. 2: 100 simulated minimum-bias
events, tracks with p_T > 500 MeV, up to 5000 hits on a cylindrical 12-layer
silicon detector centred on the collision point), which is not available.

Detector: 12 barrel layers, radii log-spaced 30..1000 mm, cylinders of
unbounded length.  Tracks: helices from the origin in a 2 T solenoid,
p_T ~ U(0.5, 5) GeV, charge +-1, phi0 ~ U(-pi, pi), eta ~ U(-2.5, 2.5); the
transverse projection is a circle through the origin with centre
(A, B) = q R (sin phi0, -cos phi0), R[mm] = 1000 p_T / (0.3 * 2).  A hit on
the layer of radius r sits at azimuth phi0 - q asin(r / 2R) and
z = 2R asin(r / 2R) sinh(eta); it is smeared by 20 um (Gaussian) along the
layer (r*phi) and in z.  Noise hits sit on a random layer at a uniform
azimuth and |z| < r sinh(2.5).  Hits are shuffled; truth labels are kept.
All coordinates are returned as float32 structure-of-arrays (mm).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

N_LAYERS = 12
LAYER_RADII = 30.0 * (1000.0 / 30.0) ** (np.arange(N_LAYERS) / (N_LAYERS - 1))
B_FIELD_T = 2.0
SMEAR_MM = 0.020
ETA_MAX = 2.5


@dataclass
class Event:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    track_id: np.ndarray          # per hit, -1 for noise
    tracks: dict = field(default_factory=dict)   # per track: pt, q, phi0, eta, a, b

    @property
    def n_hits(self) -> int:
        return int(self.x.size)


def radius_mm(pt_gev):
    return 1000.0 * np.asarray(pt_gev) / (0.3 * B_FIELD_T)


def make_event(n_tracks: int, n_noise: int, seed: int, pt_range=(0.5, 5.0),
               smear_mm: float = SMEAR_MM) -> Event:
    rng = np.random.default_rng(seed)
    pt = rng.uniform(pt_range[0], pt_range[1], n_tracks)
    q = rng.choice(np.array([-1.0, 1.0]), n_tracks)
    phi0 = rng.uniform(-np.pi, np.pi, n_tracks)
    eta = rng.uniform(-ETA_MAX, ETA_MAX, n_tracks)
    R = radius_mm(pt)
    a = q * R * np.sin(phi0)
    b = -q * R * np.cos(phi0)

    r = np.broadcast_to(LAYER_RADII[None, :], (n_tracks, N_LAYERS))
    half = np.arcsin(r / (2.0 * R[:, None]))
    phi = phi0[:, None] - q[:, None] * half
    z = 2.0 * R[:, None] * half * np.sinh(eta)[:, None]
    phi = phi + rng.normal(0.0, 1.0, phi.shape) * (smear_mm / r)
    z = z + rng.normal(0.0, smear_mm, z.shape)
    tx, ty, tz = (r * np.cos(phi)).ravel(), (r * np.sin(phi)).ravel(), z.ravel()
    tid = np.repeat(np.arange(n_tracks), N_LAYERS)

    lay = rng.integers(0, N_LAYERS, n_noise)
    rn = LAYER_RADII[lay]
    pn = rng.uniform(-np.pi, np.pi, n_noise)
    zn = rng.uniform(-1.0, 1.0, n_noise) * rn * np.sinh(ETA_MAX)
    nx, ny = rn * np.cos(pn), rn * np.sin(pn)

    X = np.concatenate([tx, nx])
    Y = np.concatenate([ty, ny])
    Z = np.concatenate([tz, zn])
    T = np.concatenate([tid, -np.ones(n_noise, np.int64)])
    perm = rng.permutation(X.size)
    return Event(x=X[perm].astype(np.float32), y=Y[perm].astype(np.float32),
                 z=Z[perm].astype(np.float32), track_id=T[perm],
                 tracks=dict(pt=pt, q=q, phi0=phi0, eta=eta, a=a, b=b))


# ---------------------------------------------------------------------------
# The five workloads.  Binning tuples are (n_theta, n_phi, n_a, n_b).
# ---------------------------------------------------------------------------

PAPER_BINNING = (4, 16, 1024, 1024)
UPGRADE_BINNING = (8, 32, 2048, 2048)
TINY_BINNING = (2, 4, 64, 64)


def tiny_event() -> Event:
    """10 noiseless tracks (120 hits), seed 0."""
    return make_event(10, 0, seed=0)


def paper_event(seed: int = 1, n_tracks: int = 396, n_noise: int = 238) -> Event:
    """Paper-scale event: 396 tracks (4752 hits) + 238 noise hits = 4990 hits."""
    return make_event(n_tracks, n_noise, seed=seed)


def split_hits(n_hits: int, noise_frac_den: float = 12.6):
    """Tracks/noise split of a hit budget: tracks = floor(N / 12.6), the rest noise."""
    tracks = int(n_hits // noise_frac_den)
    return tracks, n_hits - N_LAYERS * tracks


def batch_events(n_events: int = 100, seed0: int = 1000, lo: int = 500, hi: int = 5000):
    """Uneven batch: hit counts uniform in [lo, hi], seeds seed0 + i."""
    rng = np.random.default_rng(seed0)
    counts = rng.integers(lo, hi + 1, n_events)
    out = []
    for i, n in enumerate(counts):
        t, k = split_hits(int(n))
        out.append(make_event(t, k, seed=seed0 + i))
    return out


def upgrade_event(i: int = 0, n_tracks: int = 3750, n_noise: int = 5000) -> Event:
    """High-occupancy event: 3750 tracks + 5000 noise = 50 000 hits, seed 2000+i."""
    return make_event(n_tracks, n_noise, seed=2000 + i)


def serving_stream(rate_hz: float, n_events: int, seed: int = 3000,
                   median_hits: float = 3000.0, sigma: float = 1.0,
                   clip=(200, 50000), upgrade_frac: float = 0.1):
    """Poisson arrivals: (arrival_s[n], n_hits[n], is_upgrade[n], seeds[n])."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_hz, n_events)
    t = np.cumsum(gaps)
    n = np.clip(np.round(rng.lognormal(np.log(median_hits), sigma, n_events)), clip[0], clip[1])
    up = rng.uniform(0.0, 1.0, n_events) < upgrade_frac
    seeds = seed * 1000 + np.arange(n_events)
    return t, n.astype(np.int64), up, seeds
