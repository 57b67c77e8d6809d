"""HEALPix RING pixelisation (input synthesis only: the library sees int32 pixels).

Written from the geometry published by Gorski et al. (2005, ApJ 622, 759,
Section 4), for N = N_side:

* 12 N^2 equal-area pixels on 4N - 1 rings of constant z = cos(theta),
  ring r = 1 .. 4N - 1 counted from the north pole.
* Polar caps (|z| > 2/3): the ring that is k rings from the nearer pole
  (k = 1 .. N - 1) has z = +/-(1 - k^2 / (3 N^2)) and 4k pixels with centres
  at phi = (j + 1/2) pi / (2k).
* Equatorial band (N <= r <= 3N): z = 4/3 - 2r / (3N), 4N pixels with centres
  at phi = (j + s/2) pi / (2N), s = 1 when r - N is even, else 0.
* RING order: ring by ring from north to south, increasing phi within a ring.

Point location (my derivation from the same construction).  In the band the
projection (X, Y) = (2 phi / pi, 3 z / 4) is equal-area and the pixels are
squares rotated by 45 degrees: the grid lines are N (X -/+ Y + 1/2) = integer,
so a point lies in the cell (a, b) = floor(N (X - Y + 1/2)), floor(N (X + Y + 1/2)),
on ring r = 2N - (b - a), at position j = (a + b + 1 - N - s) / 2 (mod 4N).
In a cap, with sigma = sqrt(3 (1 - |z|)) and t = frac(X), the grid lines are
N sigma t = integer and N sigma (1 - t) = integer; the cell
(u, v) = floor(N sigma t), floor(N sigma (1 - t)) lies on ring k = u + v + 1
from the pole, at position floor(X) k + u within it.  The two descriptions
agree on |z| = 2/3.

``xp`` is numpy or torch, so the same code runs on the host for small
problems and on a GPU for the 5.4e8-sample all-sky workload.  Pinned by
tests/test_synth_healpix.py: ring sizes and latitudes, the 12 base pixels,
pixel-centre round trips for odd and even N, and equal areas by Monte Carlo.
"""

from __future__ import annotations

import math

import numpy as np


def _is_np(xp):
    return xp is np


def _ifloor(xp, v):
    return np.floor(v).astype(np.int64) if _is_np(xp) else xp.floor(v).to(xp.int64)


def _f64(xp, v):
    return v.astype(np.float64) if _is_np(xp) else v.to(xp.float64)


def n_pixels(nside: int) -> int:
    return 12 * nside * nside


def ring_start(nside: int, r):
    """First RING index of ring r (1 .. 4N - 1), for an int or an integer array."""
    N = nside
    north = 2 * r * (r - 1)
    band = 2 * N * (N - 1) + 4 * N * (r - N)
    k = 4 * N - r
    south = 12 * N * N - 2 * k * (k + 1)
    if isinstance(r, (int, np.integer)):
        return int(north if r < N else (band if r <= 3 * N else south))
    where = np.where if isinstance(r, np.ndarray) else __import__("torch").where
    return where(r < N, north, where(r <= 3 * N, band, south))


def ring_size(nside: int, r):
    """Pixels on ring r."""
    N = nside
    k = min(r, 4 * N - r)
    return 4 * k if k < N else 4 * N


def zphi2pix(nside: int, z, phi, xp=np):
    """RING index (int64) of the pixel containing each direction (z = cos theta, phi)."""
    N = nside
    X = _f64(xp, phi) * (2.0 / math.pi)
    X = X - 4.0 * xp.floor(X / 4.0)                       # phi in [0, 2 pi)
    X = xp.where(X >= 4.0, X - 4.0, X)
    z = _f64(xp, z)
    za = xp.abs(z)
    # equatorial band
    Y = 0.75 * z
    a = _ifloor(xp, N * (X - Y + 0.5))
    b = _ifloor(xp, N * (X + Y + 0.5))
    r = 2 * N - (b - a)
    e = a + b + 1 - N
    j = (e - (e & 1)) // 2
    j = j % (4 * N)
    p_band = 2 * N * (N - 1) + 4 * N * (r - N) + j
    # polar caps
    sigma = xp.sqrt(xp.where(za < 1.0, 3.0 * (1.0 - za), 0.0 * za))
    q = _ifloor(xp, X)
    q = xp.where(q > 3, q - 1, q)
    t = X - _f64(xp, q)
    u = _ifloor(xp, N * sigma * t)
    v = _ifloor(xp, N * sigma * (1.0 - t))
    k = u + v + 1
    k = xp.where(k > N, k * 0 + N, k)                      # |z| -> 2/3 from above
    jc = q * k + xp.where(u > k - 1, u * 0 + (k - 1), u)
    p_north = 2 * k * (k - 1) + jc
    p_south = 12 * N * N - 2 * k * (k + 1) + jc
    p_cap = xp.where(z > 0, p_north, p_south)
    return xp.where(za <= 2.0 / 3.0, p_band, p_cap)


def ang2pix(nside: int, theta, phi, xp=np):
    """RING index of directions (theta, phi) in radians."""
    return zphi2pix(nside, xp.cos(_f64(xp, theta)), phi, xp)


def pix2zphi(nside: int, pix, xp=np):
    """(z, phi) of the centres of RING pixels."""
    N = nside
    if _is_np(xp):
        pix = np.asarray(pix, dtype=np.int64)
        starts = ring_start(N, np.arange(1, 4 * N, dtype=np.int64))
        r = np.searchsorted(starts, pix, side="right").astype(np.int64)
    else:
        pix = pix.to(xp.int64)
        starts = ring_start(N, xp.arange(1, 4 * N, dtype=xp.int64, device=pix.device))
        r = xp.searchsorted(starts, pix, right=True).to(xp.int64)
    j = pix - ring_start(N, r)
    k = xp.where(r < 2 * N, r, 4 * N - r)                  # rings from the nearer pole
    kf, jf = _f64(xp, k), _f64(xp, j)
    z_cap = 1.0 - kf * kf / (3.0 * N * N)
    z_cap = xp.where(r < 2 * N, z_cap, -z_cap)
    phi_cap = (jf + 0.5) * math.pi / (2.0 * kf)
    s = _f64(xp, ((r - N) % 2 == 0).to(xp.int64) if not _is_np(xp) else ((r - N) % 2 == 0).astype(np.int64))
    z_band = 4.0 / 3.0 - 2.0 * _f64(xp, r) / (3.0 * N)
    phi_band = (jf + 0.5 * s) * math.pi / (2.0 * N)
    cap = (r < N) | (r > 3 * N)
    return xp.where(cap, z_cap, z_band), xp.where(cap, phi_cap, phi_band)


def pix2ang(nside: int, pix, xp=np):
    """(theta, phi) of the centres of RING pixels."""
    z, phi = pix2zphi(nside, pix, xp)
    return xp.arccos(z), phi
