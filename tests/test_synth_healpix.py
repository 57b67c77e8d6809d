"""Pins of the all-sky input generator: HEALPix RING pixelisation and the ring scan.

The pixelisation follows the geometry published by Gorski et al. (2005,
Section 4); these tests check it against facts fixed there (12 N^2 pixels,
ring sizes and latitudes, the layout of the 12 base pixels, equal areas) and
against itself (every pixel centre falls in its own pixel) for odd and even
N_side.  The chunked oracle system used for full-size sampled checks is pinned
against the in-memory one on a small all-sky problem.
"""

from __future__ import annotations

import math

import numpy as np
import pytest

from synth import healpix
from synth.allsky import geometry, make_allsky_problem, ring_scan

NSIDES = [1, 2, 3, 4, 5, 8, 16, 33]


@pytest.mark.parametrize("N", NSIDES)
def test_rings_partition_the_pixels(N):
    rings = np.arange(1, 4 * N)
    sizes = np.array([healpix.ring_size(N, int(r)) for r in rings])
    starts = np.array([healpix.ring_start(N, int(r)) for r in rings])
    assert sizes.sum() == 12 * N * N
    assert starts[0] == 0 and np.array_equal(starts[1:], np.cumsum(sizes)[:-1])
    # 4k pixels on the k-th cap ring, 4N on every band ring
    assert np.array_equal(sizes[:N - 1], 4 * np.arange(1, N)) and np.all(sizes[N - 1:3 * N] == 4 * N)


@pytest.mark.parametrize("N", NSIDES)
def test_pixel_centres_round_trip_and_ring_latitudes(N):
    p = np.arange(12 * N * N)
    z, phi = healpix.pix2zphi(N, p)
    assert np.array_equal(healpix.zphi2pix(N, z, phi), p)
    for r in range(1, 4 * N):
        s = healpix.ring_start(N, r)
        k = min(r, 4 * N - r)
        zr = (1 - k * k / (3 * N * N)) if k < N else (4 / 3 - 2 * r / (3 * N))
        zr = zr if r <= 2 * N or k >= N else -zr
        zz = z[s:s + healpix.ring_size(N, r)]
        assert np.allclose(zz, zr, atol=1e-15)
        ph = phi[s:s + healpix.ring_size(N, r)]
        assert np.all(np.diff(ph) > 0) and ph[0] >= 0 and ph[-1] < 2 * np.pi


def test_base_pixels():
    z, phi = healpix.pix2zphi(1, np.arange(12))
    q = np.arange(4)
    assert np.allclose(z, np.repeat([2 / 3, 0.0, -2 / 3], 4))
    assert np.allclose(phi[:4], np.pi / 4 + q * np.pi / 2)
    assert np.allclose(phi[4:8], q * np.pi / 2)
    assert np.allclose(phi[8:], np.pi / 4 + q * np.pi / 2)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_pixels_have_equal_areas(N):
    rng = np.random.default_rng(N)
    n = 3_000_000
    z, phi = rng.uniform(-1, 1, n), rng.uniform(0, 2 * np.pi, n)
    c = np.bincount(healpix.zphi2pix(N, z, phi), minlength=12 * N * N)
    e = n / (12 * N * N)
    assert np.max(np.abs(c - e)) < 4.5 * math.sqrt(e)


@pytest.mark.parametrize("N", [4, 7, 16])
def test_points_land_in_a_nearby_pixel(N):
    """Every direction is within 1.5 pixel sizes of the centre of its pixel (a wrong ring
    or a wrong position along the ring would put it further away)."""
    rng = np.random.default_rng(10 + N)
    n = 200_000
    z, phi = rng.uniform(-1, 1, n), rng.uniform(-7, 7, n)
    zc, pc = healpix.pix2zphi(N, healpix.zphi2pix(N, z, phi))
    s, sc = np.sqrt(1 - z * z), np.sqrt(1 - zc * zc)
    cosd = z * zc + s * sc * np.cos(phi - pc)
    ang = np.arccos(np.clip(cosd, -1, 1))
    assert ang.max() < 1.5 * math.sqrt(4 * np.pi / (12 * N * N))


def test_torch_and_numpy_pixelisation_agree():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    z, phi = rng.uniform(-1, 1, 100_000), rng.uniform(0, 2 * np.pi, 100_000)
    for N in [3, 16, 512]:
        a = healpix.zphi2pix(N, z, phi)
        b = healpix.zphi2pix(N, torch.from_numpy(z), torch.from_numpy(phi), torch).numpy()
        assert np.array_equal(a, b)
        zc, pc = healpix.pix2zphi(N, torch.from_numpy(a), torch)
        za, pa = healpix.pix2zphi(N, a)
        assert np.array_equal(zc.numpy(), za) and np.array_equal(pc.numpy(), pa)


def test_ring_scan_geometry():
    """Boresight on an 85-degree cone about an ecliptic spin axis; the detector offset
    across the scan; the polariser angle relative to the scan direction."""
    g = geometry(0)
    n = 3 * g["samples_per_ring"]
    z0, p0, s0 = ring_scan(np, 0, n, g["samples_per_ring"], g["step_arcmin"], 0.0, 0.0)
    z1, p1, s1 = ring_scan(np, 0, n, g["samples_per_ring"], g["step_arcmin"], 0.5, 45.0)
    ring = np.arange(n) // g["samples_per_ring"]
    lam = np.radians(ring * g["step_arcmin"] / 60.0)
    st = np.sqrt(1 - z0 * z0)
    cosang = st * np.cos(p0) * np.cos(lam) + st * np.sin(p0) * np.sin(lam)
    assert np.allclose(cosang, math.cos(math.radians(85.0)), atol=1e-12)
    st1 = np.sqrt(1 - z1 * z1)
    sep = np.arccos(np.clip(z0 * z1 + st * st1 * np.cos(p0 - p1), -1, 1))
    assert np.allclose(np.degrees(sep), 0.5, atol=1e-9)
    # polariser turned 45 degrees from the scan direction v towards n x v, which is the
    # sense opposite to north -> east: psi drops by 45 degrees (up to the small change
    # of the local meridian across 0.5 degrees)
    dpsi = np.degrees(np.angle(np.exp(1j * (s1 - s0))))
    far = np.abs(z0) < 0.7          # meridians converge by at most 0.5 deg there
    assert np.all(np.abs(dpsi[far] + 45.0) < 0.6)


def test_allsky_problem_shape():
    p = make_allsky_problem(scale=10, n_det=8)
    g = geometry(10)
    assert p.n_pix == 12 * g["nside"] ** 2 and p.n_samples == 8 * g["samples_per_det"]
    L = np.diff(p.interval_offsets)
    assert L.min() > 0 and L.max() <= g["period"][1] and np.sum(L >= g["period"][0]) >= p.n_intervals - 8
    assert p.pix.dtype == np.int32 and p.psi.dtype == np.float32 and p.d.dtype == np.float32
    assert p.pix.min() >= 0 and p.pix.max() < p.n_pix
    assert np.all((p.psi >= 0) & (p.psi <= np.float32(np.pi)))
    q = make_allsky_problem(scale=10, n_det=8)
    assert np.array_equal(p.pix, q.pix) and np.array_equal(p.d, q.d)


def test_streamed_system_matches_in_memory_system():
    """The chunked oracle used for full-size sampled checks gives the rows of the
    in-memory system: same observed pixels, classification and H x, b rows."""
    from oracle.noise import filter_lags
    from oracle.solver import StreamedSystem, System
    p = make_allsky_problem(scale=12, n_det=8)
    lags = filter_lags(p.n_lags, p.fs, *p.noise_params[0])[None, :]
    pix = p.pix.copy()
    unseen = np.setdiff1d(np.arange(p.n_pix), pix)
    pix[[100, 5000]] = unseen[0]             # two hits: excised
    pix[[7, 9000, 20000]] = -1               # flagged samples
    args = (pix, p.psi, p.n_pix, 3, p.interval_offsets, p.interval_filter, lags)
    S = System(*args, ninv="direct")
    T = StreamedSystem(*args, chunk=1000)
    assert np.array_equal(S.obs2glob, T.obs2glob)
    assert np.array_equal(S.excised, T.excised) and np.array_equal(S.fp64, T.fp64)
    assert np.allclose(S.Pinv, T.Pinv, rtol=1e-11, atol=1e-11 * np.abs(S.Pinv).max())
    assert S.excised.sum() > 0 and (~S.excised).sum() > 100
    rng = np.random.default_rng(1)
    x = rng.standard_normal((S.n_obs, 3))
    pk = rng.choice(S.n_obs, 20, replace=False)
    full = S.H(x)[pk]
    assert np.allclose(T.H_sampled(x, pk), full, rtol=1e-11, atol=1e-11 * np.abs(full).max())
    b = S.rhs(p.d[0])[pk]
    assert np.allclose(T.rhs_sampled(p.d[0], pk), b, rtol=1e-11, atol=1e-11 * np.abs(b).max())
