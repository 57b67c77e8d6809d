"""All-sky spinning ring scan on a HEALPix RING grid (input synthesis only).

A Planck-shaped stand-in for the paper's satellite workload (Section 7.1),
whose pointing is not available here:

* Scan.  The spin axis lies in the ecliptic plane and advances step_arcmin
  per ring; the line of sight sweeps a cone of half-angle 85 degrees about it
  at 1 rpm, sampled at 180 Hz (10,800 samples per ring).
* Focal plane.  32 detectors = 8 cross-scan offsets evenly spread over
  [-0.5, 0.5] degrees x polariser angles 0/45/90/135 degrees from the scan
  direction.  Detector d has offset d // 4 and angle d % 4, so the first four
  already constrain I, Q and U.
* Pixels.  HEALPix N_side = 512 RING (synth.healpix) of the float64 direction;
  unobserved pixels are left to the plan's compaction (Section 5.4).
  Polarisation angle psi: the polariser direction measured from the local
  meridian (towards north) towards east, stored as float32.
* Intervals.  Pointing periods of seeded U[40, 60] minutes (432,000 to
  648,000 samples), cut per detector; one shared noise filter (sigma = 1,
  f_knee = 0.03 Hz, alpha = 1.7, 2^15 lags).
* Sky.  A smooth random IQU field at the pixel centres: sums of 48 seeded
  Fisher-von Mises blobs per Stokes parameter, I with RMS 1 and Q, U with RMS 0.1.
* Data.  d = A z + n, the signal from the float32 angle in float64 (Section 3,
  Eqs. 1-2), noise coloured to sigma^2 (1 + (f_knee/f)^alpha) per interval
  (Section 4, Eq. 13), rounded to float32.

``scale`` s shrinks the workload while keeping its shape: 2^-s of the samples
per detector, of the lags and of the interval lengths; N_side, the samples per
ring, the ring step and the focal-plane offsets change by 2^(s/2), so the
swept area and the hits per pixel stay the same.

The host path (numpy, ``device=None``) serves CPU-sized test cases; with a
torch device the geometry, the sky and the noise are synthesised on the GPU
(float64 geometry, torch's seeded generator for noise), which the 5.4e8-sample
full size needs.  Both are deterministic for a given seed and platform.
"""

from __future__ import annotations

import math

import numpy as np

from . import healpix
from .flat import Problem, _streams, colored_noise

FS = 180.0
OPENING_DEG = 85.0
SAMPLES_PER_RING = 10800            # 1 rpm at 180 Hz
STEP_ARCMIN = 2.5
NSIDE = 512
SAMPLES_PER_DET = 1 << 24
N_DET = 32
N_LAGS = 1 << 15
PERIOD_MIN = (40.0, 60.0)
NOISE = (1.0, 0.03, 1.7)
ANGLES_DEG = (0.0, 45.0, 90.0, 135.0)


def geometry(scale: int = 0) -> dict:
    """Sizes of the all-sky workload shrunk by 2^scale in samples."""
    f = 2.0 ** (scale / 2.0)
    return dict(
        nside=max(1, NSIDE >> (scale // 2)),
        samples_per_det=SAMPLES_PER_DET >> scale,
        samples_per_ring=max(8, int(round(SAMPLES_PER_RING / f))),
        step_arcmin=STEP_ARCMIN * f,
        max_offset_deg=0.5 * f,
        n_lags=max(2, N_LAGS >> scale),
        period=(int(round(PERIOD_MIN[0] * 60 * FS)) >> scale, int(round(PERIOD_MIN[1] * 60 * FS)) >> scale),
    )


def ring_scan(xp, k0: int, n: int, samples_per_ring: int, step_arcmin: float, offset_deg: float,
              angle_deg: float, device=None):
    """(z, phi, psi) in float64 for samples k0 .. k0 + n - 1 of one detector."""
    if xp is np:
        k = np.arange(k0, k0 + n, dtype=np.float64)
    else:
        k = xp.arange(k0, k0 + n, dtype=xp.float64, device=device)
    ring = xp.floor(k / samples_per_ring)
    lam = ring * math.radians(step_arcmin / 60.0)             # spin-axis longitude
    om = (k - ring * samples_per_ring) * (2.0 * math.pi / samples_per_ring)
    ca, sa = math.cos(math.radians(OPENING_DEG)), math.sin(math.radians(OPENING_DEG))
    cl, sl = xp.cos(lam), xp.sin(lam)
    co, so = xp.cos(om), xp.sin(om)
    # spin axis s = (cl, sl, 0); e1 = (0, 0, 1); e2 = (sl, -cl, 0).
    # boresight n = ca s + sa (so e2 + co e1); scan direction v = dn/dom / sa.
    nx, ny, nz = ca * cl + sa * so * sl, ca * sl - sa * so * cl, sa * co
    vx, vy, vz = co * sl, -co * cl, -so
    # cross-scan direction c = n x v
    cx, cy, cz = ny * vz - nz * vy, nz * vx - nx * vz, nx * vy - ny * vx
    dc, ds = math.cos(math.radians(offset_deg)), math.sin(math.radians(offset_deg))
    px, py, pz = dc * nx + ds * cx, dc * ny + ds * cy, dc * nz + ds * cz      # detector direction
    # polariser direction in the plane of v and c
    gc, gs = math.cos(math.radians(angle_deg)), math.sin(math.radians(angle_deg))
    ex, ey, ez = gc * vx + gs * cx, gc * vy + gs * cy, gc * vz + gs * cz
    z = xp.clip(pz, -1.0, 1.0) if xp is np else xp.clamp(pz, -1.0, 1.0)
    phi = xp.arctan2(py, px)
    # local north (towards +z) and east at the detector direction, unnormalised by sin(theta)
    north = -pz * (px * ex + py * ey) + (1.0 - pz * pz) * ez
    east = -py * ex + px * ey
    psi = xp.arctan2(east, north)
    return z, phi, psi


def smooth_sky(nside: int, rng: np.random.Generator, xp=np, device=None, n_blobs: int = 48, kappa: float = 20.0):
    """float64 [12 N^2, 3] IQU field at the pixel centres (I RMS 1, Q and U RMS 0.1)."""
    npix = healpix.n_pixels(nside)
    centres = [rng.standard_normal((n_blobs, 3)) for _ in range(3)]
    amps = [rng.standard_normal(n_blobs) for _ in range(3)]
    if xp is np:
        p = np.arange(npix)
    else:
        p = xp.arange(npix, device=device)
    z, phi = healpix.pix2zphi(nside, p, xp)
    st = xp.sqrt(xp.clip(1.0 - z * z, 0.0, None) if xp is np else xp.clamp(1.0 - z * z, min=0.0))
    nvec = xp.stack([st * xp.cos(phi), st * xp.sin(phi), z], 1)
    cols = []
    for s in range(3):
        u = centres[s] / np.linalg.norm(centres[s], axis=1, keepdims=True)
        if xp is not np:
            u = xp.from_numpy(u).to(device)
            a = xp.from_numpy(amps[s]).to(device)
        else:
            a = amps[s]
        f = xp.exp(kappa * (nvec @ u.T - 1.0)) @ a
        f = f - f.mean()
        f = f * ((1.0 if s == 0 else 0.1) / xp.sqrt(xp.mean(f * f)))
        cols.append(f)
    return xp.stack(cols, 1)


def pointing_periods(n: int, lo: int, hi: int, rng: np.random.Generator) -> list[int]:
    """Uniform lengths in [lo, hi] covering n samples, the last one cut."""
    out, tot = [], 0
    while tot < n:
        L = min(int(rng.integers(lo, hi + 1)), n - tot)
        out.append(L)
        tot += L
    return out


def make_allsky_problem(scale: int = 0, n_det: int = N_DET, seed: int = 3000, device=None,
                        noiseless: bool = False) -> Problem:
    """The all-sky ring-scan workload (see the module docstring).

    With ``device`` set, pix, psi, d and sky are torch tensors on that device;
    otherwise numpy arrays.
    """
    g = geometry(scale)
    N, n_per = g["nside"], g["samples_per_det"]
    rs = _streams(seed)
    if device is None:
        xp = np
    else:
        import torch as xp
    pix_l, psi_l, lens, det_l = [], [], [], []
    for det in range(n_det):
        o, a = det // 4, det % 4
        off = (-1.0 + 2.0 * o / 7.0) * g["max_offset_deg"] if n_det > 4 else 0.0
        z, phi, psi = ring_scan(xp, 0, n_per, g["samples_per_ring"], g["step_arcmin"], off, ANGLES_DEG[a], device)
        p = healpix.zphi2pix(N, z, phi, xp)
        if xp is np:
            pix_l.append(p.astype(np.int32))
            psi_l.append(np.mod(psi, np.pi).astype(np.float32))
        else:
            pix_l.append(p.to(xp.int32))
            psi_l.append(xp.remainder(psi, math.pi).to(xp.float32))
        L = pointing_periods(n_per, g["period"][0], g["period"][1], rs["intervals"])
        lens.extend(L)
        det_l.extend([det] * len(L))
    cat = np.concatenate if xp is np else xp.cat
    pix, psi = cat(pix_l), cat(psi_l)
    del pix_l, psi_l
    offsets = np.zeros(len(lens) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lens)
    interval_det = np.asarray(det_l, dtype=np.int32)
    interval_filter = np.zeros(len(lens), dtype=np.int32)
    params = np.asarray([NOISE], dtype=np.float64)
    sky = smooth_sky(N, rs["sky"], xp, device)
    prob = Problem(name="config3", n_stokes=3, n_pix=healpix.n_pixels(N), width=N, pix=pix, psi=psi,
                   d=None, interval_offsets=offsets, interval_filter=interval_filter,
                   interval_det=interval_det, noise_params=params, fs=FS, n_lags=g["n_lags"], sky=sky,
                   meta={"seed": seed, "n_det": n_det, "pixelisation": "healpix_ring", "nside": N,
                         "scale": scale})
    if xp is np:
        two = 2.0 * psi.astype(np.float64)
        sig = sky[pix, 0] + sky[pix, 1] * np.cos(two) + sky[pix, 2] * np.sin(two)
        if not noiseless:
            for i in range(len(lens)):
                lo, hi = int(offsets[i]), int(offsets[i + 1])
                sig[lo:hi] += colored_noise(hi - lo, FS, *NOISE, rs["noise"])
        prob.d = sig.astype(np.float32)[None, :]
    else:
        from .flat import device_timestreams
        if noiseless:
            two = 2.0 * psi.to(xp.float64)
            pl = pix.to(xp.int64)
            sig = sky[pl, 0] + sky[pl, 1] * xp.cos(two) + sky[pl, 2] * xp.sin(two)
            prob.d = sig.to(xp.float32).unsqueeze(0)
        else:
            prob.d = device_timestreams(prob, 1, int(rs["noise"].integers(1 << 62)), device)
    return prob
