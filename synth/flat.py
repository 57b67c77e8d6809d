"""Flat-sky raster scans, stationary intervals, 1/f noise and a random sky.

Every array is drawn from ``numpy.random.SeedSequence(seed)`` spawned into
independent streams (sky, jitter, intervals, noise parameters, noise, target,
flags), so a problem is reproducible bit for bit from its seed on any machine.

Geometry.  A W x W pixel grid, pixel p = row * W + col.  Sweeps alternate:
even sweeps are horizontal serpentines (row by row, direction reversed on odd
rows), odd sweeps vertical serpentines (column by column).  One sample per
pixel step; the pointed position is the pixel centre plus N(0, 0.3^2) pixels
of jitter per axis, floored and clamped to the grid.  This cross-linked scan
stands in for the paper's Planck and EBEX scans (Section 7), whose pointing
data is not available here.

Polarisation.  A detector with polariser angle psi_d behind a half-wave plate
at angle theta sees psi = psi_d + 2 theta; the plate steps once per sweep.

Noise.  Each (detector, interval) gets Gaussian noise with power spectrum
p(f) = sigma^2 (1 + (f_knee / f)^alpha) (Section 4, Eq. 13), synthesised by colouring
white noise in the Fourier domain; the zero-frequency bin takes the value of
the first non-zero bin so the variance stays finite.

Data.  d = A z + n with the weights (1, cos 2 psi, sin 2 psi) for (I, Q, U)
(Section 3, Eqs. 1-2), evaluated in float64 from the float32 angle and rounded to
float32.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_STREAMS = ("sky", "jitter", "intervals", "noiseparams", "noise", "target", "flags", "extra")


@dataclass
class Problem:
    """One synthetic map-making problem (all arrays host-side numpy)."""

    name: str
    n_stokes: int                 # 1 (T) or 3 (IQU)
    n_pix: int                    # global pixel count (W * W)
    width: int                    # grid side W
    pix: np.ndarray               # int32 [n_t], global pixel index, -1 = flagged sample
    psi: np.ndarray | None        # float32 [n_t] polarisation angle (radians), None for T
    d: np.ndarray                 # float32 [n_rhs, n_t] timestreams
    interval_offsets: np.ndarray  # int64 [n_ivl + 1], 0 ... n_t
    interval_filter: np.ndarray   # int32 [n_ivl], filter used by each interval
    interval_det: np.ndarray      # int32 [n_ivl], detector of each interval
    noise_params: np.ndarray      # float64 [n_filters, 3] = (sigma, f_knee, alpha)
    fs: float                     # sample rate (Hz)
    n_lags: int                   # n_c, number of filter lags
    sky: np.ndarray               # float64 [n_pix, n_stokes] true sky z
    target: np.ndarray | None = None   # float64 [n_pix, n_stokes] (differentiable-solve loss)
    meta: dict = field(default_factory=dict)
    pix_pol: np.ndarray | None = None  # int32 [n_t]: Q/U pixel per sample (multi-resolution maps), or None
    n_pix_pol: int = 0                 # global Q/U pixel count
    sky_pol: np.ndarray | None = None  # float64 [n_pix_pol, 2] true Q, U on the Q/U pixels

    @property
    def n_samples(self) -> int:
        return int(self.pix.shape[0])

    @property
    def n_rhs(self) -> int:
        return int(self.d.shape[0])

    @property
    def n_intervals(self) -> int:
        return int(self.interval_filter.shape[0])

    @property
    def n_filters(self) -> int:
        return int(self.noise_params.shape[0])


def _streams(seed: int) -> dict:
    kids = np.random.SeedSequence(seed).spawn(len(_STREAMS))
    return {k: np.random.default_rng(s) for k, s in zip(_STREAMS, kids)}


def raster_pixels(width: int, n_samples: int, rng: np.random.Generator, jitter: float = 0.3,
                  sweep_offset: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Pixel index and sweep number of each sample of the alternating raster."""
    k = np.arange(n_samples, dtype=np.int64)
    per = width * width
    sweep = k // per + sweep_offset
    step = k % per
    line = step // width
    pos = step % width
    pos = np.where(line % 2 == 0, pos, width - 1 - pos)
    horiz = (sweep % 2) == 0
    row = np.where(horiz, line, pos).astype(np.float64)
    col = np.where(horiz, pos, line).astype(np.float64)
    jit = rng.normal(0.0, jitter, size=(2, n_samples)) if jitter > 0 else np.zeros((2, n_samples))
    r = np.clip(np.floor(row + 0.5 + jit[0]), 0, width - 1).astype(np.int64)
    c = np.clip(np.floor(col + 0.5 + jit[1]), 0, width - 1).astype(np.int64)
    return (r * width + c).astype(np.int32), sweep


def gaussian_field(width: int, rng: np.random.Generator, rms: float) -> np.ndarray:
    """Gaussian random field on the grid, P(k) ~ k^-2, k = 0 mode removed, given RMS."""
    white = rng.standard_normal((width, width))
    kx = np.fft.fftfreq(width)
    k = np.sqrt(kx[:, None] ** 2 + kx[None, :] ** 2)
    amp = np.zeros_like(k)
    amp[k > 0] = 1.0 / k[k > 0]
    f = np.real(np.fft.ifft2(np.fft.fft2(white) * amp))
    f -= f.mean()
    f *= rms / np.sqrt(np.mean(f * f))
    return f.reshape(-1)


def log_uniform_intervals(total: int, lo: int, hi: int, rng: np.random.Generator) -> list[int]:
    """Interval lengths log-uniform in [lo, hi] drawn until they cover ``total``.

    The last draw is clipped to what remains; a remnant shorter than ``lo`` is
    merged into the previous interval.
    """
    out: list[int] = []
    acc = 0
    while acc < total:
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        n = min(n, total - acc)
        if n < lo and out:
            out[-1] += n
        else:
            out.append(n)
        acc += n
    return out


def colored_noise(n: int, fs: float, sigma: float, fknee: float, alpha: float,
                  rng: np.random.Generator) -> np.ndarray:
    """Gaussian noise of length n with PSD sigma^2 (1 + (fknee/f)^alpha)."""
    w = rng.standard_normal(n)
    if n < 2 or fknee <= 0.0:
        return sigma * w
    nu = np.fft.rfftfreq(n, d=1.0 / fs)
    nu[0] = nu[1]
    amp = sigma * np.sqrt(1.0 + (fknee / nu) ** alpha)
    return np.fft.irfft(np.fft.rfft(w) * amp, n)


def make_flat_problem(
    name: str,
    seed: int,
    width: int,
    n_det: int,
    samples_per_det: int,
    n_stokes: int,
    n_lags: int,
    fs: float = 100.0,
    det_angles_deg=None,
    hwp_step_deg: float = 0.0,
    interval_lengths=None,            # callable(rng, n) -> list of lengths, or None (one interval)
    noise=(1.0, 0.1, 2.0),            # (sigma, fknee, alpha) or callable(rng, n_det) -> [n_det, 3]
    shared_filter: bool = False,
    n_rhs: int = 1,
    flag_frac: float = 0.0,
    noiseless: bool = False,
    jitter: float = 0.3,
    make_target: bool = False,
    det_sweep_offset: bool = False,
    pol_factor: int = 0,
) -> Problem:
    """Build one flat-sky problem.  See the module docstring for the recipe.

    pol_factor = k > 0 (IQU): Q and U live on a coarser (W/k) x (W/k) grid (the
    multi-resolution maps of Section 6): each sample's Q/U pixel is the coarse
    pixel containing its (jittered) fine pixel, and the true Q, U are constant
    within coarse pixels (the coarse field at each fine pixel)."""
    rs = _streams(seed)
    n_pix = width * width
    # sky
    sky = np.zeros((n_pix, n_stokes))
    sky[:, 0] = gaussian_field(width, rs["sky"], 1.0)
    if n_stokes == 3:
        sky[:, 1] = gaussian_field(width, rs["sky"], 0.1)
        sky[:, 2] = gaussian_field(width, rs["sky"], 0.1)
    # pointing per detector
    pix_l, psi_l, ivl_l, det_l = [], [], [], []
    if det_angles_deg is None:
        det_angles_deg = [0.0] * n_det
    for det in range(n_det):
        off = det if det_sweep_offset else 0
        p, sweep = raster_pixels(width, samples_per_det, rs["jitter"], jitter, sweep_offset=off)
        pix_l.append(p)
        if n_stokes == 3:
            psi = np.deg2rad(det_angles_deg[det] + 2.0 * hwp_step_deg * sweep)
            psi_l.append(np.mod(psi, np.pi).astype(np.float32))
        lens = [samples_per_det] if interval_lengths is None else interval_lengths(rs["intervals"], samples_per_det)
        assert sum(lens) == samples_per_det
        ivl_l.extend(lens)
        det_l.extend([det] * len(lens))
    pix = np.concatenate(pix_l)
    psi = np.concatenate(psi_l) if n_stokes == 3 else None
    n_t = pix.shape[0]
    offsets = np.zeros(len(ivl_l) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(ivl_l)
    interval_det = np.asarray(det_l, dtype=np.int32)
    # noise parameters per detector
    if callable(noise):
        params = np.asarray(noise(rs["noiseparams"], n_det), dtype=np.float64)
    else:
        params = np.tile(np.asarray(noise, dtype=np.float64), (n_det, 1))
    if shared_filter:
        params = params[:1]
        interval_filter = np.zeros(len(ivl_l), dtype=np.int32)
    else:
        interval_filter = interval_det.copy()
    # flags
    if flag_frac > 0:
        flagged = rs["flags"].random(n_t) < flag_frac
        pix = pix.copy()
        pix[flagged] = -1
    pix_pol, sky_pol, n_pix_pol = None, None, 0
    if pol_factor and n_stokes == 3:
        wc = width // pol_factor
        n_pix_pol = wc * wc
        okp = pix >= 0
        r_, c_ = np.where(okp, pix, 0) // width, np.where(okp, pix, 0) % width
        pix_pol = np.where(okp, (r_ // pol_factor) * wc + c_ // pol_factor, -1).astype(np.int32)
        sky_pol = np.stack([gaussian_field(wc, rs["extra"], 0.1), gaussian_field(wc, rs["extra"], 0.1)], 1)
        fine = np.arange(n_pix)
        coarse = (fine // width // pol_factor) * wc + (fine % width) // pol_factor
        sky[:, 1:] = sky_pol[coarse]
    # signal A z in float64 from the float32 angle
    ok = pix >= 0
    sig = np.zeros(n_t)
    pz = np.where(ok, pix, 0)
    sig += sky[pz, 0]
    if n_stokes == 3:
        two = 2.0 * psi.astype(np.float64)
        sig += sky[pz, 1] * np.cos(two) + sky[pz, 2] * np.sin(two)
    sig[~ok] = 0.0
    d = np.empty((n_rhs, n_t), dtype=np.float32)
    for r in range(n_rhs):
        tod = sig.copy()
        if not noiseless:
            for i in range(len(ivl_l)):
                a, b = int(offsets[i]), int(offsets[i + 1])
                s, fk, al = params[interval_filter[i]]
                tod[a:b] += colored_noise(b - a, fs, s, fk, al, rs["noise"])
        d[r] = tod.astype(np.float32)
    target = None
    if make_target:
        target = sky + rs["target"].normal(0.0, 0.01, size=sky.shape)
    return Problem(name=name, n_stokes=n_stokes, n_pix=n_pix, width=width, pix=pix.astype(np.int32),
                   psi=psi, d=d, interval_offsets=offsets, interval_filter=interval_filter,
                   interval_det=interval_det, noise_params=params, fs=fs, n_lags=n_lags, sky=sky,
                   target=target, meta={"seed": seed, "n_det": n_det}, pix_pol=pix_pol,
                   n_pix_pol=n_pix_pol, sky_pol=sky_pol)


# --------------------------------------------------------------------------------------
# The five named workloads.  Sizes follow the paper-shaped workloads; ``scale`` shrinks
# the sample count (and grid) for CPU-sized test cases of the same structure.
# --------------------------------------------------------------------------------------

def config_spec(k: int) -> dict:
    """Human-readable description of workload k (1..5)."""
    return {
        1: dict(workload="T-only FP64, 1 det, 2^18 samples, 64x64 grid, n_c=2^12, 1 interval"),
        2: dict(workload="IQU mixed, 4 det x 2^22 samples, 512x512 grid, HWP 22.5 deg/sweep, "
                         "intervals 2^16-2^20, n_c=2^14"),
        4: dict(workload="T batched 64 RHS, 64x64 grid, 500 intervals 2^12-2^20, n_c=2^12"),
        5: dict(workload="IQU differentiable, 16 det x 2^22 samples, 256x256 grid, n_c=2^12"),
    }[k]


def make_config(k: int, scale: int = 0, n_rhs: int | None = None, seed: int | None = None) -> Problem:
    """Workload k at full size (scale=0) or shrunk by 2^scale in samples and grid area."""
    seed = 1000 * k if seed is None else seed
    if k == 1:
        w = 64 >> (scale // 2)
        return make_flat_problem("config1", seed, w, 1, (1 << 18) >> scale, 1, (1 << 12) >> scale,
                                 noise=(1.0, 0.1, 2.0))
    if k == 2:
        w = 512 >> (scale // 2)
        lo, hi = (1 << 16) >> scale, (1 << 20) >> scale

        def ivls(rng, n):
            return log_uniform_intervals(n, lo, hi, rng)

        def nz(rng, nd):
            return np.stack([np.ones(nd), rng.uniform(0.05, 0.2, nd), rng.uniform(1.0, 2.0, nd)], 1)

        return make_flat_problem("config2", seed, w, 4, (1 << 22) >> scale, 3, (1 << 14) >> scale,
                                 det_angles_deg=[0.0, 45.0, 90.0, 135.0], hwp_step_deg=22.5,
                                 interval_lengths=ivls, noise=nz)
    if k == 4:
        lo, hi = (1 << 12) >> scale, (1 << 20) >> scale
        rng = _streams(seed)["extra"]
        lens = [int(round(np.exp(rng.uniform(np.log(lo), np.log(hi))))) for _ in range(500 >> min(scale, 6))]
        total = int(sum(lens))

        def ivls(_rng, n):
            assert n == total
            return lens

        return make_flat_problem("config4", seed, 64 >> (scale // 2), 1, total, 1, (1 << 12) >> scale,
                                 interval_lengths=ivls, noise=(1.0, 0.1, 2.0), shared_filter=True,
                                 n_rhs=64 if n_rhs is None else n_rhs)
    if k == 5:
        w = 256 >> (scale // 2)

        def nz(rng, nd):
            return np.array([1.0, 0.1, 2.0]) * rng.uniform(0.8, 1.2, size=(nd, 3))

        return make_flat_problem("config5", seed, w, 16, (1 << 22) >> scale, 3, (1 << 12) >> scale,
                                 det_angles_deg=[11.25 * i for i in range(16)], noise=nz,
                                 make_target=True)
    raise ValueError(f"unknown workload {k}")


def device_timestreams(problem: Problem, n_rhs: int, seed: int, device="cuda"):
    """float32 [n_rhs, n_t] timestreams d_r = A z + n_r synthesised on a GPU.

    For workloads whose many noise realisations are too large to draw on the
    host (e.g. 64 right-hand sides of 10^8 samples).  Same recipe as the host
    path (signal from the float32 angles, noise coloured to the PSD with the
    zero-frequency bin set to the first non-zero one), drawn from torch's
    seeded device generator instead of numpy's, so the values differ from the
    host path while following the same distribution.  pix, psi and sky may be
    numpy arrays or torch tensors.
    """
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    def dev(a):
        return a.to(device) if isinstance(a, torch.Tensor) else torch.from_numpy(np.asarray(a)).to(device)

    pix = dev(problem.pix).to(torch.int64)
    ok = pix >= 0
    sky = dev(problem.sky).to(torch.float64)
    sig = sky[pix.clamp(min=0), 0]
    if problem.n_stokes == 3:
        two = 2.0 * dev(problem.psi).to(torch.float64)
        sig = sig + sky[pix.clamp(min=0), 1] * torch.cos(two) + sky[pix.clamp(min=0), 2] * torch.sin(two)
    sig = torch.where(ok, sig, torch.zeros_like(sig))
    out = torch.empty((n_rhs, problem.n_samples), dtype=torch.float32, device=device)
    off = problem.interval_offsets
    for i in range(problem.n_intervals):
        a, b = int(off[i]), int(off[i + 1])
        n = b - a
        if n == 0:
            continue
        s, fk, al = problem.noise_params[problem.interval_filter[i]]
        w = torch.randn((n_rhs, n), generator=g, device=device, dtype=torch.float64)
        if n >= 2 and fk > 0:
            nu = torch.fft.rfftfreq(n, d=1.0 / problem.fs, device=device, dtype=torch.float64)
            nu[0] = nu[1]
            amp = s * torch.sqrt(1.0 + (fk / nu) ** al)
            w = torch.fft.irfft(torch.fft.rfft(w, dim=1) * amp, n=n, dim=1)
        else:
            w = s * w
        out[:, a:b] = (sig[a:b].unsqueeze(0) + w).to(torch.float32)
    return out
