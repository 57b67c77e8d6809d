"""Compressed boresight pointing for flat-sky raster scans (the input of the
on-the-fly pointing expansion), with intervals, 1/f noise and a sky.

The scan.  Sweeps alternate horizontal and vertical serpentines at one pixel
per sample, as in ``synth.flat``, but every line overshoots the W x W grid by
``step`` samples at each end and turns around outside it, as telescope scans
do.  The boresight path is piecewise linear between nodes placed every
``step`` samples (``step`` divides the line length W + 2 step, so each line
starts on a node and every segment that crosses the grid is straight); a
segment that carries a turn lies wholly outside the grid.  The focal plane
turns slowly about the boresight (one turn every ``rot_period`` samples), so
each pixel is seen at many polariser orientations.  The compressed pointing
holds the nodes in float32: (x, y, cos a, sin a).  Detectors sit at fixed
focal-plane offsets (pixel units) with their own polariser angles.

The data.  d = s + n with s the sky at each detector's true position: the
path evaluated in float64 at the sample's own time (linear between the
nodes), rotated to the detector by the exact orientation, and looked up in
the pixel grid; samples whose true position is off the grid see no signal.
The map-maker pixelises the float32 interpolated pointing, so the two differ
only by float32 rounding (samples within ~1e-5 pixel of an edge).  Noise per
(detector, interval) as in ``synth.flat``.  Everything is drawn from seeded
streams.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .flat import _streams, colored_noise, gaussian_field


@dataclass
class BoresightProblem:
    name: str
    n_stokes: int
    width: int
    height: int
    boresight: np.ndarray          # float32 [n_bore, 4]: x, y, cos a, sin a per node
    bore_step: int                 # detector samples per node interval
    det: np.ndarray                # float32 [n_det, 4]: dx, dy, cos psi_d, sin psi_d
    samples_per_det: int
    d: np.ndarray                  # float32 [n_rhs, n_t]
    interval_offsets: np.ndarray   # int64 [n_ivl + 1]
    interval_filter: np.ndarray    # int32 [n_ivl]
    interval_det: np.ndarray       # int32 [n_ivl]
    noise_params: np.ndarray       # float64 [n_filters, 3]
    fs: float
    n_lags: int
    sky: np.ndarray                # float64 [n_pix, n_stokes]
    meta: dict = field(default_factory=dict)

    @property
    def n_pix(self) -> int:
        return self.width * self.height

    @property
    def n_det(self) -> int:
        return int(self.det.shape[0])

    @property
    def n_samples(self) -> int:
        return self.n_det * self.samples_per_det

    @property
    def n_filters(self) -> int:
        return int(self.noise_params.shape[0])


def raster_nodes(width: int, step: int, k: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(x, y) of the overshooting serpentine raster at integer sample times k (the
    node positions when k is a multiple of ``step``)."""
    k = np.asarray(k, dtype=np.int64)
    L = width + 2 * step
    per = width * L
    sweep = k // per
    line = (k % per) // L
    pos = k % L
    along = np.where(line % 2 == 0, -step + 0.5 + pos, width + step - 0.5 - pos).astype(np.float64)
    across = line.astype(np.float64) + 0.5
    horiz = (sweep % 2) == 0
    return np.where(horiz, along, across), np.where(horiz, across, along)


def make_boresight_problem(name: str, seed: int, width: int, n_det: int, samples_per_det: int, step: int,
                           n_stokes: int, n_lags: int, fs: float = 100.0, det_offsets=None,
                           det_angles_deg=None, rot_period: int | None = None, interval_lengths=None,
                           noise=(1.0, 0.1, 2.0), noiseless: bool = False, n_rhs: int = 1) -> BoresightProblem:
    rs = _streams(seed)
    n_pix = width * width
    sky = np.zeros((n_pix, n_stokes))
    sky[:, 0] = gaussian_field(width, rs["sky"], 1.0)
    if n_stokes == 3:
        sky[:, 1] = gaussian_field(width, rs["sky"], 0.1)
        sky[:, 2] = gaussian_field(width, rs["sky"], 0.1)
    if rot_period is None:
        rot_period = 4 * n_pix
    if det_offsets is None:
        det_offsets = [(0.35 * np.cos(2 * np.pi * i / n_det), 0.35 * np.sin(2 * np.pi * i / n_det))
                       for i in range(n_det)]
    if det_angles_deg is None:
        det_angles_deg = [180.0 * i / n_det for i in range(n_det)]
    a0 = rs["extra"].uniform(0.0, 2.0 * np.pi)

    def orientation(k):
        return a0 + 2.0 * np.pi * np.asarray(k, dtype=np.float64) / rot_period

    assert width % step == 0, "the node step must divide the grid width"
    n_bore = (samples_per_det - 1) // step + 2 if samples_per_det > 0 else 0
    ku = np.arange(n_bore, dtype=np.int64) * step
    bx, by = raster_nodes(width, step, ku)
    ab = orientation(ku)
    boresight = np.stack([bx, by, np.cos(ab), np.sin(ab)], 1).astype(np.float32)
    pd = np.deg2rad(np.asarray(det_angles_deg, dtype=np.float64))
    det = np.stack([np.asarray(det_offsets, dtype=np.float64)[:, 0], np.asarray(det_offsets, dtype=np.float64)[:, 1],
                    np.cos(pd), np.sin(pd)], 1).astype(np.float32)
    # signal at the true positions: the path linear between the nodes
    k = np.arange(samples_per_det, dtype=np.int64)
    u = k // step
    fr = (k - u * step) / step
    x = bx[u] + fr * (bx[np.minimum(u + 1, n_bore - 1)] - bx[u]) if samples_per_det else np.zeros(0)
    y = by[u] + fr * (by[np.minimum(u + 1, n_bore - 1)] - by[u]) if samples_per_det else np.zeros(0)
    a = orientation(k)
    sig_l, ivl_l, det_l = [], [], []
    for di in range(n_det):
        dx, dy = float(det[di, 0]), float(det[di, 1])
        X = x + np.cos(a) * dx - np.sin(a) * dy
        Y = y + np.sin(a) * dx + np.cos(a) * dy
        ix, iy = np.floor(X), np.floor(Y)
        ok = (ix >= 0) & (ix < width) & (iy >= 0) & (iy < width)
        p = np.where(ok, iy * width + ix, 0).astype(np.int64)
        s = sky[p, 0].copy()
        if n_stokes == 3:
            two = 2.0 * (a + pd[di])
            s += sky[p, 1] * np.cos(two) + sky[p, 2] * np.sin(two)
        sig_l.append(np.where(ok, s, 0.0))
        lens = [samples_per_det] if interval_lengths is None else interval_lengths(rs["intervals"], samples_per_det)
        assert sum(lens) == samples_per_det
        ivl_l.extend(lens)
        det_l.extend([di] * len(lens))
    sig = np.concatenate(sig_l) if sig_l else np.zeros(0)
    n_t = sig.shape[0]
    offsets = np.zeros(len(ivl_l) + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(ivl_l)
    interval_det = np.asarray(det_l, dtype=np.int32)
    if callable(noise):
        params = np.asarray(noise(rs["noiseparams"], n_det), dtype=np.float64)
    else:
        params = np.tile(np.asarray(noise, dtype=np.float64), (n_det, 1))
    interval_filter = interval_det.copy()
    d = np.empty((n_rhs, n_t), dtype=np.float32)
    for r in range(n_rhs):
        tod = sig.copy()
        if not noiseless:
            for i in range(len(ivl_l)):
                lo, hi = int(offsets[i]), int(offsets[i + 1])
                s_, fk, al = params[interval_filter[i]]
                tod[lo:hi] += colored_noise(hi - lo, fs, s_, fk, al, rs["noise"])
        d[r] = tod.astype(np.float32)
    return BoresightProblem(name=name, n_stokes=n_stokes, width=width, height=width, boresight=boresight,
                            bore_step=int(step), det=det, samples_per_det=int(samples_per_det), d=d,
                            interval_offsets=offsets, interval_filter=interval_filter, interval_det=interval_det,
                            noise_params=params, fs=fs, n_lags=n_lags, sky=sky,
                            meta={"seed": seed, "rot_period": rot_period})


def make_boresight_config2(scale: int = 0, step: int = 16, seed: int = 2000) -> BoresightProblem:
    """The IQU workload's shape (4 detectors x 2^22 samples, 512 x 512 grid, intervals
    2^16-2^20, 2^14 lags, f_knee 0.05-0.2 Hz, alpha 1-2) with compressed pointing."""
    from .flat import log_uniform_intervals
    w = 512 >> (scale // 2)
    lo, hi = (1 << 16) >> scale, (1 << 20) >> scale

    def ivls(rng, n):
        return log_uniform_intervals(n, lo, hi, rng)

    def nz(rng, nd):
        return np.stack([np.ones(nd), rng.uniform(0.05, 0.2, nd), rng.uniform(1.0, 2.0, nd)], 1)

    return make_boresight_problem("config2-boresight", seed, w, 4, (1 << 22) >> scale, step, 3, (1 << 14) >> scale,
                                  det_angles_deg=[0.0, 45.0, 90.0, 135.0], interval_lengths=ivls, noise=nz)
