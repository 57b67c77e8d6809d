"""Extra columns of an extended pointing matrix (destriping baselines, binned
synchronous templates) and the signal they add to a timestream.

Index arrays are int32 per sample, -1 where the sample has no extra column.
One baseline (or one bin) is left without a column so that the extended
system stays non-singular (an offset on every sample is degenerate with a
constant temperature map).
"""

from __future__ import annotations

import numpy as np


def baseline_index(samples_per_det: int, n_det: int, length: int, reference: int = 0):
    """(extra_index int32 [n_det * samples_per_det], n_extra): consecutive baselines of
    ``length`` samples within each detector's stream, numbered across detectors; the
    global baseline ``reference`` gets no column."""
    per = -(-samples_per_det // length)
    j = np.arange(samples_per_det, dtype=np.int64) // length
    ids = (np.arange(n_det, dtype=np.int64)[:, None] * per + j[None, :]).reshape(-1)
    idx = np.where(ids == reference, -1, np.where(ids > reference, ids - 1, ids))
    return idx.astype(np.int32), int(n_det * per - 1)


def chop_bins(n_t: int, n_bins: int, period: float, rng: np.random.Generator, reference: int = 0):
    """(extra_index int32 [n_t], n_extra): the bin of a chopper angle sweeping
    [0, 2 pi) once every ``period`` samples from a random phase; bin ``reference``
    gets no column."""
    phase = rng.uniform(0.0, 2.0 * np.pi)
    ang = np.mod(phase + 2.0 * np.pi * np.arange(n_t) / period, 2.0 * np.pi)
    b = np.minimum((ang / (2.0 * np.pi) * n_bins).astype(np.int64), n_bins - 1)
    idx = np.where(b == reference, -1, np.where(b > reference, b - 1, b))
    return idx.astype(np.int32), n_bins - 1


def add_extra_signal(d: np.ndarray, extra_index: np.ndarray, amplitudes: np.ndarray) -> np.ndarray:
    """d + B o in float32 (B o_t = amplitudes[extra_index[t]], 0 where the index is -1)."""
    e = np.asarray(extra_index)
    add = np.where(e >= 0, np.asarray(amplitudes, dtype=np.float64)[np.maximum(e, 0)], 0.0)
    return (np.asarray(d, dtype=np.float64) + add).astype(np.float32)


def hwp_inputs(interval_offsets, fs: float, f_hwp: float, rng: np.random.Generator, group_of_interval=None):
    """(angle float32 [n_t], tau float32 [n_t], group int32 [n_ivl], n_groups) for a half-wave
    plate turning at f_hwp Hz: angle = 2 pi f_hwp t + phase (wrapped to [0, 2 pi)), tau running
    from -1 to 1 across each interval, one group per interval unless given."""
    off = np.asarray(interval_offsets, dtype=np.int64)
    n_t = int(off[-1])
    phase = rng.uniform(0.0, 2.0 * np.pi)
    t = np.arange(n_t, dtype=np.float64) / fs
    angle = np.mod(phase + 2.0 * np.pi * f_hwp * t, 2.0 * np.pi).astype(np.float32)
    tau = np.zeros(n_t)
    for i in range(off.size - 1):
        n = int(off[i + 1] - off[i])
        if n:
            tau[off[i]:off[i + 1]] = np.linspace(-1.0, 1.0, n) if n > 1 else 0.0
    grp = np.arange(off.size - 1, dtype=np.int32) if group_of_interval is None else \
        np.asarray(group_of_interval, dtype=np.int32)
    return angle, tau.astype(np.float32), grp, int(grp.max()) + 1 if grp.size else 0


def add_hwp_signal(d: np.ndarray, interval_offsets, angle, tau, group, params) -> np.ndarray:
    """d + the half-wave-plate signal sum_k (b_k + tau b_{k+8}) cos k w + (b_{k+16} + tau b_{k+24}) sin k w
    in float32, params [n_groups, 32] (groups -1 add nothing); evaluated as the real part of
    sum_k (a_k - i s_k) e^{i k w} with a_k = b_k + tau b_{k+8}, s_k = b_{k+16} + tau b_{k+24}."""
    off = np.asarray(interval_offsets, dtype=np.int64)
    g = np.repeat(np.asarray(group, dtype=np.int64), np.diff(off))
    w = np.asarray(angle, dtype=np.float32).astype(np.float64)
    t = np.asarray(tau, dtype=np.float32).astype(np.float64)
    out = np.asarray(d, dtype=np.float64).copy()
    ok = g >= 0
    P = np.asarray(params, dtype=np.float64)[np.maximum(g, 0)]
    z = np.exp(1j * w)
    zk = np.ones_like(z)
    sig = np.zeros(out.shape[0])
    for k in range(8):
        zk = zk * z
        a = P[:, k] + t * P[:, 8 + k]
        s = P[:, 16 + k] + t * P[:, 24 + k]
        sig += np.real((a - 1j * s) * zk)
    out[ok] += sig[ok]
    return out.astype(np.float32)
