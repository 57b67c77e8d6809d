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
