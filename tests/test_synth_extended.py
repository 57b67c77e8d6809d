"""Generators of the extended-pointing and compressed-pointing inputs (CPU)."""

from __future__ import annotations

import numpy as np


def test_baseline_index_numbers_baselines_across_detectors_and_skips_the_reference():
    from synth.extended import baseline_index
    idx, n = baseline_index(10, 3, 4, reference=1)
    # 3 baselines per detector (4, 4, 2 samples), 9 in all, baseline 1 without a column
    assert n == 8 and idx.shape == (30,) and idx.dtype == np.int32
    assert list(idx[:10]) == [0] * 4 + [-1] * 4 + [1] * 2
    assert list(idx[10:14]) == [2] * 4 and idx[-1] == 7
    assert set(np.unique(idx)) == set(range(-1, 8))


def test_chop_bins_cover_the_angle_range():
    from synth.extended import chop_bins
    idx, n = chop_bins(5000, 10, 37.0, np.random.default_rng(0))
    assert n == 9 and set(np.unique(idx)) == set(range(-1, 9))
    # a full sweep of 37 samples visits every bin at most ceil(37/10)+1 times in a row
    runs = np.diff(np.flatnonzero(np.diff(idx) != 0))
    assert runs.max() <= 5


def test_hwp_signal_equals_the_column_sum():
    """The generator's complex-exponential synthesis equals sum_i C_i b_i written from the
    column list (cos k w, tau cos k w, sin k w, tau sin k w)."""
    from synth.extended import add_hwp_signal, hwp_inputs
    off = np.array([0, 300, 700])
    ang, tau, grp, ng = hwp_inputs(off, 50.0, 0.7, np.random.default_rng(1))
    assert ng == 2 and list(grp) == [0, 1] and abs(tau[0] + 1) < 1e-7 and abs(tau[299] - 1) < 1e-7
    b = np.random.default_rng(2).normal(size=(2, 32))
    d = add_hwp_signal(np.zeros(700, np.float32), off, ang, tau, grp, b)
    t = 450
    w, tt, g = float(ang[t]), float(tau[t]), 1
    ref = sum((b[g, k - 1] + tt * b[g, 7 + k]) * np.cos(k * w) + (b[g, 15 + k] + tt * b[g, 23 + k]) * np.sin(k * w)
              for k in range(1, 9))
    assert abs(float(d[t]) - ref) < 1e-5 * max(1.0, abs(ref))


def test_boresight_nodes_start_lines_and_turn_off_the_grid():
    from synth.boresight import raster_nodes
    W, step = 16, 4
    L = W + 2 * step
    k = np.arange(0, 3 * W * L, step)
    x, y = raster_nodes(W, step, k)
    # every line starts on a node, outside the grid
    starts = (k % L) == 0
    assert np.all((x[starts] < 0) | (x[starts] > W) | (y[starts] < 0) | (y[starts] > W))
    # consecutive nodes within a line are step pixels apart along one axis
    same_line = (k[1:] // L) == (k[:-1] // L)
    dist = np.hypot(np.diff(x), np.diff(y))[same_line]
    assert np.allclose(dist, step)


def test_boresight_problem_shapes():
    from synth.boresight import make_boresight_problem
    p = make_boresight_problem("s", 3, 8, 2, 500, 4, 3, 6, noise=(1.0, 2.0, 1.5),
                               interval_lengths=lambda rng, n: [200, 300])
    assert p.boresight.shape == ((500 - 1) // 4 + 2, 4) and p.boresight.dtype == np.float32
    assert p.det.shape == (2, 4) and p.d.shape == (1, 1000) and p.n_pix == 64
    assert list(p.interval_offsets) == [0, 200, 500, 700, 1000]
    assert np.allclose(p.boresight[:, 2] ** 2 + p.boresight[:, 3] ** 2, 1.0, atol=1e-6)
