"""Small seeded problems shared by the oracle pins and the GPU parity tests."""

from __future__ import annotations

import numpy as np

from synth import make_flat_problem
from synth.flat import log_uniform_intervals


def tiny_T(seed=1, n=600, width=4, n_lags=8, ivls=(200, 250, 150), noiseless=False, flag_frac=0.0):
    def lens(_rng, tot):
        assert sum(ivls) == tot
        return list(ivls)
    return make_flat_problem("tinyT", seed, width, 1, n, 1, n_lags, interval_lengths=lens,
                             noise=(1.3, 5.0, 1.5), noiseless=noiseless, flag_frac=flag_frac)


def tiny_IQU(seed=2, n_per_det=320, width=4, n_lags=8, noiseless=False, n_ivl_lo=60, n_ivl_hi=200,
             flag_frac=0.0):
    def lens(rng, tot):
        return log_uniform_intervals(tot, n_ivl_lo, n_ivl_hi, rng)

    def nz(rng, nd):
        return np.stack([rng.uniform(0.8, 1.2, nd), rng.uniform(2.0, 8.0, nd), rng.uniform(1.0, 2.0, nd)], 1)

    return make_flat_problem("tinyIQU", seed, width, 4, n_per_det, 3, n_lags,
                             det_angles_deg=[0.0, 45.0, 90.0, 135.0], hwp_step_deg=22.5,
                             interval_lengths=lens, noise=nz, noiseless=noiseless, flag_frac=flag_frac,
                             det_sweep_offset=True)


def lags_for(problem, n_lags=None):
    """Oracle filter lags for every filter of a problem (oracle side only)."""
    from oracle.noise import filter_lags
    n_lags = problem.n_lags if n_lags is None else n_lags
    return np.stack([filter_lags(n_lags, problem.fs, *problem.noise_params[k])
                     for k in range(problem.n_filters)])


def system_for(problem, lags=None, **kw):
    from oracle.solver import System
    lags = lags_for(problem) if lags is None else lags
    return System(problem.pix, problem.psi, problem.n_pix, problem.n_stokes, problem.interval_offsets,
                  problem.interval_filter, lags, **kw)


def rel_rms(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.sqrt(np.sum((a - b) ** 2)) / max(np.sqrt(np.sum(b * b)), 1e-300))
