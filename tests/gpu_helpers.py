"""Helpers for the GPU parity tests: build library plans from synthetic problems.

The library side gets its filter lags from the library's own builder
(madmap_noise_filter); the oracle side from the oracle's.  Inputs shared by
both come from the seeded generators in ``synth`` or from the test itself.
"""

from __future__ import annotations

import numpy as np


def lib_lags(problem, n_lags=None):
    import paper_0906_1775_gb300 as mm
    n_lags = problem.n_lags if n_lags is None else n_lags
    return np.stack([mm.noise_filter(n_lags, problem.fs, *problem.noise_params[k]) for k in range(problem.n_filters)])


def make_plan(problem, lags=None, **kw):
    import torch
    from paper_0906_1775_gb300 import Plan
    lags = lib_lags(problem) if lags is None else lags

    def dev(a):
        return a.cuda() if isinstance(a, torch.Tensor) else torch.from_numpy(a).cuda()

    pix = dev(problem.pix)
    psi = dev(problem.psi) if problem.psi is not None else None
    return Plan(pix, psi, problem.n_pix, problem.interval_offsets, problem.interval_filter, lags, **kw)


def dominant_lags(n_filters, n_lags, seed=0):
    """Seeded strictly diagonally dominant (hence positive definite) filter lags."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((n_filters, n_lags)) * np.exp(-np.arange(n_lags) / 5.0)
    f[:, 0] = 1.0 + 2.0 * np.abs(f[:, 1:]).sum(axis=1)
    return f


def cuda(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().cpu().numpy()
