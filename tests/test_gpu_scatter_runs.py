"""The operator's scatter with run sums (lanes of one pixel add once).

When consecutive samples stay in one pixel, the column kernels sum each run
of lanes that hold the same map row before a single atomic.  The product
A^T N^-1 A x (Eq. 15) and the right-hand side A^T N^-1 d must be those of the
oracle within the usual tolerances whether the run sums are on or off, for
temperature and IQU maps, on scans whose runs are ragged (1 to 9 samples) and
cross window, tile and warp boundaries.  The plan's repeat fraction is the
exact count of samples whose successor hits the same observed pixel.
"""

from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_helpers import cuda, host, make_plan
from tests.helpers import rel_rms, system_for, tiny_IQU, tiny_T

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 2e-5


def _slow_scan(p, seed):
    """Hold each pointing for a ragged number of samples (1 .. 9)."""
    rng = np.random.default_rng(seed)
    n = p.n_samples
    lens = rng.integers(1, 10, size=n)
    starts = np.cumsum(np.concatenate([[0], lens]))[:-1]
    starts = starts[starts < n]
    src = np.repeat(starts, np.diff(np.concatenate([starts, [n]])))
    p.pix = np.ascontiguousarray(p.pix[src])
    return p


def _problems():
    t = _slow_scan(tiny_T(seed=71, n=60000, width=24, n_lags=300, ivls=(11000, 21000, 28000)), 1)
    q = _slow_scan(tiny_IQU(seed=72, n_per_det=12000, width=16, n_lags=300, n_ivl_lo=2000, n_ivl_hi=7000), 2)
    # flagged samples (pixel -1) inside and between the runs
    f = _slow_scan(tiny_IQU(seed=74, n_per_det=12000, width=16, n_lags=300, n_ivl_lo=2000, n_ivl_hi=7000,
                            flag_frac=0.05), 3)
    return {"T": t, "IQU": q, "IQU_flagged": f}


@pytest.fixture(scope="module")
def problems():
    return {k: (p, system_for(p)) for k, p in _problems().items()}


def _repeat_frac(p, S):
    pix = p.pix.astype(np.int64)
    row = np.full(p.n_pix, -1, dtype=np.int64)
    row[S.obs2glob[~S.excised]] = 1
    obs = (pix >= 0) & (row[np.maximum(pix, 0)] >= 0)
    same = obs[:-1] & (pix[:-1] == pix[1:])
    return int(same.sum()) / p.n_samples


# FFT lengths 2^13, 2^16, 2^20: runs of lanes of 32, 16 and 4 samples in the
# float32 kernels (the window columns each CTA holds)
@pytest.mark.parametrize("kind", ["T", "IQU", "IQU_flagged"])
@pytest.mark.parametrize("runs", [1, -1])
@pytest.mark.parametrize("fft_len", [1 << 13, 1 << 16, 1 << 20])
def test_operator_and_rhs_match_oracle_with_and_without_run_sums(problems, kind, runs, fft_len):
    import torch
    p, S = problems[kind]
    plan = make_plan(p, fft_len=fft_len, scatter_runs=runs)
    st = plan.stats
    assert st["scatter_runs"] == (1 if runs == 1 else 0)
    assert st["fft_len"] == fft_len and st["n_tiles"] >= (3 if fft_len == 1 << 13 else 2)
    x = np.random.default_rng(7).standard_normal((S.n_obs, p.n_stokes))
    bref = S.rhs(p.d[0])
    for prec, tol, dt in [("fp64", FP64_TOL, torch.float64), ("df64", FP64_TOL, torch.float64),
                          ("fp32", FP32_TOL, torch.float32)]:
        y = host(plan.apply_ATNA(cuda(x, dt), precision=prec))[0]
        ref = S.H(x.astype(np.float32).astype(np.float64) if prec == "fp32" else x)
        assert rel_rms(y, ref) < tol, (kind, runs, prec, rel_rms(y, ref))
        b = host(plan.rhs(cuda(p.d), precision=prec))[0]
        assert rel_rms(b, bref) < tol, (kind, runs, prec, rel_rms(b, bref))


def test_batched_operator_with_run_sums_matches_oracle(problems):
    """Three right-hand sides in one application (tile sets whose lanes carry
    their right-hand side) through the run-summed scatter."""
    import torch
    p, S = problems["IQU_flagged"]
    plan = make_plan(p, fft_len=1 << 13, scatter_runs=1)
    xs = np.random.default_rng(8).standard_normal((3, S.n_obs, 3))
    y = host(plan.apply_ATNA(cuda(xs, torch.float32), precision="fp32"))
    for k in range(3):
        ref = S.H(xs[k].astype(np.float32).astype(np.float64))
        assert rel_rms(y[k], ref) < FP32_TOL, (k, rel_rms(y[k], ref))


@pytest.mark.parametrize("kind", ["T", "IQU"])
def test_repeat_fraction_and_default_rule(problems, kind):
    p, S = problems[kind]
    plan = make_plan(p, fft_len=1 << 13)
    st = plan.stats
    frac = _repeat_frac(p, S)
    assert frac > 0.5
    assert st["repeat_frac"] == pytest.approx(frac, abs=0.5 / p.n_samples)
    assert st["scatter_runs"] == 1


def test_fast_scan_keeps_the_per_sample_scatter():
    p = tiny_IQU(seed=73, n_per_det=6000, width=16, n_lags=300, n_ivl_lo=2000, n_ivl_hi=5000)
    S = system_for(p)
    st = make_plan(p, fft_len=1 << 13).stats
    frac = _repeat_frac(p, S)
    assert st["repeat_frac"] == pytest.approx(frac, abs=0.5 / p.n_samples)
    assert st["scatter_runs"] == (1 if frac >= 0.25 else 0)
