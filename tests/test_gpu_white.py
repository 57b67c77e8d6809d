"""White noise (one filter lag): the operator takes a single diagonal pass
(k_diag) instead of the FFT windows.  Every pointing layout against the FP64
oracle, and against the FFT path that batched solves still take.

Tolerances as in test_gpu_parity (1e-11 FP64 and double-float operator,
2e-5 float32 operator, 1e-10 FP64 maps, 1e-6 mixed maps).
"""

from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_helpers import cuda, host
from tests.helpers import rel_rms, tiny_IQU, tiny_T

pytestmark = pytest.mark.gpu

FP64_OP_TOL = 1e-11
FP32_OP_TOL = 2e-5
FP64_MAP_TOL = 1e-10


def _white(n_filters, seed=0):
    return np.random.default_rng(seed).uniform(0.5, 2.0, (n_filters, 1))


def _layout(kind):
    """(oracle system, plan factory, d) of one pointing layout with white noise."""
    import torch
    from paper_0906_1775_gb300 import Plan
    from oracle.solver import System
    if kind in ("T", "IQU"):
        p = tiny_T(seed=91, n=5000, width=10, ivls=(1, 2000, 1999, 1000), n_lags=1, flag_frac=0.05) if kind == "T" \
            else tiny_IQU(seed=92, n_per_det=2000, width=8, n_lags=1, flag_frac=0.03)
        lags = _white(p.n_filters, 1)
        S = System(p.pix, p.psi, p.n_pix, p.n_stokes, p.interval_offsets, p.interval_filter, lags, ninv="direct")
        def make(**kw):
            psi = torch.from_numpy(p.psi).cuda() if p.psi is not None else None
            return Plan(torch.from_numpy(p.pix).cuda(), psi, p.n_pix, p.interval_offsets, p.interval_filter, lags, **kw)
        return S, make, p.d[0]
    if kind == "multires":
        from synth import make_flat_problem
        from synth.flat import log_uniform_intervals
        from oracle.multires import MultiResSystem
        p = make_flat_problem("mrw", 93, 8, 4, 1500, 3, 1, det_angles_deg=[0.0, 45.0, 90.0, 135.0],
                              hwp_step_deg=22.5, interval_lengths=lambda rng, n: log_uniform_intervals(n, 80, 600, rng),
                              noise=(1.0, 4.0, 1.5), det_sweep_offset=True, pol_factor=2)
        lags = _white(p.n_filters, 2)
        S = MultiResSystem(p.pix, p.pix_pol, p.psi, p.n_pix, p.n_pix_pol, p.interval_offsets, p.interval_filter, lags,
                           ninv="direct")

        def make(**kw):
            return Plan(torch.from_numpy(p.pix).cuda(), torch.from_numpy(p.psi).cuda(), p.n_pix, p.interval_offsets,
                        p.interval_filter, lags, pix_pol=torch.from_numpy(p.pix_pol).cuda(), n_pix_pol=p.n_pix_pol,
                        **kw)
        return S, make, p.d[0]
    if kind == "boresight":
        from synth.boresight import make_boresight_problem
        from synth.flat import log_uniform_intervals
        from oracle.gcp import expand
        p = make_boresight_problem("bw", 94, 16, 4, 3000, 4, 3, 1, det_angles_deg=[0.0, 45.0, 90.0, 135.0],
                                   interval_lengths=lambda rng, n: log_uniform_intervals(n, 200, 1500, rng),
                                   noise=(1.0, 3.0, 1.5))
        lags = _white(p.n_filters, 3)
        pix, c2, s2 = expand(p.boresight, p.bore_step, p.det, p.samples_per_det, p.width, p.height)
        S = System(pix, None, p.n_pix, 3, p.interval_offsets, p.interval_filter, lags, ninv="direct", weights=(c2, s2))

        def make(**kw):
            return Plan.from_boresight(torch.from_numpy(p.boresight).cuda(), p.bore_step, p.det, p.samples_per_det,
                                       p.width, p.height, True, p.interval_offsets, p.interval_filter, lags, **kw)
        return S, make, p.d[0]
    if kind == "extended":
        from synth.extended import add_extra_signal, baseline_index
        from oracle.extended import ExtendedSystem
        p = tiny_IQU(seed=95, n_per_det=2500, width=10, n_lags=1, n_ivl_lo=200, n_ivl_hi=1500)
        idx, n_extra = baseline_index(2500, 4, 128)
        lags = _white(p.n_filters, 4)
        d = add_extra_signal(p.d[0], idx, np.random.default_rng(5).normal(0.0, 2.0, n_extra))
        S = ExtendedSystem(p.pix, p.psi, p.n_pix, 3, p.interval_offsets, p.interval_filter, lags, idx, n_extra,
                           ninv="direct")

        def make(**kw):
            return Plan(torch.from_numpy(p.pix).cuda(), torch.from_numpy(p.psi).cuda(), p.n_pix, p.interval_offsets,
                        p.interval_filter, lags, extra_index=torch.from_numpy(idx).cuda(), n_extra=n_extra, **kw)
        return S, make, d
    raise ValueError(kind)


KINDS = ["T", "IQU", "multires", "boresight", "extended"]


@pytest.fixture(scope="module")
def layouts():
    return {k: _layout(k) for k in KINDS}


def _mask(S):
    return S.active() if hasattr(S, "active") else np.repeat(~S.excised[:, None], S.n_s, 1)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_diagonal_operator_vs_oracle(layouts, kind, prec):
    import torch
    S, make, _ = layouts[kind]
    plan = make()
    ms, n = plan.time_operator("fp32", reps=1)
    assert list(n) == [1, 0, 0]          # one diagonal pass, no FFT kernels
    act = _mask(S)
    x = np.random.default_rng(6).standard_normal((S.n_obs, S.n_s)) * act
    dt = torch.float32 if prec == "fp32" else torch.float64
    y = host(plan.apply_ATNA(cuda(x, dt), precision=prec))[0]
    xin = x.astype(np.float32).astype(np.float64) if prec == "fp32" else x
    assert rel_rms(y, S.H(xin)) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_diagonal_rhs_and_weighting_vs_oracle(layouts, kind, prec):
    import torch
    S, make, d = layouts[kind]
    plan = make()
    b = host(plan.rhs(cuda(d[None, :]), precision=prec))[0]
    assert rel_rms(b, S.rhs(d)) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)
    if prec != "df64":
        dt = torch.float32 if prec == "fp32" else torch.float64
        w = host(plan.apply_ninv(cuda(d[None, :], dt), precision=prec))[0]
        assert rel_rms(w, S.ninv(d.astype(np.float64))) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


@pytest.mark.parametrize("kind", KINDS)
def test_diagonal_solves_match_oracle_and_fft_path(layouts, kind):
    S, make, d = layouts[kind]
    plan = make()
    m, info = plan.solve(cuda(d), precision="fp64", rel_tol=1e-13, max_iter=3000)
    x, oi = S.solve(d, rel_tol=1e-13, max_iter=3000)
    assert rel_rms(host(m), x) < FP64_MAP_TOL
    mm_, _ = plan.solve(cuda(d), precision="mixed", rel_tol=1e-12, max_iter=3000, max_outer=30)
    act = _mask(S)
    assert rel_rms(host(mm_)[act], x[act]) < 1e-6
    # batched solves keep the FFT windows: the same map through the other path
    mb, _ = plan.solve_batched(cuda(d[None, :]), precision="fp64", rel_tol=1e-13, max_iter=3000)
    assert rel_rms(host(mb[0]), host(m)) < FP64_MAP_TOL
