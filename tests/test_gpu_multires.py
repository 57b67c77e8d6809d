"""Multi-resolution Stokes maps on the GPU (Section 6: I on one pixelisation,
Q and U on a coarser one) against the FP64 oracle ``oracle.multires``.

Tolerances as in test_gpu_parity: operator applications 1e-11 (FP64 and
double-float) and 2e-5 (float32) relative RMS, maps 1e-10; indexing and
excision bit for bit.
"""

from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_helpers import cuda, host, lib_lags
from tests.helpers import lags_for, rel_rms

pytestmark = pytest.mark.gpu

FP64_OP_TOL = 1e-11
FP32_OP_TOL = 2e-5
FP64_MAP_TOL = 1e-10
MIXED_MAP_TOL = 1e-6


def _problem(seed=5, noiseless=False, width=8, factor=2, n=600, n_lags=10, lo=80, hi=300, flag_frac=0.0):
    from synth import make_flat_problem
    from synth.flat import log_uniform_intervals

    def lens(rng, tot):
        return log_uniform_intervals(tot, lo, hi, rng)
    return make_flat_problem("mr", seed, width, 4, n, 3, n_lags, det_angles_deg=[0.0, 45.0, 90.0, 135.0],
                             hwp_step_deg=22.5, interval_lengths=lens, noise=(1.0, 4.0, 1.5),
                             noiseless=noiseless, det_sweep_offset=True, pol_factor=factor, flag_frac=flag_frac)


def _planted(p):
    """A new I pixel and a new Q/U pixel seen only by five samples at one angle (the Q/U
    pixel is excised with its rows, which leaves the I pixel without rows), and a few
    samples flagged in one pixelisation only."""
    pix, pol, psi = p.pix.copy(), p.pix_pol.copy(), p.psi.copy()
    pix[:5], pol[:5], psi[:5] = p.n_pix, p.n_pix_pol, 0.3
    pix[40:43] = -1
    pol[90:94] = -1
    return pix, pol, psi, p.n_pix + 1, p.n_pix_pol + 1


def _inputs(p, kind):
    if kind == "planted":
        return _planted(p)
    return p.pix, p.pix_pol, p.psi, p.n_pix, p.n_pix_pol


def _system(p, kind="plain"):
    from oracle.multires import MultiResSystem
    pix, pol, psi, n_pix, n_pol = _inputs(p, kind)
    return MultiResSystem(pix, pol, psi, n_pix, n_pol, p.interval_offsets, p.interval_filter, lags_for(p))


def _plan(p, kind="plain", **kw):
    import torch
    from paper_0906_1775_gb300 import Plan
    pix, pol, psi, n_pix, n_pol = _inputs(p, kind)
    return Plan(torch.from_numpy(pix).cuda(), torch.from_numpy(psi).cuda(), n_pix, p.interval_offsets,
                p.interval_filter, lib_lags(p), pix_pol=torch.from_numpy(pol).cuda(), n_pix_pol=n_pol, **kw)


CASES = {
    "small": lambda: _problem(seed=5),
    "ragged": lambda: _problem(seed=11, n=3000, n_lags=33, lo=1, hi=2500, flag_frac=0.03),
    "factor4": lambda: _problem(seed=12, width=16, factor=4, n=2000, n_lags=16),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kind", ["plain", "planted"])
def test_indexing_and_excision_bit_exact(case, kind):
    p = CASES[case]()
    M = _system(p, kind)
    plan = _plan(p, kind)
    st = plan.stats
    assert plan.n_obs == M.n_obs and st["n_obs_pol"] == M.n_obs_pol
    o2g, exc = plan.observed()
    assert np.array_equal(host(o2g).astype(np.int64), M.obs2glob)
    assert np.array_equal(host(exc).astype(bool), M.excised[:M.n_obs_i])
    q2g, excq = plan.observed_pol()
    assert np.array_equal(host(q2g).astype(np.int64), M.obs2glob_pol)
    assert np.array_equal(host(excq).astype(bool), M.excised_pol[:M.n_obs_pol])
    assert st["n_excised"] == int(M.excised[:M.n_obs_i].sum())
    assert st["n_excised_pol"] == int(M.excised_pol[:M.n_obs_pol].sum())
    if kind == "planted":
        assert st["n_excised"] >= 1 and st["n_excised_pol"] >= 1


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kind", ["plain", "planted"])
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("fft_len", [0, 256])
def test_apply_ATNA_vs_oracle(case, kind, prec, fft_len):
    import torch
    p = CASES[case]()
    M = _system(p, kind)
    plan = _plan(p, kind, fft_len=fft_len)
    x = np.random.default_rng(3).standard_normal((M.n_obs, 3))
    dt = torch.float32 if prec == "fp32" else torch.float64
    y = host(plan.apply_ATNA(cuda(x, dt), precision=prec))[0]
    xin = x.astype(np.float32).astype(np.float64) if prec == "fp32" else x
    assert rel_rms(y, M.H(xin)) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_rhs_vs_oracle(case, prec):
    p = CASES[case]()
    M = _system(p, "planted")
    plan = _plan(p, "planted")
    b = host(plan.rhs(cuda(p.d), precision=prec))[0]
    assert rel_rms(b, M.rhs(p.d[0])) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


def test_same_pixelisation_equals_single_resolution_plan():
    """pix_pol = pix gives the single-resolution operator, right-hand side and map."""
    import torch
    from tests.gpu_helpers import make_plan
    from tests.helpers import tiny_IQU
    from paper_0906_1775_gb300 import Plan
    p = tiny_IQU(seed=41, n_per_det=800)
    single = make_plan(p)
    pix = torch.from_numpy(p.pix).cuda()
    multi = Plan(pix, torch.from_numpy(p.psi).cuda(), p.n_pix, p.interval_offsets, p.interval_filter, lib_lags(p),
                 pix_pol=pix, n_pix_pol=p.n_pix)
    assert multi.n_obs == single.n_obs
    x = cuda(np.random.default_rng(4).standard_normal((single.n_obs, 3)), torch.float64)
    ys, ym = host(single.apply_ATNA(x))[0], host(multi.apply_ATNA(x))[0]
    _, exc = single.observed()
    keep = ~host(exc).astype(bool)
    assert rel_rms(ym[keep], ys[keep]) < FP64_OP_TOL
    d = cuda(p.d[0])
    ms, _ = single.solve(d, precision="fp64", rel_tol=1e-13, max_iter=500)
    mm_, _ = multi.solve(d, precision="fp64", rel_tol=1e-13, max_iter=500)
    assert rel_rms(host(mm_)[keep], host(ms)[keep]) < FP64_MAP_TOL


@pytest.mark.parametrize("case", list(CASES))
def test_solve_fp64_matches_oracle(case):
    p = CASES[case]()
    M = _system(p, "planted")
    plan = _plan(p, "planted")
    d = cuda(p.d[0])
    for tol, maxit in [(1e-13, 1000), (1e-5, 1000), (1e-30, 7)]:
        m, info = plan.solve(d, precision="fp64", rel_tol=tol, max_iter=maxit)
        x, oi = M.solve(p.d[0], rel_tol=tol, max_iter=maxit)
        assert abs(info["iters"] - oi["iters"]) <= 1
        assert rel_rms(host(m), x) < (FP64_MAP_TOL if tol < 1e-10 else 1e-6)
        assert np.all(host(m)[~M.active()] == 0.0)


@pytest.mark.parametrize("refine", ["df64", "fp64"])
def test_solve_mixed_reaches_fp64_map(refine):
    p = CASES["factor4"]()
    M = _system(p, "planted")
    plan = _plan(p, "planted")
    m, info = plan.solve(cuda(p.d[0]), precision="mixed", rel_tol=1e-12, max_iter=1000, max_outer=20, refine=refine)
    x, _ = M.solve(p.d[0], rel_tol=1e-13, max_iter=1000)
    act = M.active()
    for s in range(3):
        assert rel_rms(host(m)[act[:, s], s], x[act[:, s], s]) < MIXED_MAP_TOL
    assert info["status"] == 0


def test_noiseless_recovery_on_gpu():
    p = _problem(seed=8, noiseless=True, n=1200)
    M = _system(p)
    plan = _plan(p)
    m, _ = plan.solve(cuda(p.d[0]), precision="fp64", rel_tol=1e-14, max_iter=2000)
    m = host(m)
    act = M.active()
    ki, kq = act[:, 0], act[:, 1]
    assert rel_rms(m[ki, 0], p.sky[M.obs2glob[ki[:M.n_obs_i]], 0]) < 1e-6
    assert rel_rms(m[kq, 1:], p.sky_pol[M.obs2glob_pol[kq[:M.n_obs_pol]]]) < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_batched_matches_single_solves(prec):
    p = CASES["small"]()
    M = _system(p, "planted")
    plan = _plan(p, "planted")
    rng = np.random.default_rng(5)
    D = np.stack([p.d[0], p.d[0] * 0.5 + rng.standard_normal(p.d[0].shape).astype(np.float32),
                  rng.standard_normal(p.d[0].shape).astype(np.float32)])
    ms, infos = plan.solve_batched(cuda(D), precision=prec, rel_tol=1e-12, max_iter=1000, max_outer=20)
    for k in range(3):
        x, _ = M.solve(D[k], rel_tol=1e-13, max_iter=1000)
        assert rel_rms(host(ms[k]), x) < (FP64_MAP_TOL if prec == "fp64" else MIXED_MAP_TOL)


def test_set_filters_matches_new_plan():
    import torch
    p = CASES["small"]()
    plan = _plan(p, "planted")
    lags2 = lib_lags(p) * 1.7
    lags2[:, 1:] *= 0.5
    plan.set_filters(lags2)
    from paper_0906_1775_gb300 import Plan
    pix, pol, psi, n_pix, n_pol = _planted(p)
    fresh = Plan(torch.from_numpy(pix).cuda(), torch.from_numpy(psi).cuda(), n_pix, p.interval_offsets,
                 p.interval_filter, lags2, pix_pol=torch.from_numpy(pol).cuda(), n_pix_pol=n_pol)
    assert plan.stats["n_excised"] == fresh.stats["n_excised"]
    assert plan.stats["n_excised_pol"] == fresh.stats["n_excised_pol"]
    d = cuda(p.d[0])
    m1, i1 = plan.solve(d, precision="fp64", rel_tol=1e-13, max_iter=800)
    m2, i2 = fresh.solve(d, precision="fp64", rel_tol=1e-13, max_iter=800)
    assert i1["iters"] == i2["iters"] and rel_rms(host(m1), host(m2)) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_backward_matches_oracle_adjoint(prec):
    from oracle.adjoint import solve_backward
    p = _problem(seed=14, n=1500, n_lags=12)
    M = _system(p, "planted")
    plan = _plan(p, "planted")
    d = cuda(p.d[0])
    m, _ = plan.solve(d, precision="fp64", rel_tol=1e-13, max_iter=2000)
    g = np.random.default_rng(6).standard_normal(m.shape)
    gd, gl, info = plan.solve_backward(d, m, cuda(g), precision=prec, rel_tol=1e-12, max_iter=2000)
    ogd, ogl, _ = solve_backward(M, p.d[0].astype(np.float64), host(m), g)
    assert rel_rms(host(gd), ogd) < 2e-5
    assert rel_rms(host(gl), ogl) < 2e-5


def test_checkpoint_and_resume():
    import paper_0906_1775_gb300 as mm
    p = CASES["factor4"]()
    plan = _plan(p, "planted")
    d = cuda(p.d[0])
    kw = dict(precision="fp64", rel_tol=1e-12, max_iter=1000)
    m0, i0 = plan.solve(d, **kw)
    states = []
    m_stop, i_stop = plan.solve(d, checkpoint_every=5, on_checkpoint=lambda s: states.append(s) or True, **kw)
    assert i_stop["status"] == mm._lib.MADMAP_STOPPED and i_stop["iters"] == 5
    m1, i1 = _plan(p, "planted").solve_resume(states[0], rel_tol=kw["rel_tol"], max_iter=kw["max_iter"])
    assert i1["iters"] == i0["iters"] and rel_rms(host(m1), host(m0)) < 1e-11


def test_bad_multires_inputs_are_rejected():
    import torch
    import paper_0906_1775_gb300 as mm
    from paper_0906_1775_gb300 import Plan
    p = CASES["small"]()
    pix = torch.from_numpy(p.pix).cuda()
    psi = torch.from_numpy(p.psi).cuda()
    bad = p.pix_pol.copy()
    bad[7] = p.n_pix_pol
    with pytest.raises(mm.MadmapError) as e:
        Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, lib_lags(p),
             pix_pol=torch.from_numpy(bad).cuda(), n_pix_pol=p.n_pix_pol)
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG and "pix_pol" in str(e.value)
    with pytest.raises(mm.MadmapError) as e:   # temperature-only plans have no Q/U
        Plan(pix, None, p.n_pix, p.interval_offsets, p.interval_filter, lib_lags(p),
             pix_pol=torch.from_numpy(p.pix_pol).cuda(), n_pix_pol=p.n_pix_pol)
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG
    with pytest.raises(mm.MadmapError):
        Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, lib_lags(p),
             pix_pol=torch.from_numpy(p.pix_pol).cuda(), n_pix_pol=0)


def test_all_samples_flagged_in_one_pixelisation():
    """Every sample flagged in the Q/U pixelisation: nothing is observed, the solve is empty."""
    import torch
    from paper_0906_1775_gb300 import Plan
    p = CASES["small"]()
    pol = np.full_like(p.pix_pol, -1)
    plan = Plan(torch.from_numpy(p.pix).cuda(), torch.from_numpy(p.psi).cuda(), p.n_pix, p.interval_offsets,
                p.interval_filter, lib_lags(p), pix_pol=torch.from_numpy(pol).cuda(), n_pix_pol=p.n_pix_pol)
    assert plan.n_obs == 0 and plan.stats["n_obs_pol"] == 0
    m, info = plan.solve(cuda(p.d[0]), precision="fp64")
    assert m.numel() == 0
