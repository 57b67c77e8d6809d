"""Extended pointing on the GPU (Section 6, Eq. 40: destriping offsets and
binned synchronous templates as extra unit-weight columns) against the FP64
oracle ``oracle.extended``.

Tolerances as in test_gpu_parity: 1e-11 for FP64 and double-float operator
applications, 2e-5 for the float32 operator, 1e-10 for FP64 maps and 1e-6
for mixed maps; indexing and excision bit for bit.
"""

from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_helpers import cuda, host, lib_lags
from tests.helpers import lags_for, rel_rms, tiny_IQU, tiny_T

pytestmark = pytest.mark.gpu

FP64_OP_TOL = 1e-11
FP32_OP_TOL = 2e-5
FP64_MAP_TOL = 1e-10
MIXED_MAP_TOL = 1e-6
WHITE = np.array([[1.0]])


def _case(kind):
    """(problem, extra_index, n_extra, oracle lags, library lags, d)"""
    from synth.extended import add_extra_signal, baseline_index, chop_bins
    if kind == "destripe_T":       # white noise: one lag, no correlations
        p = tiny_T(seed=81, n=6000, width=12, ivls=(2500, 2300, 1200), n_lags=1)
        idx, n_extra = baseline_index(6000, 1, 100)
        o = np.random.default_rng(1).normal(0.0, 2.0, n_extra)
        return p, idx, n_extra, WHITE, WHITE, add_extra_signal(p.d[0], idx, o)
    if kind == "destripe_IQU":     # offsets on top of 1/f noise
        p = tiny_IQU(seed=82, n_per_det=2500, width=10, n_lags=16, n_ivl_lo=200, n_ivl_hi=1500)
        idx, n_extra = baseline_index(2500, 4, 128)
        o = np.random.default_rng(2).normal(0.0, 2.0, n_extra)
        return p, idx, n_extra, lags_for(p), lib_lags(p), add_extra_signal(p.d[0], idx, o)
    if kind == "template_IQU":     # a chopper-synchronous signal in 12 angle bins, flags, unused columns
        p = tiny_IQU(seed=83, n_per_det=2000, width=8, n_lags=12, flag_frac=0.03)
        idx, n_extra = chop_bins(p.n_samples, 12, 41.0, np.random.default_rng(3))
        amp = np.random.default_rng(4).normal(0.0, 1.0, n_extra)
        return p, idx, n_extra + 2, lags_for(p), lib_lags(p), add_extra_signal(p.d[0], idx, amp)
    if kind in ("hwp_IQU", "hwp_destripe"):   # the 32-parameter half-wave-plate model (+ offsets)
        from synth.extended import add_hwp_signal, hwp_inputs
        p = tiny_IQU(seed=85, n_per_det=2400, width=8, n_lags=12, n_ivl_lo=400, n_ivl_hi=1500)
        ang, tau, grp, n_groups = hwp_inputs(p.interval_offsets, p.fs, 1.7, np.random.default_rng(9))
        grp = grp.copy()
        grp[::3] = -1                          # some intervals without the term
        grp = np.where(grp >= 0, grp % 3, -1)  # three groups shared by several intervals
        b = np.random.default_rng(10).normal(0.0, 0.3, (3, 32))
        d = add_hwp_signal(p.d[0], p.interval_offsets, ang, tau, grp, b)
        if kind == "hwp_IQU":
            idx, n_extra = np.full(p.n_samples, -1, np.int32), 0
        else:
            idx, n_extra = baseline_index(2400, 4, 200)
            d = add_extra_signal(d, idx, np.random.default_rng(11).normal(0.0, 1.0, n_extra))
        return p, idx, n_extra, lags_for(p), lib_lags(p), d, (ang, tau, grp, 3)
    raise ValueError(kind)


CASES = ["destripe_T", "destripe_IQU", "template_IQU", "hwp_IQU", "hwp_destripe"]


def _system(c):
    from oracle.extended import ExtendedSystem
    p, idx, n_extra, olags = c[:4]
    return ExtendedSystem(p.pix, p.psi, p.n_pix, p.n_stokes, p.interval_offsets, p.interval_filter, olags, idx,
                          n_extra, hwp=c[6] if len(c) > 6 else None)


def _plan(c, **kw):
    import torch
    from paper_0906_1775_gb300 import Plan
    p, idx, n_extra, _, llags = c[:5]
    psi = torch.from_numpy(p.psi).cuda() if p.psi is not None else None
    ext = dict(extra_index=torch.from_numpy(idx).cuda(), n_extra=n_extra) if n_extra else {}
    if len(c) > 6:
        ang, tau, grp, ng = c[6]
        ext["hwp"] = (torch.from_numpy(ang).cuda(), torch.from_numpy(tau).cuda(), grp, ng)
    return Plan(torch.from_numpy(p.pix).cuda(), psi, p.n_pix, p.interval_offsets, p.interval_filter, llags,
                **ext, **kw)


@pytest.fixture(scope="module")
def cases():
    return {k: _case(k) for k in CASES}


@pytest.mark.parametrize("case", CASES)
def test_layout_and_excision(cases, case):
    c = cases[case]
    E = _system(c)
    plan = _plan(c)
    st = plan.stats
    assert plan.n_obs == E.n_obs and st["n_extra"] == E.n_extra
    o2g, exc = plan.observed()
    assert np.array_equal(host(o2g).astype(np.int64), E.obs2glob)
    assert np.array_equal(host(exc).astype(bool), E.excised_sky)
    assert st["n_excised"] == int(E.excised_sky.sum())
    assert st["n_excised_extra"] == int(E.excised_extra.sum())
    assert st["n_hwp_params"] == E.n_hwp and st["n_excised_hwp"] == int(E.excised_hwp.sum())
    if case == "template_IQU":
        assert st["n_excised_extra"] == 2


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("fft_len", [0, 256])
def test_apply_ATNA_vs_oracle(cases, case, prec, fft_len):
    import torch
    c = cases[case]
    E = _system(c)
    plan = _plan(c, fft_len=fft_len)
    x = np.random.default_rng(5).standard_normal((E.n_obs, E.n_s))
    dt = torch.float32 if prec == "fp32" else torch.float64
    y = host(plan.apply_ATNA(cuda(x, dt), precision=prec))[0]
    xin = x.astype(np.float32).astype(np.float64) if prec == "fp32" else x
    ref = E.H(xin * E.active())
    # inactive unknowns of the input (unused slots of the extra rows, excised pixels) have no row
    assert rel_rms(y * E.active(), ref) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_rhs_vs_oracle(cases, case, prec):
    c = cases[case]
    E = _system(c)
    plan = _plan(c)
    d = c[5]
    b = host(plan.rhs(cuda(d[None, :]), precision=prec))[0]
    assert rel_rms(b, E.rhs(d)) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


@pytest.mark.parametrize("case", CASES)
def test_solve_fp64_matches_oracle(cases, case):
    c = cases[case]
    E = _system(c)
    plan = _plan(c)
    d = c[5]
    for tol, maxit in [(1e-13, 3000), (1e-5, 3000), (1e-30, 7)]:
        m, info = plan.solve(cuda(d), precision="fp64", rel_tol=tol, max_iter=maxit)
        x, oi = E.solve(d, rel_tol=tol, max_iter=maxit)
        assert abs(info["iters"] - oi["iters"]) <= 1
        assert rel_rms(host(m), x) < (FP64_MAP_TOL if tol < 1e-10 else 1e-6)
        assert np.all(host(m)[~E.active()] == 0.0)


@pytest.mark.parametrize("case", ["destripe_T", "template_IQU", "hwp_destripe"])
def test_solve_mixed_reaches_fp64_map(cases, case):
    c = cases[case]
    E = _system(c)
    plan = _plan(c)
    d = c[5]
    m, info = plan.solve(cuda(d), precision="mixed", rel_tol=1e-12, max_iter=3000, max_outer=30)
    x, _ = E.solve(d, rel_tol=1e-13, max_iter=3000)
    act = E.active()
    for s in range(E.n_s):
        assert rel_rms(host(m)[act[:, s], s], x[act[:, s], s]) < MIXED_MAP_TOL


def test_destriping_recovers_offsets_on_gpu():
    """Noiseless T data with offsets and white noise: the GPU solution is the sky and the
    offsets (the reference baseline fixes the level)."""
    from synth.extended import add_extra_signal, baseline_index
    import torch
    from paper_0906_1775_gb300 import Plan
    p = tiny_T(seed=84, n=5000, width=10, ivls=(2500, 2500), n_lags=1, noiseless=True)
    idx, n_extra = baseline_index(5000, 1, 50)
    o = np.random.default_rng(6).normal(0.0, 3.0, n_extra)
    d = add_extra_signal(p.d[0], idx, o)
    plan = Plan(torch.from_numpy(p.pix).cuda(), None, p.n_pix, p.interval_offsets, p.interval_filter, WHITE,
                extra_index=torch.from_numpy(idx).cuda(), n_extra=n_extra)
    m, _ = plan.solve(cuda(d), precision="fp64", rel_tol=1e-14, max_iter=5000)
    m = host(m)
    o2g, _ = plan.observed()
    n_sky = plan.n_obs - n_extra
    assert rel_rms(m[:n_sky, 0], p.sky[host(o2g).astype(np.int64), 0]) < 1e-5
    assert rel_rms(m[n_sky:, 0], o) < 1e-5


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_batched_matches_oracle(cases, prec):
    c = cases["destripe_IQU"]
    E = _system(c)
    plan = _plan(c)
    rng = np.random.default_rng(7)
    D = np.stack([c[5], rng.standard_normal(c[5].shape).astype(np.float32)])
    ms, _ = plan.solve_batched(cuda(D), precision=prec, rel_tol=1e-12, max_iter=3000, max_outer=30)
    for k in range(2):
        x, _ = E.solve(D[k], rel_tol=1e-13, max_iter=3000)
        assert rel_rms(host(ms[k]), x) < (FP64_MAP_TOL if prec == "fp64" else MIXED_MAP_TOL)


@pytest.mark.parametrize("case", ["destripe_T", "template_IQU", "hwp_destripe"])
def test_backward_matches_oracle_adjoint(cases, case):
    from oracle.adjoint import solve_backward
    c = cases[case]
    E = _system(c)
    plan = _plan(c)
    d = c[5]
    m, _ = plan.solve(cuda(d), precision="fp64", rel_tol=1e-13, max_iter=3000)
    g = np.random.default_rng(8).standard_normal(m.shape)
    gd, gl, _ = plan.solve_backward(cuda(d), m, cuda(g), precision="fp64", rel_tol=1e-12, max_iter=3000)
    ogd, ogl, _ = solve_backward(E, d.astype(np.float64), host(m), g)
    assert rel_rms(host(gd), ogd) < 2e-5
    # The lag gradient sums products a_t r_t' (a = A lambda, r = d - A m) in float32:
    # its error is a few 1e-7 of ||a|| ||r||.  With a white-noise filter the lag-0
    # gradient vanishes at the ML map (A^T r = 0), so the bound is taken against
    # ||a|| ||r|| rather than the gradient itself.
    lam, _ = E.pcg(g * E.active(), rel_tol=1e-13, max_iter=3000)
    a = E.unpoint(lam)
    r = d.astype(np.float64) - E.unpoint(host(m))
    err = float(np.linalg.norm(host(gl) - ogl))
    assert err <= 2e-5 * max(float(np.linalg.norm(ogl)), float(np.linalg.norm(a) * np.linalg.norm(r)))
    if case != "destripe_T":
        assert rel_rms(host(gl), ogl) < 2e-5


def test_set_filters_matches_new_plan(cases):
    c = cases["template_IQU"]
    p = c[0]
    plan = _plan(c)
    lags2 = c[4] * 1.3
    lags2[:, 1:] *= 0.5
    plan.set_filters(lags2)
    fresh = _plan((c[0], c[1], c[2], c[3], lags2) + tuple(c[5:]))
    d = cuda(c[5])
    m1, i1 = plan.solve(d, precision="fp64", rel_tol=1e-13, max_iter=3000)
    m2, i2 = fresh.solve(d, precision="fp64", rel_tol=1e-13, max_iter=3000)
    assert i1["iters"] == i2["iters"] and rel_rms(host(m1), host(m2)) < 1e-12
    del p


def test_bad_extra_columns_are_rejected(cases):
    import torch
    import paper_0906_1775_gb300 as mm
    from paper_0906_1775_gb300 import Plan
    p, idx, n_extra, _, llags = cases["destripe_IQU"][:5]
    pix, psi = torch.from_numpy(p.pix).cuda(), torch.from_numpy(p.psi).cuda()
    bad = idx.copy()
    bad[11] = n_extra
    with pytest.raises(mm.MadmapError) as e:
        Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, llags, extra_index=torch.from_numpy(bad).cuda(),
             n_extra=n_extra)
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG and "extra_index" in str(e.value)
    with pytest.raises(mm.MadmapError):       # extended pointing is for single-resolution stored pointing
        Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, llags, extra_index=torch.from_numpy(idx).cuda(),
             n_extra=n_extra, pix_pol=pix, n_pix_pol=p.n_pix)
    with pytest.raises(mm.MadmapError):
        Plan(pix, psi, p.n_pix, p.interval_offsets, p.interval_filter, llags, extra_index=torch.from_numpy(idx).cuda(),
             n_extra=0)


def test_hwp_noiseless_recovery_on_gpu():
    """An injected half-wave-plate signal on an IQU sky, noiseless: the GPU solution holds the
    sky and the 32 parameters of each group."""
    import torch
    from synth.extended import add_hwp_signal, hwp_inputs
    from paper_0906_1775_gb300 import Plan
    p = tiny_IQU(seed=86, n_per_det=1500, width=5, noiseless=True, n_ivl_lo=500, n_ivl_hi=1500)
    ang, tau, grp, ng = hwp_inputs(p.interval_offsets, p.fs, 1.3, np.random.default_rng(12))
    b = np.random.default_rng(13).normal(0.0, 0.3, (ng, 32))
    d = add_hwp_signal(p.d[0], p.interval_offsets, ang, tau, grp, b)
    plan = Plan(torch.from_numpy(p.pix).cuda(), torch.from_numpy(p.psi).cuda(), p.n_pix, p.interval_offsets,
                p.interval_filter, lib_lags(p), hwp=(torch.from_numpy(ang).cuda(), torch.from_numpy(tau).cuda(), grp, ng))
    m, _ = plan.solve(cuda(d), precision="fp64", rel_tol=1e-14, max_iter=5000)
    m = host(m)
    n_sky = plan.n_obs - 32 * ng
    o2g, _ = plan.observed()
    for s in range(3):
        assert rel_rms(m[:n_sky, s], p.sky[host(o2g).astype(np.int64), s]) < 1e-5
    assert rel_rms(m[n_sky:, 0].reshape(ng, 32), b) < 1e-5
