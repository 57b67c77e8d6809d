"""Pointing expanded on the fly from compressed boresight pointing (Section 5.3)
on the GPU, against the oracle's expansion (``oracle.gcp``) fed to the FP64
oracle system.

Pixel indexing and excision are compared bit for bit; operator outputs and
maps with the tolerances of test_gpu_parity (1e-11 FP64 and double-float
operator, 2e-5 float32 operator, 1e-10 FP64 maps, 1e-6 mixed maps).  The
weights are float32 on both sides (the same operations), so the FP64 path is
held to the FP64 tolerances.
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


def _problem(kind):
    from synth.boresight import make_boresight_problem
    from synth.flat import log_uniform_intervals

    def ivl(lo, hi):
        return lambda rng, n: log_uniform_intervals(n, lo, hi, rng)
    if kind == "iqu":
        return make_boresight_problem("b", 31, 16, 4, 3000, 4, 3, 16, det_angles_deg=[0.0, 45.0, 90.0, 135.0],
                                      interval_lengths=ivl(200, 1500), noise=(1.0, 3.0, 1.5))
    if kind == "t":
        return make_boresight_problem("bt", 32, 16, 2, 4000, 8, 1, 24, interval_lengths=ivl(300, 2500),
                                      noise=(1.0, 3.0, 1.5))
    if kind == "ragged":
        return make_boresight_problem("br", 33, 32, 6, 5000, 8, 3, 33, interval_lengths=ivl(1, 2500),
                                      noise=(1.0, 5.0, 1.5), rot_period=3000)
    if kind == "slow":   # polarisers at 0 and 90 deg and a slow turn: pixels differ in conditioning
        return make_boresight_problem("bs", 36, 16, 2, 3000, 4, 3, 16, det_angles_deg=[0.0, 90.0],
                                      rot_period=60000, interval_lengths=ivl(200, 1500), noise=(1.0, 3.0, 1.5))
    raise ValueError(kind)


CASES = ["iqu", "t", "ragged", "slow"]


def _rc(p):
    """An excision threshold inside the widest relative gap of the oracle's rcond values
    (no pixel within a few percent of it, so both sides decide alike), or 0 for T."""
    if p.n_stokes == 1:
        return 0.0
    r = np.sort(_system(p).rcond)
    rel = r[1:] / np.maximum(r[:-1], 1e-300)
    i = int(np.argmax(rel))
    assert rel[i] > 1.02
    return float(np.sqrt(r[i] * r[i + 1]))


def _expand(p):
    """The oracle's expansion of a problem, kept with the problem."""
    from oracle.gcp import expand
    if "oracle_expansion" not in p.meta:
        p.meta["oracle_expansion"] = expand(p.boresight, p.bore_step, p.det, p.samples_per_det, p.width, p.height,
                                            polarised=p.n_stokes == 3)
    return p.meta["oracle_expansion"]


def _system(p, **kw):
    from oracle.solver import System
    pix, c2, s2 = _expand(p)
    return System(pix, None, p.n_pix, p.n_stokes, p.interval_offsets, p.interval_filter, lags_for(p),
                  weights=(c2, s2) if p.n_stokes == 3 else None, **kw)


def _plan(p, lags=None, **kw):
    import torch
    from paper_0906_1775_gb300 import Plan
    return Plan.from_boresight(torch.from_numpy(p.boresight).cuda(), p.bore_step, p.det, p.samples_per_det,
                               p.width, p.height, p.n_stokes == 3, p.interval_offsets, p.interval_filter,
                               lib_lags(p) if lags is None else lags, **kw)


@pytest.fixture(scope="module")
def problems():
    return {k: _problem(k) for k in CASES}


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("gap", [False, True])
def test_observed_and_excised_bit_exact(problems, case, gap):
    p = problems[case]
    rc = _rc(p) if gap else 0.0
    S = _system(p, **({"rcond_excise": rc} if rc else {}))
    plan = _plan(p, rcond_excise=rc)
    o2g, exc = plan.observed()
    assert plan.n_obs == S.n_obs
    assert np.array_equal(host(o2g).astype(np.int64), S.obs2glob)
    assert np.array_equal(host(exc).astype(bool), S.excised)
    assert plan.stats["n_excised"] == int(S.excised.sum())
    if rc and p.n_stokes == 3:
        assert 0 < S.excised.sum() < S.n_obs


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("fft_len", [0, 256])
def test_apply_ATNA_vs_oracle(problems, case, prec, fft_len):
    import torch
    p = problems[case]
    rc = _rc(p)
    S = _system(p, **({"rcond_excise": rc} if rc else {}))
    plan = _plan(p, rcond_excise=rc, fft_len=fft_len)
    x = np.random.default_rng(7).standard_normal((S.n_obs, p.n_stokes))
    dt = torch.float32 if prec == "fp32" else torch.float64
    y = host(plan.apply_ATNA(cuda(x, dt), precision=prec))[0]
    xin = x.astype(np.float32).astype(np.float64) if prec == "fp32" else x
    assert rel_rms(y, S.H(xin)) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_rhs_vs_oracle(problems, case, prec):
    p = problems[case]
    S = _system(p)
    plan = _plan(p)
    b = host(plan.rhs(cuda(p.d), precision=prec))[0]
    assert rel_rms(b, S.rhs(p.d[0])) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


@pytest.mark.parametrize("case", CASES)
def test_solve_fp64_matches_oracle(problems, case):
    p = problems[case]
    rc = _rc(p)
    S = _system(p, **({"rcond_excise": rc} if rc else {}))
    plan = _plan(p, rcond_excise=rc)
    d = cuda(p.d[0])
    for tol, maxit in [(1e-13, 600), (1e-5, 600), (1e-30, 7)]:
        m, info = plan.solve(d, precision="fp64", rel_tol=tol, max_iter=maxit)
        x, oi = S.solve(p.d[0], rel_tol=tol, max_iter=maxit)
        assert abs(info["iters"] - oi["iters"]) <= 1
        assert rel_rms(host(m), x) < (FP64_MAP_TOL if tol < 1e-10 else 1e-6)


@pytest.mark.parametrize("case", ["iqu", "ragged", "slow"])
@pytest.mark.parametrize("refine", ["df64", "fp64"])
def test_solve_mixed_reaches_fp64_map(problems, case, refine):
    p = problems[case]
    S = _system(p)
    plan = _plan(p)
    m, info = plan.solve(cuda(p.d[0]), precision="mixed", rel_tol=1e-12, max_iter=600, max_outer=20, refine=refine)
    x, _ = S.solve(p.d[0], rel_tol=1e-13, max_iter=600)
    keep = ~S.excised
    for s in range(p.n_stokes):
        assert rel_rms(host(m)[keep, s], x[keep, s]) < MIXED_MAP_TOL


def test_noiseless_recovery_on_gpu():
    from synth.boresight import make_boresight_problem
    p = make_boresight_problem("bn", 34, 16, 4, 6000, 4, 3, 16, det_angles_deg=[0.0, 45.0, 90.0, 135.0],
                               noiseless=True, noise=(1.0, 3.0, 1.5),
                               interval_lengths=lambda rng, n: [2000, 2500, 1500])
    plan = _plan(p)
    m, _ = plan.solve(cuda(p.d[0]), precision="fp64", rel_tol=1e-14, max_iter=1000)
    o2g, exc = plan.observed()
    keep = ~host(exc).astype(bool)
    sky = p.sky[host(o2g).astype(np.int64)]
    for s in range(3):
        assert rel_rms(host(m)[keep, s], sky[keep, s]) < 1e-5


def test_same_maps_as_stored_pointing():
    """The plan over stored pointing (the oracle's expansion: pixels, and angles
    psi = atan2(sin, cos) / 2 in float32) observes the same pixels and reaches the same
    map within the float32 rounding of the angles."""
    import torch
    from paper_0906_1775_gb300 import Plan
    p = _problem("iqu")
    pix, c2, s2 = _expand(p)
    psi = (0.5 * np.arctan2(s2.astype(np.float64), c2.astype(np.float64))).astype(np.float32)
    stored = Plan(torch.from_numpy(pix.astype(np.int32)).cuda(), torch.from_numpy(psi).cuda(), p.n_pix,
                  p.interval_offsets, p.interval_filter, lib_lags(p))
    otf = _plan(p)
    assert np.array_equal(host(stored.observed()[0]), host(otf.observed()[0]))
    d = cuda(p.d[0])
    m1, _ = stored.solve(d, precision="fp64", rel_tol=1e-12, max_iter=500)
    m2, _ = otf.solve(d, precision="fp64", rel_tol=1e-12, max_iter=500)
    assert rel_rms(host(m2), host(m1)) < 1e-5
    assert otf.stats["device_bytes"] < stored.stats["device_bytes"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_batched_matches_oracle(problems, prec):
    p = problems["iqu"]
    S = _system(p)
    plan = _plan(p)
    rng = np.random.default_rng(8)
    D = np.stack([p.d[0], rng.standard_normal(p.d[0].shape).astype(np.float32)])
    ms, _ = plan.solve_batched(cuda(D), precision=prec, rel_tol=1e-12, max_iter=600, max_outer=20)
    for k in range(2):
        x, _ = S.solve(D[k], rel_tol=1e-13, max_iter=600)
        assert rel_rms(host(ms[k]), x) < (FP64_MAP_TOL if prec == "fp64" else MIXED_MAP_TOL)


@pytest.mark.parametrize("case", ["iqu", "t"])
def test_backward_matches_oracle_adjoint(problems, case):
    from oracle.adjoint import solve_backward
    p = problems[case]
    S = _system(p)
    plan = _plan(p)
    d = cuda(p.d[0])
    m, _ = plan.solve(d, precision="fp64", rel_tol=1e-13, max_iter=1000)
    g = np.random.default_rng(9).standard_normal(m.shape)
    gd, gl, _ = plan.solve_backward(d, m, cuda(g), precision="fp64", rel_tol=1e-12, max_iter=1000)
    ogd, ogl, _ = solve_backward(S, p.d[0].astype(np.float64), host(m), g)
    assert rel_rms(host(gd), ogd) < 2e-5
    assert rel_rms(host(gl), ogl) < 2e-5


def test_set_filters_matches_new_plan(problems):
    p = problems["slow"]
    rc = _rc(p)
    plan = _plan(p, rcond_excise=rc)
    lags2 = lib_lags(p) * 0.7
    lags2[:, 1:] *= 0.6
    plan.set_filters(lags2)
    fresh = _plan(p, lags=lags2, rcond_excise=rc)
    assert plan.stats["n_excised"] == fresh.stats["n_excised"]
    d = cuda(p.d[0])
    m1, i1 = plan.solve(d, precision="fp64", rel_tol=1e-13, max_iter=800)
    m2, i2 = fresh.solve(d, precision="fp64", rel_tol=1e-13, max_iter=800)
    assert i1["iters"] == i2["iters"] and rel_rms(host(m1), host(m2)) < 1e-12


def test_bad_compressed_pointing_is_rejected(problems):
    import torch
    import paper_0906_1775_gb300 as mm
    from paper_0906_1775_gb300 import Plan
    p = problems["iqu"]
    bore = torch.from_numpy(p.boresight).cuda()
    lags = lib_lags(p)

    def make(**kw):
        a = dict(boresight=bore, bore_step=p.bore_step, det_pointing=p.det, samples_per_det=p.samples_per_det,
                 width=p.width, height=p.height, polarised=True, interval_offsets=p.interval_offsets,
                 interval_filter=p.interval_filter, filter_lags=lags)
        a.update(kw)
        return Plan.from_boresight(**a)

    cases = [
        dict(boresight=bore[:-1].contiguous()),                        # one node short
        dict(bore_step=0),
        dict(interval_offsets=np.array([0, p.n_samples // 2 + 1, p.n_samples]),   # spans two detectors
             interval_filter=np.array([0, 1], dtype=np.int32)),
    ]
    nan = p.boresight.copy()
    nan[3, 1] = np.nan
    cases.append(dict(boresight=torch.from_numpy(nan).cuda()))
    for kw in cases:
        with pytest.raises(mm.MadmapError) as e:
            make(**kw)
        assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG, kw
    plan = make()     # the valid description still plans
    assert plan.n_obs > 0


def test_no_rotation_single_angle_excises_every_pixel():
    """One detector whose focal plane never turns sees each pixel at one angle: every
    IQU pixel is excised and the solve returns zeros."""
    from synth.boresight import make_boresight_problem
    p = make_boresight_problem("b1", 35, 8, 1, 900, 4, 3, 8, rot_period=10 ** 12, noise=(1.0, 3.0, 1.5))
    S = _system(p)
    plan = _plan(p)
    assert S.excised.all() and plan.stats["n_excised"] == S.n_obs == plan.n_obs
    m, info = plan.solve(cuda(p.d[0]), precision="fp64", rel_tol=1e-10, max_iter=50)
    assert np.all(host(m) == 0.0)


@pytest.fixture(scope="module")
def config2_boresight():
    from synth.boresight import make_boresight_config2
    p = make_boresight_config2()
    S = _system(p)
    return p, S


def test_config2_boresight_observed_and_sampled_outputs(config2_boresight):
    """The IQU workload's shape (4 x 2^22 samples, 512 x 512) with compressed pointing:
    the observed set bit for bit and a sample of operator outputs against the oracle."""
    import torch
    p, S = config2_boresight
    plan = _plan(p)
    gp, _, _ = plan.expand_pointing()
    assert np.array_equal(host(gp).astype(np.int64), _expand(p)[0])
    assert plan.n_obs == S.n_obs
    o2g, exc = plan.observed()
    assert np.array_equal(host(o2g).astype(np.int64), S.obs2glob)
    assert np.array_equal(host(exc).astype(bool), S.excised)
    x = np.random.default_rng(2).standard_normal((S.n_obs, 3))
    pk = np.random.default_rng(3).choice(S.n_obs, 12, replace=False)
    ref = S.H_sampled(x, pk)
    for prec, tol in [("fp64", FP64_OP_TOL), ("fp32", 1e-4)]:
        dt = torch.float32 if prec == "fp32" else torch.float64
        y = host(plan.apply_ATNA(cuda(x, dt), precision=prec))[0]
        assert rel_rms(y[pk], ref) < tol, prec


@pytest.mark.parametrize("case", CASES)
def test_expanded_pointing_equals_oracle_bit_for_bit(problems, case):
    """Pixels and float32 weights of every sample, as the kernels compute them, equal the
    oracle's expansion exactly (the same float32 operations in the same order)."""
    p = problems[case]
    pix, c2, s2 = _expand(p)
    plan = _plan(p)
    gp, gc, gs = plan.expand_pointing()
    assert np.array_equal(host(gp).astype(np.int64), pix)
    if p.n_stokes == 3:
        ok = pix >= 0
        assert np.array_equal(host(gc)[ok], c2[ok]) and np.array_equal(host(gs)[ok], s2[ok])
    else:
        assert gc is None and gs is None


def test_expand_pointing_rejects_stored_pointing_plans():
    import paper_0906_1775_gb300 as mm
    from tests.gpu_helpers import make_plan
    from tests.helpers import tiny_IQU
    plan = make_plan(tiny_IQU(seed=3))
    with pytest.raises(mm.MadmapError) as e:
        plan.expand_pointing()
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG


@pytest.mark.parametrize("step,width,n_per", [(3, 24, 5000), (7, 21, 4000), (12, 24, 6000), (1, 8, 700)])
def test_expansion_with_other_node_steps(step, width, n_per):
    """Node steps that are not powers of two take the multiply-high division and the IEEE
    division of the interpolation fraction: pixels and weights still equal the oracle's."""
    from synth.boresight import make_boresight_problem
    p = make_boresight_problem("bstep", 40 + step, width, 3, n_per, step, 3, 8, noise=(1.0, 3.0, 1.5),
                               rot_period=5000)
    pix, c2, s2 = _expand(p)
    gp, gc, gs = _plan(p).expand_pointing()
    assert np.array_equal(host(gp).astype(np.int64), pix)
    ok = pix >= 0
    assert ok.sum() > 0.3 * pix.size
    assert np.array_equal(host(gc)[ok], c2[ok]) and np.array_equal(host(gs)[ok], s2[ok])


def test_expansion_of_a_long_detector_stream():
    """2^24 samples of one detector with a node every 7 samples (indices up to 2^24 through
    the step division), temperature only: every pixel equals the oracle's."""
    import torch
    from oracle.gcp import expand
    from paper_0906_1775_gb300 import Plan
    n_per, step, width = 1 << 24, 7, 448
    n_bore = (n_per - 1) // step + 2
    u = np.arange(n_bore, dtype=np.float64)
    bore = np.stack([width / 2 + 200 * np.sin(u * 1.1e-4), width / 2 + 200 * np.cos(u * 1.3e-4),
                     np.cos(u * 1e-5), np.sin(u * 1e-5)], 1).astype(np.float32)
    det = np.array([[0.3, -0.2, 1.0, 0.0]], dtype=np.float32)
    pix, _, _ = expand(bore, step, det, n_per, width, width, polarised=False)
    plan = Plan.from_boresight(torch.from_numpy(bore).cuda(), step, det, n_per, width, width, False,
                               np.array([0, n_per]), np.zeros(1, np.int32), np.array([[1.0, 0.1]]))
    gp, _, _ = plan.expand_pointing()
    assert np.array_equal(host(gp).astype(np.int64), pix)
