"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances.  FP64 path: relative RMS <= 1e-10 for maps (the stated target)
and <= 1e-11 for single operator applications (an FFT of length M = 2^k has
relative error ~ k * 2^-53; a four-step transform and a few hundred summed
terms stay far below 1e-12).  FP32 operator: relative RMS <= 2e-5 (k * 2^-24
~ 1e-6 for the transforms, plus float32 accumulation of the scatter; 2e-5
leaves a 10x margin).  Pixel indexing is compared bit for bit.
"""

from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_helpers import cuda, dominant_lags, host, lib_lags, make_plan
from tests.helpers import lags_for, rel_rms, system_for, tiny_IQU, tiny_T

pytestmark = pytest.mark.gpu

FP64_OP_TOL = 1e-11
FP32_OP_TOL = 2e-5
FP64_MAP_TOL = 1e-10
MIXED_MAP_TOL = 1e-6


def _torch():
    import torch
    return torch


def _ragged(seed=0, n_stokes=1, lens=(1, 7, 300, 1000, 0, 2500, 77, 4096), width=8, n_lags=33, flag_frac=0.05):
    from synth import make_flat_problem

    def ivl(_rng, tot):
        return list(lens)

    n = sum(lens)
    return make_flat_problem("ragged", seed, width, 1 if n_stokes == 1 else 1, n, n_stokes, n_lags,
                             interval_lengths=ivl, noise=(1.0, 5.0, 1.5), flag_frac=flag_frac,
                             det_angles_deg=[10.0], hwp_step_deg=22.5)


# ------------------------------------------------------------------ indexing
@pytest.mark.parametrize("maker", [lambda: tiny_T(flag_frac=0.1), lambda: tiny_IQU(flag_frac=0.05),
                                   lambda: _ragged(3, 3)])
def test_observed_pixels_bit_exact(maker):
    p = maker()
    S = system_for(p)
    plan = make_plan(p)
    o2g, exc = plan.observed()
    assert plan.n_obs == S.n_obs
    assert np.array_equal(host(o2g).astype(np.int64), S.obs2glob)
    assert np.array_equal(host(exc).astype(bool), S.excised)


# ------------------------------------------------------------------ N^-1
@pytest.mark.parametrize("fft_len,tpc", [(0, 0), (256, 0), (256, 3), (1024, 1)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_ninv_vs_direct_sum(fft_len, tpc, prec):
    from oracle.noise import apply_ninv_direct
    torch = _torch()
    p = _ragged(1)
    lags = dominant_lags(1, p.n_lags, seed=5)
    plan = make_plan(p, lags=lags, fft_len=fft_len, tiles_per_chunk=tpc)
    y = np.random.default_rng(7).standard_normal(p.n_samples)
    dt = torch.float64 if prec == "fp64" else torch.float32
    w = host(plan.apply_ninv(cuda(y, dt), precision=prec))[0]
    ref = apply_ninv_direct(y.astype(np.float32).astype(np.float64) if prec == "fp32" else y, p.interval_offsets,
                            p.interval_filter, lags)
    assert rel_rms(w, ref) < (FP64_OP_TOL if prec == "fp64" else FP32_OP_TOL)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_ninv_multifilter_intervals(prec):
    from oracle.noise import apply_ninv_direct
    torch = _torch()
    p = tiny_IQU(n_per_det=700, n_lags=21, n_ivl_lo=20, n_ivl_hi=300)
    lags = dominant_lags(p.n_filters, p.n_lags, seed=9)
    plan = make_plan(p, lags=lags, fft_len=256)
    y = np.random.default_rng(3).standard_normal(p.n_samples)
    dt = torch.float64 if prec == "fp64" else torch.float32
    w = host(plan.apply_ninv(cuda(y, dt), precision=prec))[0]
    ref = apply_ninv_direct(y.astype(np.float32).astype(np.float64) if prec == "fp32" else y, p.interval_offsets,
                            p.interval_filter, lags)
    assert rel_rms(w, ref) < (FP64_OP_TOL if prec == "fp64" else FP32_OP_TOL)


# ------------------------------------------------------------------ H and b
CASES = {
    "tinyT": lambda: tiny_T(flag_frac=0.05),
    "tinyIQU": lambda: tiny_IQU(flag_frac=0.03),
    "raggedT": lambda: _ragged(2, 1),
    "raggedIQU": lambda: _ragged(4, 3, width=6),
}


# "df64": the double-float operator (float32 pairs, about 48 significant bits)
# is held to the float64 tolerance.
@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("fft_len", [0, 512])
def test_apply_ATNA_vs_oracle(case, prec, fft_len):
    torch = _torch()
    p = CASES[case]()
    S = system_for(p)
    plan = make_plan(p, fft_len=fft_len)
    x = np.random.default_rng(11).standard_normal((S.n_obs, p.n_stokes))
    dt = torch.float32 if prec == "fp32" else torch.float64
    y = host(plan.apply_ATNA(cuda(x, dt), precision=prec))[0]
    xin = x.astype(np.float32).astype(np.float64) if prec == "fp32" else x
    ref = S.H(xin)
    assert rel_rms(y, ref) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_rhs_vs_oracle(case, prec):
    p = CASES[case]()
    S = system_for(p)
    plan = make_plan(p)
    b = host(plan.rhs(cuda(p.d), precision=prec))[0]
    ref = S.rhs(p.d[0])
    assert rel_rms(b, ref) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL)


def test_operator_symmetric_positive_definite_on_gpu():
    torch = _torch()
    p = tiny_IQU(seed=31)
    plan = make_plan(p)
    rng = np.random.default_rng(0)
    o2g, exc = plan.observed()
    keep = ~host(exc).astype(bool)
    x = rng.standard_normal((plan.n_obs, 3)) * keep[:, None]
    y = rng.standard_normal((plan.n_obs, 3)) * keep[:, None]
    Hx = host(plan.apply_ATNA(cuda(x, torch.float64)))[0]
    Hy = host(plan.apply_ATNA(cuda(y, torch.float64)))[0]
    a, b = float(np.sum(y * Hx)), float(np.sum(x * Hy))
    assert abs(a - b) <= 1e-12 * abs(a)
    assert float(np.sum(x * Hx)) > 0


# ------------------------------------------------------------------ solves
@pytest.mark.parametrize("case", list(CASES))
def test_solve_fp64_matches_oracle(case):
    p = CASES[case]()
    S = system_for(p)
    plan = make_plan(p)
    d = cuda(p.d[0])
    for tol, maxit in [(1e-13, 400), (1e-5, 400), (1e-30, 7)]:
        m, info = plan.solve(d, precision="fp64", rel_tol=tol, max_iter=maxit)
        x, oi = S.solve(p.d[0], rel_tol=tol, max_iter=maxit)
        assert abs(info["iters"] - oi["iters"]) <= 1
        if info["iters"] == oi["iters"]:
            assert info["best_iter"] == oi["best_iter"]
        assert rel_rms(host(m), x) < (FP64_MAP_TOL if tol < 1e-10 else 1e-6)
        assert info["best_rel_res"] == pytest.approx(oi["best_res"], rel=1e-6, abs=1e-14)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("refine", ["df64", "fp64"])
@pytest.mark.parametrize("restart", [False, True])
def test_solve_mixed_reaches_fp64_map(case, refine, restart):
    """Both refinement schemes: the float32 PCG continued across refinement steps by
    residual replacement (default) and restarted from zero at every step."""
    p = CASES[case]()
    S = system_for(p)
    plan = make_plan(p)
    m, info = plan.solve(cuda(p.d[0]), precision="mixed", rel_tol=1e-12, max_iter=600, max_outer=20, refine=refine,
                         inner_restart=restart)
    x, _ = S.solve(p.d[0], rel_tol=1e-13, max_iter=600)
    keep = ~S.excised
    for s in range(p.n_stokes):
        assert rel_rms(host(m)[keep, s], x[keep, s]) < MIXED_MAP_TOL
    # single-resolution stored pointing: the right-hand side is a float32 application and each
    # refinement residual b - H x = A^T N^-1 (d - A x) (Eq. 10) one full-precision application;
    # a continued solve may end on its recursive residual without the last one
    assert info["outer_iters"] >= 1
    if restart:
        assert info["fp64_applies"] == info["outer_iters"]
    else:
        assert info["outer_iters"] - 1 <= info["fp64_applies"] <= info["outer_iters"]
    assert info["fp32_applies"] == info["iters"] + 1


def test_continued_refinement_needs_no_more_iterations_than_restarts():
    """Residual replacement keeps the search direction across refinement steps, so
    the mixed solve to a tight tolerance needs at most the restarted scheme's inner
    iterations, and about as many as the float64 solve."""
    p = tiny_IQU(seed=9, n_per_det=2000, n_lags=64)
    S = system_for(p)
    plan = make_plan(p)
    d = cuda(p.d[0])
    x, _ = S.solve(p.d[0], rel_tol=1e-12, max_iter=1000)
    keep = ~S.excised
    its = {}
    for restart in (False, True):
        m, info = plan.solve(d, precision="mixed", rel_tol=1e-10, max_iter=1000, max_outer=20,
                             inner_restart=restart)
        assert info["status"] == 0 and info["best_rel_res"] <= 1e-10
        for s_ in range(3):
            assert rel_rms(host(m)[keep, s_], x[keep, s_]) < MIXED_MAP_TOL
        its[restart] = info["iters"]
    _, i64 = plan.solve(d, precision="fp64", rel_tol=1e-10, max_iter=1000)
    assert its[False] <= its[True]
    assert its[False] <= i64["iters"] + 5, (its, i64["iters"])


@pytest.mark.parametrize("case", ["tinyT", "tinyIQU"])
def test_mixed_stop_on_recursive_residual_is_honest(case):
    """A continued mixed solve that stops on its float32 recursive residual (after a
    full-precision residual replaced it) reports a residual that the oracle's own
    b - H m of the returned map confirms, and confirming every stop with a
    full-precision residual (final_residual) changes the map only at that level."""
    p = CASES[case]()
    S = system_for(p)
    plan = make_plan(p)
    d = cuda(p.d[0])
    keep = ~S.excised
    bref = S.rhs(p.d[0])
    bn = np.linalg.norm(bref[keep])
    maps = {}
    for fr in (False, True):
        m, info = plan.solve(d, precision="mixed", rel_tol=1e-9, max_iter=600, max_outer=20, inner_rel_tol=1e-3,
                             final_residual=fr)
        assert info["status"] == 0 and info["outer_iters"] >= 2
        mh = host(m)
        true = np.linalg.norm((bref - S.H(mh))[keep]) / bn
        assert true <= 2e-9, (fr, true, info["final_rel_res"])
        assert abs(true - info["final_rel_res"]) <= 0.5 * max(true, info["final_rel_res"]) + 1e-12
        if not fr:
            assert info["fp64_applies"] == info["outer_iters"] - 1
        maps[fr] = mh
    assert rel_rms(maps[False], maps[True]) < 1e-7


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_iteration_drivers_agree(prec):
    """Device-side loop (2), host-checked graph chunks (1) and direct launches (0)."""
    p = tiny_IQU(seed=5)
    plan = make_plan(p)
    d = cuda(p.d[0])
    runs = [plan.solve(d, precision=prec, rel_tol=1e-10, max_iter=200, use_graph=g, iters_per_sync=k)
            for g, k in ((2, 8), (1, 8), (0, 3))]
    for m, info in runs[1:]:
        # dot products reduce in a fixed order, but the scatter's float atomics do
        # not: float64 solves agree to rounding; mixed solves, whose float32 inner
        # products carry the atomics' order, agree to the stopping tolerance and
        # may stop one iteration apart when a residual lands at a threshold
        assert abs(info["iters"] - runs[0][1]["iters"]) <= (0 if prec == "fp64" else 1)
        assert rel_rms(host(m), host(runs[0][0])) < (1e-12 if prec == "fp64" else 1e-9)


def test_chunks_on_two_streams_match_one_launch():
    """Several chunks per application run on two plan streams (inside the solver's
    graphs too); operator and solves agree with the one-launch plan and the oracle."""
    torch = _torch()
    p = tiny_IQU(seed=23, n_per_det=2000, n_ivl_lo=100, n_ivl_hi=900)
    S = system_for(p)
    one = make_plan(p, fft_len=256)
    many = make_plan(p, fft_len=256, tiles_per_chunk=2)
    assert many.stats["n_tiles"] >= 8 and many.stats["tiles_per_chunk"] == 2
    x = np.random.default_rng(2).standard_normal((S.n_obs, 3))
    ref = S.H(x)
    for prec, tol in [("fp64", FP64_OP_TOL), ("df64", FP64_OP_TOL), ("fp32", FP32_OP_TOL)]:
        dt = torch.float32 if prec == "fp32" else torch.float64
        xin = x.astype(np.float32).astype(np.float64) if prec == "fp32" else x
        y = host(many.apply_ATNA(cuda(x, dt), precision=prec))[0]
        assert rel_rms(y, S.H(xin)) < tol, prec
    d = cuda(p.d[0])
    m1, i1 = one.solve(d, precision="mixed", rel_tol=1e-10, max_iter=300, max_outer=10)
    for g in (2, 1, 0):
        m2, i2 = many.solve(d, precision="mixed", rel_tol=1e-10, max_iter=300, max_outer=10, use_graph=g)
        assert i2["iters"] == i1["iters"] and rel_rms(host(m2), host(m1)) < 1e-9, g
    assert rel_rms(host(many.apply_ATNA(cuda(x, torch.float64)))[0], ref) < FP64_OP_TOL


def test_iteration_drivers_agree_batched():
    p = _batched_problem("T", 3)
    plan = make_plan(p)
    d = cuda(p.d)
    m2, i2 = plan.solve_batched(d, rel_tol=1e-11, max_iter=400, use_graph=2)
    m1, i1 = plan.solve_batched(d, rel_tol=1e-11, max_iter=400, use_graph=1, iters_per_sync=5)
    for r in range(3):
        assert i1[r]["iters"] == i2[r]["iters"]
        assert rel_rms(host(m1[r]), host(m2[r])) < 1e-12


def test_max_iter_cap_with_device_loop():
    p = tiny_IQU(seed=15)
    plan = make_plan(p)
    m, info = plan.solve(cuda(p.d[0]), rel_tol=1e-30, max_iter=4, use_graph=2)
    assert info["iters"] == 4 and info["status"] == 1


def test_white_noise_solve_is_binned_average():
    p = tiny_T(seed=8, ivls=(600,))
    plan = make_plan(p, lags=np.array([[1.0]]))
    m, info = plan.solve(cuda(p.d[0]), rel_tol=1e-14, max_iter=10)
    assert info["iters"] == 1
    o2g, _ = plan.observed()
    for q, g in enumerate(host(o2g)):
        assert host(m)[q, 0] == pytest.approx(float(np.mean(p.d[0][p.pix == g].astype(np.float64))), rel=1e-12)


def test_noiseless_recovery_on_gpu():
    p = tiny_IQU(seed=6, noiseless=True)
    plan = make_plan(p)
    m, _ = plan.solve(cuda(p.d[0]), rel_tol=1e-13, max_iter=500)
    o2g, exc = plan.observed()
    keep = ~host(exc).astype(bool)
    z = p.sky[host(o2g)]
    assert rel_rms(host(m)[keep], z[keep]) < 1e-6


# ------------------------------------------------------------------ full-size workloads
def test_config1_full_size_fp64():
    from synth import make_config
    p = make_config(1)
    S = system_for(p)
    plan = make_plan(p)
    d = cuda(p.d[0])
    m, info = plan.solve(d, precision="fp64", rel_tol=1e-8, max_iter=300)
    x, oi = S.solve(p.d[0], rel_tol=1e-8, max_iter=300)
    assert info["iters"] == oi["iters"]
    assert rel_rms(host(m), x) < FP64_MAP_TOL
    m2, _ = plan.solve(d, precision="fp64", rel_tol=1e-13, max_iter=300)
    x2, _ = S.solve(p.d[0], rel_tol=1e-13, max_iter=300)
    assert rel_rms(host(m2), x2) < FP64_MAP_TOL


@pytest.mark.parametrize("case", ["T", "IQU"])
def test_residual_history_matches_oracle(case):
    """The per-iteration relative residuals of a float64 solve equal the oracle PCG's
    (Section 5: ||r_k|| / ||b|| after every iteration), and the mixed solve's history
    follows its refinement steps down to the reported residual."""
    p = tiny_T(seed=3) if case == "T" else tiny_IQU(seed=4)
    S = system_for(p)
    plan = make_plan(p)
    d = cuda(p.d[0])
    m, info = plan.solve(d, precision="fp64", rel_tol=1e-12, max_iter=300, history=True)
    _, oi = S.solve(p.d[0], rel_tol=1e-12, max_iter=300)
    h = info["history"]
    assert info["history_len"] == info["iters"] + 1 == len(h)
    ref = np.asarray(oi["history"])
    n = min(len(h), len(ref))
    assert abs(len(h) - len(ref)) <= 1
    big = ref[:n] > 1e-9
    assert h[0] == 1.0
    assert np.max(np.abs(h[:n][big] - ref[:n][big]) / ref[:n][big]) < 1e-6
    assert info["t_pcg_ms"] > 0 and info["t_refine_ms"] == 0
    m2, i2 = plan.solve(d, precision="mixed", rel_tol=1e-10, max_iter=300, max_outer=10, history=True)
    h2 = i2["history"]
    assert i2["history_len"] == i2["iters"] + 1 == len(h2) and h2[0] == 1.0
    assert np.all(np.isfinite(h2)) and h2.min() <= 10 * i2["best_rel_res"]
    assert i2["t_pcg_ms"] > 0 and i2["t_refine_ms"] > 0
    assert i2["t_pcg_ms"] + i2["t_refine_ms"] + i2["t_rhs_ms"] <= i2["t_solve_ms"] + 1.0


@pytest.fixture(scope="module")
def config2():
    """The IQU flat-sky workload at full size (4 x 2^22 samples, 512 x 512 pixels, n_c = 2^14),
    its oracle system and the oracle's own PCG map solved to relative residual 1e-12."""
    from synth import make_config
    p = make_config(2)
    S = system_for(p)
    x_ref, info = S.solve(p.d[0], rel_tol=1e-12, max_iter=3000)
    assert info["best_res"] <= 1e-12
    return p, S, x_ref


def _stokes_errors(m, ref, keep):
    return [rel_rms(m[keep, s], ref[keep, s]) for s in range(ref.shape[1])]


def test_config2_operator_every_pixel(config2):
    """H x in the benchmark's launch configuration (compile-time geometry, M = 2^17 in
    two chunks on two streams) against the oracle's H x on every observed pixel."""
    torch = _torch()
    p, S, _ = config2
    plan = make_plan(p)
    assert plan.n_obs == S.n_obs
    o2g, exc = plan.observed()
    assert np.array_equal(host(o2g).astype(np.int64), S.obs2glob)
    assert np.array_equal(host(exc).astype(bool), S.excised)
    st = plan.stats
    assert st["fft_len"] == 1 << 17 and st["n_tiles"] > st["tiles_per_chunk"]
    x = np.random.default_rng(2).standard_normal((S.n_obs, 3))
    x[S.excised] = 0.0
    ref = S.H(x)
    for prec, tol in [("fp64", FP64_OP_TOL), ("df64", FP64_OP_TOL), ("fp32", FP32_OP_TOL)]:
        dt = torch.float32 if prec == "fp32" else torch.float64
        y = host(plan.apply_ATNA(cuda(x, dt), precision=prec))[0]
        assert rel_rms(y, ref) < tol, (prec, rel_rms(y, ref))
        for s in range(3):
            assert rel_rms(y[:, s], ref[:, s]) < tol, (prec, s)
    b = S.rhs(p.d[0])
    for prec, tol in [("fp64", FP64_OP_TOL), ("df64", FP64_OP_TOL), ("fp32", FP32_OP_TOL)]:
        bb = host(plan.rhs(cuda(p.d), precision=prec))[0]
        assert rel_rms(bb, b) < tol, (prec, rel_rms(bb, b))


def test_config2_maps_match_oracle_map(config2):
    """Maps of the benchmark's solvers against the oracle's PCG map (relative RMS per
    Stokes map over observed, non-excised pixels): float64 GPU PCG to 1e-12 within
    1e-10; the mixed solve (inner float32 tolerance 1e-4) and the float64 solve,
    both stopped at relative residual 1e-8, within 1e-6."""
    p, S, x_ref = config2
    plan = make_plan(p)
    keep = ~S.excised
    d = cuda(p.d[0])
    m64, i64 = plan.solve(d, precision="fp64", rel_tol=1e-12, max_iter=3000)
    assert max(_stokes_errors(host(m64), x_ref, keep)) < FP64_MAP_TOL, _stokes_errors(host(m64), x_ref, keep)
    mmx, imx = plan.solve(d, precision="mixed", rel_tol=1e-8, max_iter=3000, max_outer=30, inner_rel_tol=1e-4)
    errs = _stokes_errors(host(mmx), x_ref, keep)
    assert max(errs) < MIXED_MAP_TOL, errs
    m8, _ = plan.solve(d, precision="fp64", rel_tol=1e-8, max_iter=3000)
    errs = _stokes_errors(host(m8), x_ref, keep)
    assert max(errs) < MIXED_MAP_TOL, errs


def test_config2_mixed_solve_residual_by_oracle(config2):
    p, S, _ = config2
    plan = make_plan(p)
    m, info = plan.solve(cuda(p.d[0]), precision="mixed", rel_tol=1e-8, max_iter=400, max_outer=10)
    b = S.rhs(p.d[0])
    r = b - S.H(host(m))
    res = float(np.sqrt(np.sum(r * r) / np.sum(b * b)))
    assert res <= max(2.0 * info["best_rel_res"], 1e-8 * 1.5)


# ------------------------------------------------------------------ edge cases and errors
def test_empty_plan():
    torch = _torch()
    from paper_0906_1775_gb300 import Plan
    plan = Plan(torch.empty(0, dtype=torch.int32, device="cuda"), None, 16, np.array([0]), np.zeros(0, np.int32),
                np.array([[1.0, 0.1]]))
    assert plan.n_obs == 0
    m, info = plan.solve(torch.empty(0, dtype=torch.float32, device="cuda"))
    assert m.shape == (0, 1) and info["iters"] == 0


def test_invalid_pixel_is_rejected():
    torch = _torch()
    import paper_0906_1775_gb300 as mm
    pix = torch.tensor([0, 1, 5, 2], dtype=torch.int32, device="cuda")
    with pytest.raises(mm.MadmapError) as e:
        mm.Plan(pix, None, 4, np.array([0, 4]), np.array([0], np.int32), np.array([[1.0]]))
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG


def test_non_positive_definite_filter_is_rejected():
    torch = _torch()
    import paper_0906_1775_gb300 as mm
    pix = torch.tensor([0, 1, 2, 3] * 10, dtype=torch.int32, device="cuda")
    with pytest.raises(mm.MadmapError) as e:
        mm.Plan(pix, None, 4, np.array([0, 40]), np.array([0], np.int32), np.array([[1.0, 0.9, 0.9]]))
    assert e.value.status == mm._lib.MADMAP_ERR_NOT_PD


def test_bad_offsets_are_rejected():
    torch = _torch()
    import paper_0906_1775_gb300 as mm
    pix = torch.zeros(10, dtype=torch.int32, device="cuda")
    for off in ([0, 5], [0, 6, 4, 10], [1, 10]):
        with pytest.raises(mm.MadmapError):
            mm.Plan(pix, None, 4, np.array(off), np.zeros(len(off) - 1, np.int32), np.array([[1.0]]))


def test_injected_allocation_failure_reports_oom():
    import subprocess
    import sys
    code = (
        "import numpy as np, torch, paper_0906_1775_gb300 as mm\n"
        "pix = torch.zeros(10, dtype=torch.int32, device='cuda')\n"
        "try:\n"
        "    mm.Plan(pix, None, 4, np.array([0, 10]), np.zeros(1, np.int32), np.array([[1.0]]))\n"
        "    print('NOERR')\n"
        "except mm.MadmapError as e:\n"
        "    print('STATUS', e.status)\n")
    import os
    env = dict(os.environ, MADMAP_FAULT_ALLOC_FAIL_AT="3")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=root, timeout=300)
    assert "STATUS -3" in out.stdout, out.stdout + out.stderr


def test_single_sample_and_short_intervals():
    p = _ragged(8, 1, lens=(1, 1, 2, 3, 5, 8, 13, 21), width=3, n_lags=6, flag_frac=0.0)
    S = system_for(p)
    plan = make_plan(p)
    m, info = plan.solve(cuda(p.d[0]), rel_tol=1e-13, max_iter=200)
    x, _ = S.solve(p.d[0], rel_tol=1e-13, max_iter=200)
    assert rel_rms(host(m), x) < FP64_MAP_TOL


def test_set_filters_matches_new_plan():
    torch = _torch()
    p = tiny_IQU(seed=13)
    plan = make_plan(p)
    new = lib_lags(p) * 0.5
    new[:, 1:] *= 0.3
    new[:, 0] = 1.0 + 2 * np.abs(new[:, 1:]).sum(axis=1)
    plan.set_filters(new)
    fresh = make_plan(p, lags=new)
    x = np.random.default_rng(1).standard_normal((plan.n_obs, 3))
    a = host(plan.apply_ATNA(cuda(x, torch.float64)))
    b = host(fresh.apply_ATNA(cuda(x, torch.float64)))
    assert np.allclose(a, b, rtol=0, atol=1e-13 * np.abs(b).max())
    d = cuda(p.d[0])
    m1, _ = plan.solve(d, rel_tol=1e-12, max_iter=300)
    m2, _ = fresh.solve(d, rel_tol=1e-12, max_iter=300)
    assert rel_rms(host(m1), host(m2)) < 1e-12


def test_oracle_lags_agree_with_library_lags():
    p = tiny_IQU()
    assert np.allclose(lib_lags(p), lags_for(p), rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ batched right-hand sides
def _batched_problem(kind, n_rhs):
    from synth import make_config, make_flat_problem
    if kind == "T":
        return make_flat_problem("bT", 51, 6, 1, 3000, 1, 24, interval_lengths=lambda r, n: [700, 1300, 1000],
                                 noise=(1.0, 3.0, 1.7), n_rhs=n_rhs, flag_frac=0.02)
    if kind == "IQU":
        return make_flat_problem("bIQU", 52, 5, 4, 900, 3, 16, det_angles_deg=[0.0, 45.0, 90.0, 135.0],
                                 hwp_step_deg=22.5, noise=(1.0, 4.0, 1.5), n_rhs=n_rhs, det_sweep_offset=True)
    return make_config(4, scale=6, n_rhs=n_rhs)


@pytest.mark.parametrize("kind,n_rhs", [("T", 5), ("IQU", 3), ("IQU", 2), ("cfg4", 7)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_solve_batched_matches_single_solves_and_oracle(kind, n_rhs, prec):
    p = _batched_problem(kind, n_rhs)
    S = system_for(p)
    plan = make_plan(p)
    d = cuda(p.d)
    tol = 1e-12 if prec == "fp64" else 1e-10
    kw = dict(precision=prec, rel_tol=tol, max_iter=800, max_outer=20)
    mb, infos = plan.solve_batched(d, **kw)
    assert mb.shape == (n_rhs, plan.n_obs, p.n_stokes) and len(infos) == n_rhs
    keep = ~S.excised
    for r in range(n_rhs):
        m1, i1 = plan.solve(d[r].contiguous(), **kw)
        x, _ = S.solve(p.d[r], rel_tol=1e-13, max_iter=800)
        if prec == "fp64":
            assert infos[r]["iters"] == i1["iters"]
            assert rel_rms(host(mb[r]), host(m1)) < 1e-11
            assert rel_rms(host(mb[r]), x) < FP64_MAP_TOL
        else:
            for s in range(p.n_stokes):
                assert rel_rms(host(mb[r])[keep, s], x[keep, s]) < MIXED_MAP_TOL
        assert infos[r]["best_rel_res"] <= tol * 1.0001


def test_solve_batched_of_one_equals_solve():
    p = _batched_problem("IQU", 1)
    plan = make_plan(p)
    d = cuda(p.d)
    mb, ib = plan.solve_batched(d, rel_tol=1e-11, max_iter=300)
    m1, i1 = plan.solve(d[0].contiguous(), rel_tol=1e-11, max_iter=300)
    assert ib[0]["iters"] == i1["iters"]
    assert rel_rms(host(mb[0]), host(m1)) < 1e-12


def test_solve_batched_reuses_and_grows_buffers():
    p = _batched_problem("T", 6)
    plan = make_plan(p)
    d = cuda(p.d)
    m3, _ = plan.solve_batched(d[:3].contiguous(), rel_tol=1e-12, max_iter=500)
    m6, _ = plan.solve_batched(d, rel_tol=1e-12, max_iter=500)
    m3b, _ = plan.solve_batched(d[:3].contiguous(), rel_tol=1e-12, max_iter=500)
    for r in range(3):
        assert rel_rms(host(m6[r]), host(m3[r])) < 1e-11
        assert rel_rms(host(m3b[r]), host(m3[r])) < 1e-11


# ------------------------------------------------------------------ backward
def _bw_problem(kind):
    from synth import make_config
    if kind == "cfg5":
        return make_config(5, scale=8)
    return tiny_IQU(seed=71, n_per_det=500, n_lags=12, n_ivl_lo=40, n_ivl_hi=300)


@pytest.mark.parametrize("kind", ["tiny", "cfg5"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_backward_matches_oracle_adjoint(kind, prec):
    from oracle.adjoint import solve_backward
    p = _bw_problem(kind)
    S = system_for(p)
    plan = make_plan(p)
    d = cuda(p.d[0])
    m, _ = plan.solve(d, precision="fp64", rel_tol=1e-13, max_iter=2000)
    target = p.target[S.obs2glob] if p.target is not None else np.random.default_rng(1).standard_normal(m.shape)
    g = 2.0 * (host(m) - target)
    gd, gl, info = plan.solve_backward(d, m, cuda(g), precision=prec, rel_tol=1e-12, max_iter=2000)
    ogd, ogl, _ = solve_backward(S, p.d[0].astype(np.float64), host(m), g)
    assert rel_rms(host(gd), ogd) < 2e-5
    assert rel_rms(host(gl), ogl) < 2e-5
    assert info["best_rel_res"] <= 1e-12 * 1.0001


def test_backward_params_match_finite_differences():
    import torch
    import paper_0906_1775_gb300 as mm
    p = _bw_problem("cfg5")
    plan = make_plan(p)
    d = cuda(p.d[0])
    o2g, exc = plan.observed()
    keep = torch.from_numpy(~host(exc).astype(bool)).cuda()
    target = cuda(p.target[host(o2g)])
    kw = dict(precision="fp64", rel_tol=1e-13, max_iter=3000)

    def loss(params, dd):
        m = mm.MadmapSolve.apply(dd, params, plan, p.fs, kw)
        return ((m - target) ** 2)[keep].sum()

    params = torch.tensor(p.noise_params, dtype=torch.float64, requires_grad=True)
    dd = d.clone().requires_grad_(True)
    L = loss(params, dd)
    L.backward()
    gp = params.grad.numpy().copy()
    base = p.noise_params.copy()
    rng = np.random.default_rng(0)
    for k in rng.choice(p.n_filters, 3, replace=False):
        for j in range(3):
            h = 1e-4 * base[k, j]
            vals = []
            for sgn in (1, -1):
                prm = base.copy()
                prm[k, j] += sgn * h
                with torch.no_grad():
                    vals.append(float(loss(torch.tensor(prm), d)))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert gp[k, j] == pytest.approx(fd, rel=2e-3, abs=2e-3 * np.abs(gp).max())
    # d-gradient: exact directional derivative for a quadratic loss.  dL/dd comes from the
    # float32 weighting N^-1 (A lambda), so its error is relative to sum |g_t v_t|, not to the
    # (possibly cancelling) sum itself.
    v = torch.randn(d.shape, generator=torch.Generator(device="cuda").manual_seed(0), device="cuda")
    eps = 1e-2
    with torch.no_grad():
        fd = (float(loss(torch.tensor(base), d + eps * v)) - float(loss(torch.tensor(base), d - eps * v))) / (2 * eps)
    gv = dd.grad * v
    assert float(gv.sum()) == pytest.approx(fd, rel=1e-4, abs=1e-5 * float(gv.abs().sum()))
    # a common scale of every sigma leaves the map unchanged
    assert abs(float(np.sum(base[:, 0] * gp[:, 0]))) <= 1e-4 * float(np.sum(np.abs(base[:, 0] * gp[:, 0])))


# ------------------------------------------------------------------ small maps under many samples
@pytest.mark.parametrize("kind", ["T", "IQU"])
def test_replicated_scatter_of_small_heavily_hit_maps(kind):
    """A map of at most a few dozen rows under more than 1024 samples per row: the
    operator scatters into eight replicas and adds them up; every product still
    matches the oracle, including several right-hand sides in one call."""
    torch = _torch()
    if kind == "T":
        p = tiny_T(seed=101, n=40000, width=4, ivls=(15000, 15000, 10000), n_lags=16)
    else:
        p = tiny_IQU(seed=102, n_per_det=10000, width=3, n_lags=12, n_ivl_lo=2000, n_ivl_hi=6000)
    S = system_for(p)
    plan = make_plan(p)
    assert plan.stats["n_map_replicas"] == 8
    x = np.random.default_rng(12).standard_normal((3, S.n_obs, p.n_stokes))
    for prec in ("fp64", "df64", "fp32"):
        dt = torch.float32 if prec == "fp32" else torch.float64
        y = host(plan.apply_ATNA(cuda(x, dt), precision=prec))
        for k in range(3):
            xin = x[k].astype(np.float32).astype(np.float64) if prec == "fp32" else x[k]
            assert rel_rms(y[k], S.H(xin)) < (FP32_OP_TOL if prec == "fp32" else FP64_OP_TOL), prec
    b = host(plan.rhs(cuda(p.d), precision="fp64"))[0]
    assert rel_rms(b, S.rhs(p.d[0])) < FP64_OP_TOL
    m, info = plan.solve(cuda(p.d[0]), precision="fp64", rel_tol=1e-13, max_iter=400)
    xo, _ = S.solve(p.d[0], rel_tol=1e-13, max_iter=400)
    assert rel_rms(host(m), xo) < FP64_MAP_TOL
    mm_, _ = plan.solve(cuda(p.d[0]), precision="mixed", rel_tol=1e-12, max_iter=400, max_outer=20)
    keep = ~S.excised
    assert rel_rms(host(mm_)[keep], xo[keep]) < MIXED_MAP_TOL
