"""The measuring autotuner (FFT length and tiles per launch chunk).

Section 5.2 picks the FFT length by a cost model; a plan created with
autotune times the float32 operator for candidate lengths and launch chunk
sizes and keeps the fastest.  Every candidate it may pick must give the same
exact product: each candidate's N^-1 is checked against the Eq. 15 direct sum,
and the tuned plan's operator and solve against the oracle.
"""

from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_helpers import cuda, host, make_plan
from tests.helpers import lags_for, rel_rms, system_for, tiny_IQU

pytestmark = pytest.mark.gpu


def _problem():
    return tiny_IQU(seed=51, n_per_det=6000, n_lags=300, n_ivl_lo=200, n_ivl_hi=5000)


def test_autotuned_plan_reports_candidates_and_keeps_the_fastest():
    p = _problem()
    plan = make_plan(p, autotune=True)
    st = plan.stats
    tuned = st["tuned"]
    assert st["n_tuned"] == len(tuned) >= 3
    lens = {m for m, _, _, _, _ in tuned}
    assert len(lens) >= 2 and all(m & (m - 1) == 0 and m > 2 * (p.n_lags - 1) for m in lens)
    assert all(ms > 0 for _, _, ms, _, _ in tuned)
    m_best, t_best, _, r_best, n2_best = min(tuned, key=lambda c: c[2])
    assert (st["fft_len"], st["tiles_per_chunk"], st["scatter_runs"], st["n2"]) == (m_best, t_best, r_best, n2_best)
    # both scatter modes and both column lengths were timed at the chosen length
    assert {r for m, t, _, r, _ in tuned if (m, t) == (m_best, t_best)} == {0, 1}
    lg = m_best.bit_length() - 1
    n_splits = 2 if 7 <= (lg + 1) // 2 - 1 and lg - ((lg + 1) // 2 - 1) <= 10 else 1
    assert len({n2 for m, t, _, _, n2 in tuned if (m, t) == (m_best, t_best)}) == n_splits


def test_every_candidate_length_gives_the_exact_product():
    import torch
    from oracle.noise import apply_ninv_direct
    p = _problem()
    tuned = make_plan(p, autotune=True).stats["tuned"]
    lags = lags_for(p)
    y = np.random.default_rng(3).standard_normal(p.n_samples)
    ref = apply_ninv_direct(y, p.interval_offsets, p.interval_filter, lags)
    for m, tpc, _, _, n2 in tuned:
        split = 1 if n2 < 1 << ((m.bit_length()) // 2) else 0
        plan = make_plan(p, fft_len=m, tiles_per_chunk=tpc, fft_split=split)
        assert plan.stats["n2"] == n2
        for prec, tol, dt in (("fp64", 1e-11, torch.float64), ("fp32", 2e-5, torch.float32)):
            w = host(plan.apply_ninv(cuda(y, dt), precision=prec))[0]
            assert rel_rms(w, ref) < tol, (m, tpc, prec, rel_rms(w, ref))


def test_autotuned_plan_operator_and_solve_match_oracle():
    import torch
    p = _problem()
    S = system_for(p)
    plan = make_plan(p, autotune=True)
    x = np.random.default_rng(4).standard_normal((S.n_obs, 3))
    x[S.excised] = 0.0
    y = host(plan.apply_ATNA(cuda(x, torch.float64), precision="fp64"))[0]
    assert rel_rms(y, S.H(x)) < 1e-11
    m, _ = plan.solve(cuda(p.d[0]), precision="fp64", rel_tol=1e-12, max_iter=1000)
    xo, _ = S.solve(p.d[0], rel_tol=1e-12, max_iter=1000)
    assert rel_rms(host(m), xo) < 1e-10


@pytest.mark.parametrize("fft_len", [1 << 13, 1 << 16, 1 << 17])
def test_shorter_columns_give_the_same_operator(fft_len):
    """fft_split = 1 (columns half the default length, rows twice): N^-1 against
    the Eq. 15 direct sum, A^T N^-1 A and the right-hand side against the oracle."""
    import torch
    from oracle.noise import apply_ninv_direct
    p = _problem()
    S = system_for(p)
    plan = make_plan(p, fft_len=fft_len, fft_split=1)
    lg = fft_len.bit_length() - 1
    assert plan.stats["n2"] == 1 << ((lg + 1) // 2 - 1) and plan.stats["n1"] * plan.stats["n2"] == fft_len
    y = np.random.default_rng(5).standard_normal(p.n_samples)
    ref = apply_ninv_direct(y, p.interval_offsets, p.interval_filter, lags_for(p))
    x = np.random.default_rng(6).standard_normal((S.n_obs, 3))
    for prec, tol, dt in (("fp64", 1e-11, torch.float64), ("df64", 1e-11, torch.float64),
                          ("fp32", 2e-5, torch.float32)):
        if prec != "df64":
            w = host(plan.apply_ninv(cuda(y, dt), precision=prec))[0]
            assert rel_rms(w, ref) < tol, (prec, rel_rms(w, ref))
        h = host(plan.apply_ATNA(cuda(x, dt), precision=prec))[0]
        href = S.H(x.astype(np.float32).astype(np.float64) if prec == "fp32" else x)
        assert rel_rms(h, href) < tol, (prec, rel_rms(h, href))
        b = host(plan.rhs(cuda(p.d), precision=prec))[0]
        assert rel_rms(b, S.rhs(p.d[0])) < tol, (prec, rel_rms(b, S.rhs(p.d[0])))


def test_shorter_columns_are_refused_where_rows_would_exceed_1024_points():
    import paper_0906_1775_gb300 as mm
    p = _problem()
    with pytest.raises(mm.MadmapError) as e:
        make_plan(p, fft_len=1 << 20, fft_split=1)
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG and "fft_split" in str(e.value)
