"""Pins for the FP64 oracle: each ties an oracle function to something other than itself
(a closed form, an invariant, brute force on tiny inputs, or the paper's own algebra).

CPU only (no GPU marker).
"""

from __future__ import annotations

import math

import numpy as np
import pytest

from oracle import noise as nz
from oracle import pointing as pt
from oracle.solver import System, pcg
from tests.helpers import lags_for, rel_rms, system_for, tiny_IQU, tiny_T


# ----------------------------------------------------------------------------- pointing
def test_observed_pixels_bruteforce():
    rng = np.random.default_rng(5)
    n_pix = 50
    pix = rng.integers(-1, n_pix, size=300).astype(np.int32)
    pix[pix == 17] = 3                                      # leave some pixels unobserved
    o2g, g2o = pt.observed_pixels(pix, n_pix)
    # Section 5.4 bit array, written as plain Python loops
    bits = [0] * n_pix
    for p in pix.tolist():
        if p >= 0:
            bits[p] = 1
    want = [g for g in range(n_pix) if bits[g]]
    assert o2g.tolist() == want
    for g in range(n_pix):
        assert g2o[g] == (want.index(g) if bits[g] else -1)


def test_weights_closed_form():
    psi = np.array([0.0, np.pi / 4, np.pi / 2, 3 * np.pi / 4], dtype=np.float32)
    w = pt.weights(psi, 3)
    want = np.array([[1, 1, 0], [1, 0, 1], [1, -1, 0], [1, 0, -1]], dtype=np.float64)
    assert np.allclose(w, want, atol=1e-7)
    assert pt.weights(psi, 1) is None


def test_point_is_transpose_of_unpoint():
    p = tiny_IQU()
    S = system_for(p)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((S.n_obs, 3))
    y = rng.standard_normal(p.n_samples)
    lhs = float(np.sum(S.unpoint(x) * y))
    rhs = float(np.sum(x * S.point(y)))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    A = pt.dense_pointing(S.pixl, S.w, S.n_obs, 3)
    assert np.allclose(A @ x.reshape(-1), S.unpoint(x), atol=1e-12)


# ----------------------------------------------------------------------------- N^-1
def _rand_lags(n_c, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n_c) * np.exp(-np.arange(n_c) / 3.0)


def test_ninv_impulse_and_constant_closed_forms():
    n_c = 6
    f = _rand_lags(n_c, 1)
    offs = np.array([0, 40, 55])
    filt = np.array([0, 0])
    lags = f[None, :]
    # impulse at t0 inside interval 0: response f(|t - t0|) inside the interval only
    y = np.zeros(55)
    y[37] = 1.0
    w = nz.apply_ninv_direct(y, offs, filt, lags)
    for t in range(55):
        want = f[abs(t - 37)] if (t < 40 and abs(t - 37) < n_c) else 0.0
        assert w[t] == pytest.approx(want, abs=1e-15)
    # constant input: interior = symbol at zero frequency; first sample = one-sided sum
    y = np.ones(55)
    w = nz.apply_ninv_direct(y, offs, filt, lags)
    assert w[20] == pytest.approx(f[0] + 2 * f[1:].sum(), rel=1e-14)
    assert w[0] == pytest.approx(f.sum(), rel=1e-14)
    assert w[40] == pytest.approx(f.sum(), rel=1e-14)     # first sample of interval 1


def test_ninv_sinusoid_eigen_interior():
    n_c = 9
    f = _rand_lags(n_c, 2)
    n = 200
    th = 0.37
    t = np.arange(n)
    y = np.cos(th * t)
    w = nz.apply_ninv_direct(y, np.array([0, n]), np.array([0]), f[None, :])
    S = f[0] + 2 * np.sum(f[1:] * np.cos(th * np.arange(1, n_c)))
    inner = slice(n_c, n - n_c)
    assert np.allclose(w[inner], S * y[inner], atol=1e-12)


@pytest.mark.parametrize("n_f", [None, 32, 64, 256])
def test_ninv_fft_overlap_save_equals_direct(n_f):
    rng = np.random.default_rng(3)
    n_c = 11
    lags = np.stack([_rand_lags(n_c, 4), _rand_lags(n_c, 5)])
    lens = [1, 7, 30, 31, 100, 333]
    offs = np.concatenate([[0], np.cumsum(lens)])
    filt = np.array([0, 1, 0, 1, 1, 0])
    y = rng.standard_normal(offs[-1])
    nf = nz.fft_length(n_c, max(lens)) if n_f is None else n_f
    a = nz.apply_ninv_fft(y, offs, filt, lags, nf)
    b = nz.apply_ninv_direct(y, offs, filt, lags)
    assert np.max(np.abs(a - b)) < 1e-12 * np.max(np.abs(b))


def test_ninv_direct_equals_dense_matrix():
    n_c = 5
    lags = np.stack([_rand_lags(n_c, 6), _rand_lags(n_c, 7)])
    offs = np.array([0, 3, 20, 33])
    filt = np.array([1, 0, 1])
    y = np.random.default_rng(8).standard_normal(33)
    M = nz.dense_ninv(offs, filt, lags)
    assert np.allclose(M, M.T)
    assert np.allclose(M @ y, nz.apply_ninv_direct(y, offs, filt, lags), atol=1e-13)


# ----------------------------------------------------------------------------- filter lags
def test_filter_white_noise_limit():
    f = nz.filter_lags(64, 100.0, 2.0, 0.0, 1.5)
    want = np.zeros(64)
    want[0] = 0.25
    assert np.allclose(f, want, atol=1e-15)


@pytest.mark.parametrize("fk", [0.05, 0.1, 0.2])
def test_filter_alpha2_lorentzian_closed_form(fk):
    # 1/p = (1/s^2) [1 - fk^2/(f^2 + fk^2)]; the Lorentzian transforms to
    # pi fk exp(-2 pi fk |t|), so c_tau = (1/s^2)[delta - (pi fk/fs) exp(-2 pi fk tau/fs)]
    # up to the band edge at fs/2, the finite-DC bin and aliasing (all < 1e-5 here).
    n_c, fs, s = 4096, 100.0, 1.7
    f = nz.filter_lags(n_c, fs, s, fk, 2.0)
    tau = np.arange(n_c)
    c = (tau == 0) - (math.pi * fk / fs) * np.exp(-2 * math.pi * fk * tau / fs)
    want = (1.0 - tau / n_c) * c / s ** 2
    assert np.max(np.abs(f - want)) < 2e-5 / s ** 2


def test_filter_sigma_scaling_and_taper():
    f1 = nz.filter_lags(128, 100.0, 1.0, 0.1, 1.3)
    f2 = nz.filter_lags(128, 100.0, 3.0, 0.1, 1.3)
    assert np.allclose(f2, f1 / 9.0, rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("params", [(1.0, 0.1, 2.0), (1.0, 0.05, 1.0), (1.0, 0.2, 2.0), (0.7, 0.03, 1.7),
                                    (1.0, 5.0, 1.5)])
def test_filter_toeplitz_positive_definite(params):
    n_c = 64
    f = nz.filter_lags(n_c, 100.0, *params)
    n = 3 * n_c
    T = np.array([[f[abs(i - j)] if abs(i - j) < n_c else 0.0 for j in range(n)] for i in range(n)])
    ev = np.linalg.eigvalsh(T)
    sym = nz.toeplitz_symbol(f, 8 * n_c)
    assert sym.min() > 0
    assert ev.min() > 0
    assert ev.min() >= sym.min() * (1 - 1e-9) - 1e-14      # Toeplitz spectrum within the symbol's range
    assert ev.max() <= sym.max() * (1 + 1e-9) + 1e-14


@pytest.mark.parametrize("k", [0, 1, 2])
def test_filter_gradient_central_difference(k):
    base = np.array([1.1, 0.12, 1.6])
    f, g = nz.filter_lags(256, 100.0, *base, with_grad=True)
    h = 1e-5 * base[k]
    up, dn = base.copy(), base.copy()
    up[k] += h
    dn[k] -= h
    fd = (nz.filter_lags(256, 100.0, *up) - nz.filter_lags(256, 100.0, *dn)) / (2 * h)
    assert np.max(np.abs(fd - g[k])) < 1e-6 * np.max(np.abs(g[k]))


# ----------------------------------------------------------------------------- FFT length
@pytest.mark.parametrize("n_c", [2 ** 8, 2 ** 10, 2 ** 12])
def test_optimal_nf_is_integer_argmin_of_h(n_c):
    root = nz.optimal_nf(n_c)
    n = np.arange(2 * n_c + 1, 60 * n_c, dtype=np.float64)
    hv = n * np.log(n) / (n - 2 * n_c)
    assert abs(n[np.argmin(hv)] - root) <= 1.0
    assert nz.hsecond(root, n_c) > 0                        # Appendix A


@pytest.mark.parametrize("x", [3000.0, 10000.0, 50000.0, 200000.0])
def test_hprime_matches_numerical_derivative(x):
    n_c = 1024
    e = 1e-5 * x
    fd = (nz.h(x + e, n_c) - nz.h(x - e, n_c)) / (2 * e)
    assert nz.hprime(x, n_c) == pytest.approx(fd, rel=1e-5)
    e2 = 1e-4 * x
    fd2 = (nz.hprime(x + e2, n_c) - nz.hprime(x - e2, n_c)) / (2 * e2)
    assert nz.hsecond(x, n_c) == pytest.approx(fd2, rel=1e-3)


@pytest.mark.parametrize("n_c,longest", [(2 ** 12, 2 ** 18), (2 ** 14, 2 ** 20), (2 ** 15, 648000),
                                          (2 ** 12, 5000), (16, 100)])
def test_fft_length_rule_brackets_optimum(n_c, longest):
    n_f = nz.fft_length(n_c, longest)
    assert n_f & (n_f - 1) == 0 and n_f > 2 * n_c
    opt = nz.optimal_nf(n_c)
    top = 1 << int(math.ceil(math.log2(longest + 1)))
    if n_f < top:                                 # the rule halved: optimum sits in (n_f/2, n_f]
        assert n_f / 2 < opt <= n_f or n_f // 2 <= 2 * n_c


# ----------------------------------------------------------------------------- preconditioner
def test_preconditioner_blocks_inverse_and_excision_closed_form():
    # pixel 0: angles 0/45/90/135 deg, m hits each -> A^T A = m diag(4,2,2), rcond = 1/2
    # pixel 1: angles 0/90 only -> U column zero -> singular -> excised
    m = 5
    ang = np.deg2rad(np.array([0.0, 45.0, 90.0, 135.0] * m + [0.0, 90.0] * m))
    pix = np.array([0] * (4 * m) + [1] * (2 * m), dtype=np.int32)
    offs = np.array([0, pix.size])
    lags = np.array([[2.0, 0.3]])
    S = System(pix, ang.astype(np.float32), 2, 3, offs, np.array([0]), lags)
    assert S.rcond[0] == pytest.approx(0.5, rel=1e-6)
    assert not S.excised[0] and S.excised[1]
    assert np.allclose(S.blocks[0], 2.0 * m * np.diag([4.0, 2.0, 2.0]), atol=1e-5)
    assert np.allclose(S.Pinv[0] @ S.blocks[0], np.eye(3), atol=1e-12)
    assert np.all(S.pixl[4 * m:] == -1)


def test_preconditioner_matches_dense_AtWA():
    p = tiny_IQU()
    S = system_for(p)
    A = pt.dense_pointing(S.pixl, S.w, S.n_obs, 3)
    f0 = np.repeat(S.lags[S.ivl_filter, 0], np.diff(S.offsets))
    AtWA = A.T @ (f0[:, None] * A)
    for q in range(S.n_obs):
        if S.excised[q]:
            continue
        blk = AtWA[3 * q:3 * q + 3, 3 * q:3 * q + 3]
        assert np.allclose(S.blocks[q], blk, rtol=1e-12, atol=1e-12)
        assert np.allclose(S.Pinv[q] @ blk, np.eye(3), atol=1e-10)


# ----------------------------------------------------------------------------- solve
@pytest.mark.parametrize("maker,ninv", [(tiny_T, "fft"), (tiny_T, "direct"), (tiny_IQU, "fft")])
def test_pcg_matches_dense_cholesky(maker, ninv):
    p = maker()
    S = system_for(p, ninv=ninv)
    x, info = S.solve(p.d[0], rel_tol=1e-14, max_iter=500)
    xd = S.dense_solve(p.d[0])
    assert rel_rms(x, xd) < 1e-10
    assert info["best_res"] <= 1e-13


def test_finite_termination():
    p = tiny_T(n=300, ivls=(300,), width=3)
    S = system_for(p)
    n_unk = S.n_obs
    _, info = S.solve(p.d[0], rel_tol=1e-12, max_iter=n_unk + 5)
    assert info["best_res"] <= 1e-12
    assert info["iters"] <= n_unk + 5


def test_h_norm_error_monotone_and_lowest_residual_rule():
    p = tiny_IQU(seed=7)
    S = system_for(p)
    b = S.rhs(p.d[0])
    xs = S.dense_solve(p.d[0])
    x, info = S.pcg(b, rel_tol=1e-30, max_iter=25, keep_history=True)
    errs = []
    for xi in info["iterates"]:
        e = (xi - xs).reshape(-1)
        errs.append(float(e @ S.H(e.reshape(S.n_obs, 3)).reshape(-1)))
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-9) + 1e-20 for i in range(len(errs) - 1))
    k = int(np.argmin(info["history"]))
    assert info["best_iter"] == k
    assert np.array_equal(x, info["iterates"][k])


def test_lowest_residual_rule_returns_earlier_iterate_when_residual_rises():
    # 2x2 SPD system where CG's residual goes up at step 1 (non-monotone residual norm)
    H = np.array([[1.0, 0.0], [0.0, 100.0]])
    b = np.array([1.0, 0.1])
    x, info = pcg(lambda v: H @ v, lambda r: r, b, 1e-30, 1, keep_history=True)
    hist = info["history"]
    assert hist[1] > hist[0]
    assert info["best_iter"] == 0 and np.all(x == 0)


def test_white_noise_limit_is_binned_average_T():
    p = tiny_T(seed=11, ivls=(600,))
    S = system_for(p, lags=np.array([[1.0]]))
    x, info = S.solve(p.d[0], rel_tol=1e-14, max_iter=10)
    assert info["iters"] == 1                      # exact block preconditioner: one step
    for q, g in enumerate(S.obs2glob):
        sel = p.pix == g
        assert x[q, 0] == pytest.approx(float(np.mean(p.d[0][sel].astype(np.float64))), rel=1e-12, abs=1e-12)


def test_white_noise_limit_is_binned_average_IQU():
    p = tiny_IQU(seed=12)
    lags = np.ones((p.n_filters, 1)) * 0.5
    S = system_for(p, lags=lags)
    x, info = S.solve(p.d[0], rel_tol=1e-14, max_iter=10)
    assert info["iters"] == 1
    two = 2.0 * p.psi.astype(np.float64)
    for q, g in enumerate(S.obs2glob):
        if S.excised[q]:
            continue
        sel = p.pix == g
        Ap = np.stack([np.ones(sel.sum()), np.cos(two[sel]), np.sin(two[sel])], 1)
        want = np.linalg.lstsq(Ap, p.d[0][sel].astype(np.float64), rcond=None)[0]
        assert np.allclose(x[q], want, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("maker", [tiny_T, tiny_IQU])
def test_noiseless_recovery(maker):
    p = maker(noiseless=True)
    S = system_for(p)
    x, _ = S.solve(p.d[0], rel_tol=1e-13, max_iter=500)
    z = p.sky[S.obs2glob]
    keep = ~S.excised
    assert rel_rms(x[keep], z[keep]) < 1e-6            # d is stored in float32


def test_operator_symmetric_positive_definite():
    p = tiny_IQU(seed=3)
    S = system_for(p)
    rng = np.random.default_rng(1)
    x = rng.standard_normal((S.n_obs, 3))
    y = rng.standard_normal((S.n_obs, 3))
    x[S.excised] = 0
    y[S.excised] = 0
    a = float(np.sum(x * S.H(y)))
    b = float(np.sum(y * S.H(x)))
    assert abs(a - b) <= 1e-12 * abs(a)
    assert float(np.sum(x * S.H(x))) > 0


def test_polarisation_relabelling():
    """Paper's row (1/2)[i + q sin 2a + u cos 2a] versus (I + Q cos 2psi + U sin 2psi)."""
    p = tiny_IQU(seed=4)
    S = system_for(p)
    xs = S.dense_solve(p.d[0])
    two = 2.0 * p.psi.astype(np.float64)
    keep_rows = S.pixl >= 0
    Ap = np.zeros((p.n_samples, S.n_obs * 3))
    for t in np.flatnonzero(keep_rows):
        q = S.pixl[t]
        Ap[t, 3 * q:3 * q + 3] = 0.5 * np.array([1.0, np.sin(two[t]), np.cos(two[t])])
    _, N, _ = S.dense_H()
    keep = np.repeat(~S.excised, 3)
    Hp = (Ap.T @ N @ Ap)[np.ix_(keep, keep)]
    bp = (Ap.T @ N @ p.d[0].astype(np.float64))[keep]
    iqu = np.zeros(S.n_obs * 3)
    iqu[keep] = np.linalg.solve(Hp, bp)
    iqu = iqu.reshape(S.n_obs, 3)
    ours = np.stack([iqu[:, 0] / 2, iqu[:, 2] / 2, iqu[:, 1] / 2], 1)
    assert rel_rms(xs, ours) < 1e-10


def test_flagged_samples_are_zero_rows():
    p = tiny_T(seed=9, flag_frac=0.2)
    S = system_for(p)
    y = np.random.default_rng(2).standard_normal(p.n_samples)
    y2 = y.copy()
    y2[p.pix < 0] += 1e6                           # data on flagged rows never reaches the map
    assert np.allclose(S.point(y), S.point(y2))
    xs = S.dense_solve(p.d[0])
    x, _ = S.solve(p.d[0], rel_tol=1e-13, max_iter=300)
    assert rel_rms(x, xs) < 1e-10


def test_sampled_operator_matches_full_operator():
    p = tiny_IQU(seed=21)
    S = system_for(p)
    x = np.random.default_rng(4).standard_normal((S.n_obs, 3))
    full = S.H(x)
    pk = [0, 5, S.n_obs // 2, S.n_obs - 1]
    assert np.allclose(S.H_sampled(x, pk), full[pk], rtol=1e-12, atol=1e-12 * np.abs(full).max())


# ----------------------------------------------------------------------------- adjoint
def _loss_setup(seed=61):
    from oracle.adjoint import solve_backward  # noqa: F401
    p = tiny_IQU(seed=seed, n_per_det=400, n_lags=12, n_ivl_lo=40, n_ivl_hi=250)
    rng = np.random.default_rng(seed)
    return p, rng


def _loss(S, d, target):
    m, _ = S.solve(d, rel_tol=1e-14, max_iter=3000)
    keep = ~S.excised
    return float(np.sum((m - target)[keep] ** 2)), m


def test_adjoint_grad_d_matches_finite_difference():
    from oracle.adjoint import solve_backward
    p, rng = _loss_setup()
    S = system_for(p)
    d = p.d[0].astype(np.float64)
    target = rng.standard_normal((S.n_obs, 3))
    L0, m = _loss(S, d, target)
    g = 2.0 * (m - target)
    gd, _, _ = solve_backward(S, d, m, g)
    for _ in range(3):
        v = rng.standard_normal(d.shape)
        eps = 1e-3
        fd = (_loss(S, d + eps * v, target)[0] - _loss(S, d - eps * v, target)[0]) / (2 * eps)
        assert float(gd @ v) == pytest.approx(fd, rel=1e-8)


def test_adjoint_lag_gradient_matches_finite_difference():
    from oracle.adjoint import solve_backward
    p, rng = _loss_setup(62)
    lags = lags_for(p)
    S = system_for(p, lags=lags)
    d = p.d[0].astype(np.float64)
    target = rng.standard_normal((S.n_obs, 3))
    _, m = _loss(S, d, target)
    _, gf, _ = solve_backward(S, d, m, 2.0 * (m - target))
    for _ in range(3):
        delta = rng.standard_normal(lags.shape) * np.abs(lags).max() * 1e-2
        eps = 1e-3
        lp = system_for(p, lags=lags + eps * delta)
        lm = system_for(p, lags=lags - eps * delta)
        fd = (_loss(lp, d, target)[0] - _loss(lm, d, target)[0]) / (2 * eps)
        assert float(np.sum(gf * delta)) == pytest.approx(fd, rel=1e-6)


def test_adjoint_psd_parameter_gradient_and_sigma_invariance():
    from oracle.adjoint import params_gradient, solve_backward
    p, rng = _loss_setup(63)
    S = system_for(p)
    d = p.d[0].astype(np.float64)
    target = rng.standard_normal((S.n_obs, 3))
    _, m = _loss(S, d, target)
    _, gf, _ = solve_backward(S, d, m, 2.0 * (m - target))
    gp = params_gradient(gf, p.n_lags, p.fs, p.noise_params)
    base = p.noise_params.copy()
    for k in range(p.n_filters):
        for j in range(3):
            h = 1e-4 * base[k, j]
            vals = []
            for sgn in (1, -1):
                prm = base.copy()
                prm[k, j] += sgn * h
                from oracle.noise import filter_lags
                lg = np.stack([filter_lags(p.n_lags, p.fs, *prm[q]) for q in range(p.n_filters)])
                vals.append(_loss(system_for(p, lags=lg), d, target)[0])
            fd = (vals[0] - vals[1]) / (2 * h)
            assert gp[k, j] == pytest.approx(fd, rel=2e-4, abs=1e-9 * np.abs(gp).max())
    # scaling every sigma together scales N^-1 uniformly: the map does not move
    s_dot = float(np.sum(base[:, 0] * gp[:, 0]))
    assert abs(s_dot) <= 1e-8 * float(np.sum(np.abs(base[:, 0] * gp[:, 0])))


# ------------------------------------------------------------------ multi-resolution maps (Section 6)
def _mr_problem(seed=5, noiseless=False, width=8, factor=2, n=600):
    from synth import make_flat_problem
    from synth.flat import log_uniform_intervals

    def lens(rng, tot):
        return log_uniform_intervals(tot, 80, 300, rng)
    return make_flat_problem("mr", seed, width, 4, n, 3, 10, det_angles_deg=[0.0, 45.0, 90.0, 135.0],
                             hwp_step_deg=22.5, interval_lengths=lens, noise=(1.0, 4.0, 1.5),
                             noiseless=noiseless, det_sweep_offset=True, pol_factor=factor)


def _mr_system(p, pix_pol=None, n_pix_pol=None, **kw):
    from oracle.multires import MultiResSystem
    from tests.helpers import lags_for
    pp = p.pix_pol if pix_pol is None else pix_pol
    npp = p.n_pix_pol if n_pix_pol is None else n_pix_pol
    return MultiResSystem(p.pix, pp, p.psi, p.n_pix, npp, p.interval_offsets, p.interval_filter, lags_for(p), **kw)


def test_multires_reduces_to_single_resolution():
    """With the same pixel for I and Q/U the operator and the right-hand side are those of
    the single-resolution system (Eq. 10), and so is the map."""
    p = _mr_problem(seed=6)
    M = _mr_system(p, pix_pol=p.pix, n_pix_pol=p.n_pix)
    S = system_for(p)
    assert M.n_obs == S.n_obs and not S.excised.any() and not M.excised.any() and not M.excised_pol.any()
    x = np.random.default_rng(1).standard_normal((S.n_obs, 3))
    assert np.allclose(M.H(x), S.H(x), rtol=1e-12, atol=1e-12 * np.abs(S.H(x)).max())
    assert np.allclose(M.rhs(p.d[0]), S.rhs(p.d[0]), rtol=1e-12, atol=1e-12)
    xm, _ = M.solve(p.d[0], rel_tol=1e-13, max_iter=500)
    xs, _ = S.solve(p.d[0], rel_tol=1e-13, max_iter=500)
    assert rel_rms(xm, xs) < 1e-10


def test_multires_pcg_matches_dense_cholesky_and_is_symmetric():
    p = _mr_problem(seed=7)
    M = _mr_system(p)
    assert M.n_obs_pol < M.n_obs_i
    xd = M.dense_solve(p.d[0])
    xp, info = M.solve(p.d[0], rel_tol=1e-13, max_iter=1000)
    assert info["best_res"] < 1e-12
    act = M.active()
    assert rel_rms(xp[act], xd[act]) < 1e-10 and np.all(xp[~act] == 0)
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal((2, M.n_obs, 3)) * act
    a, b = float(np.sum(y * M.H(x))), float(np.sum(x * M.H(y)))
    assert abs(a - b) <= 1e-12 * abs(a) and float(np.sum(x * M.H(x))) > 0


def test_multires_noiseless_recovery():
    """Noiseless data whose Q and U are constant within Q/U pixels: the map recovers I on the
    fine pixels and Q, U on the coarse ones."""
    p = _mr_problem(seed=8, noiseless=True, n=1200)
    M = _mr_system(p)
    x, _ = M.solve(p.d[0], rel_tol=1e-14, max_iter=2000)
    act = M.active()
    ki = act[:, 0]
    kq = act[:, 1]
    assert ki.sum() > 50 and kq.sum() > 10
    assert rel_rms(x[ki, 0], p.sky[M.obs2glob[ki[:M.n_obs_i]], 0]) < 1e-6
    assert rel_rms(x[kq, 1:], p.sky_pol[M.obs2glob_pol[kq[:M.n_obs_pol]]]) < 1e-6


def test_multires_excision_drops_rows():
    """A Q/U pixel seen at a single angle cannot separate Q from U: it is excised, its rows
    are zero, and an I pixel seen only through those rows is excised too."""
    p = _mr_problem(seed=9)
    pix, pol, psi = p.pix.copy(), p.pix_pol.copy(), p.psi.copy()
    n_pix_pol = p.n_pix_pol + 1
    n_pix = p.n_pix + 1
    pix[:5], pol[:5], psi[:5] = p.n_pix, p.n_pix_pol, 0.3     # new I and Q/U pixels, one angle
    from oracle.multires import MultiResSystem
    from tests.helpers import lags_for
    M = MultiResSystem(pix, pol, psi, n_pix, n_pix_pol, p.interval_offsets, p.interval_filter, lags_for(p))
    k_pol = int(np.searchsorted(M.obs2glob_pol, p.n_pix_pol))
    k_i = int(np.searchsorted(M.obs2glob, p.n_pix))
    assert M.excised_pol[k_pol] and M.excised[k_i]
    assert np.all(M.pi[:5] == -1) and np.all(M.pq[:5] == -1)
    assert not M.excised[:M.n_obs_i][np.arange(M.n_obs_i) != k_i].any()


# ------------------------------------------------------------------ compressed pointing (Section 5.3)
def _exact_expand(bore, step, det, n_per_det, width, height):
    """The expansion in exact rational arithmetic (one sample at a time)."""
    from fractions import Fraction as Fr
    out = []
    for d in range(len(det)):
        dx, dy, cd, sd = (Fr(float(v)) for v in det[d])
        for j in range(n_per_det):
            u, r = divmod(j, step)
            f = Fr(r, step)
            q = [Fr(float(bore[u][k])) + f * (Fr(float(bore[u + 1][k])) - Fr(float(bore[u][k]))) for k in range(4)]
            x, y, c, s = q
            X, Y = x + c * dx - s * dy, y + s * dx + c * dy
            ix, iy = X.numerator // X.denominator, Y.numerator // Y.denominator
            C, S = c * cd - s * sd, s * cd + c * sd
            n = C * C + S * S
            ok = 0 <= ix < width and 0 <= iy < height and n > 0
            out.append((iy * width + ix if ok else -1, (C * C - S * S) / n if n else None,
                        2 * C * S / n if n else None))
    return out


def test_gcp_dyadic_cases_equal_rational_arithmetic():
    """Nodes, offsets and orientations chosen so every float32 step is exact: the pixels
    and weights equal those of exact rational arithmetic (interpolation from node u to
    u + 1, the rotation's signs, the pixel's row-major order, the double angle)."""
    from oracle.gcp import expand
    rng = np.random.default_rng(3)
    width, height, step, n_per = 7, 5, 4, 37
    n_bore = (n_per - 1) // step + 2
    bore = np.zeros((n_bore, 4), dtype=np.float32)
    bore[:, 0] = rng.integers(-4, 64, n_bore) / 8.0
    bore[:, 1] = rng.integers(-4, 44, n_bore) / 8.0
    rots = np.array([(1, 0), (0, 1), (-1, 0), (0, -1), (0.5, 0.5), (0.75, -0.25)], dtype=np.float32)
    bore[:, 2:] = rots[rng.integers(0, len(rots), n_bore)]
    det = np.array([[0.0, 0.0, 1.0, 0.0], [0.25, -0.5, 0.0, 1.0], [-0.375, 0.125, 0.5, -0.5]], dtype=np.float32)
    pix, c2, s2 = expand(bore, step, det, n_per, width, height)
    exact = _exact_expand(bore, step, det, n_per, width, height)
    assert np.array_equal(pix, np.array([e[0] for e in exact]))
    assert (pix >= 0).sum() > 60 and (pix < 0).sum() > 0
    for t, (p, ce, se) in enumerate(exact):
        if ce is not None:
            assert abs(float(c2[t]) - float(ce)) <= 2e-7 and abs(float(s2[t]) - float(se)) <= 2e-7


def test_gcp_weights_are_the_double_angle_of_the_summed_orientation():
    from oracle.gcp import expand
    rng = np.random.default_rng(4)
    a = rng.uniform(-np.pi, np.pi, 50)
    b = rng.uniform(-np.pi, np.pi, 3)
    bore = np.stack([np.full(50, 3.3), np.full(50, 2.2), np.cos(a), np.sin(a)], 1).astype(np.float32)
    det = np.stack([np.zeros(3), np.zeros(3), np.cos(b), np.sin(b)], 1).astype(np.float32)
    pix, c2, s2 = expand(bore, 1, det, 49, 8, 8)        # step 1: every sample sits on a node
    ang = (a[None, :49] + b[:, None]).reshape(-1)
    assert np.all(pix == 2 * 8 + 3)
    assert np.max(np.abs(c2 - np.cos(2 * ang))) < 1e-6 and np.max(np.abs(s2 - np.sin(2 * ang))) < 1e-6


def test_gcp_pixels_follow_the_float64_position_away_from_edges():
    """On a random smooth path the float32 expansion and the same geometry in float64
    agree on the pixel wherever the float64 position is 1e-3 pixel or more from an edge."""
    from oracle.gcp import expand
    rng = np.random.default_rng(5)
    width, step, n_per = 32, 8, 3000
    n_bore = (n_per - 1) // step + 2
    t = np.arange(n_bore)
    ang = 0.01 * t + 0.3
    bore = np.stack([16 + 12 * np.sin(0.013 * t), 16 + 12 * np.cos(0.017 * t), np.cos(ang), np.sin(ang)], 1)
    bore = bore.astype(np.float32)
    det = np.array([[0.4, -0.3, 1.0, 0.0], [-0.45, 0.2, 0.0, 1.0]], dtype=np.float32)
    pix, _, _ = expand(bore, step, det, n_per, width, width)
    b64 = bore.astype(np.float64)
    for d in range(2):
        j = np.arange(n_per)
        u, f = j // step, (j % step) / step
        q = b64[u] + f[:, None] * (b64[u + 1] - b64[u])
        X = q[:, 0] + q[:, 2] * det[d, 0] - q[:, 3] * det[d, 1]
        Y = q[:, 1] + q[:, 3] * det[d, 0] + q[:, 2] * det[d, 1]
        far = (np.abs(X - np.round(X)) > 1e-3) & (np.abs(Y - np.round(Y)) > 1e-3)
        ref = np.floor(Y).astype(np.int64) * width + np.floor(X).astype(np.int64)
        got = pix[d * n_per:(d + 1) * n_per]
        assert far.sum() > 0.9 * n_per
        assert np.array_equal(got[far], ref[far])


def test_gcp_flags_outside_and_degenerate_orientation():
    from oracle.gcp import expand
    bore = np.array([[-0.5, 1.5, 1, 0], [0.5, 1.5, 1, 0], [3.5, 1.5, 0, 0], [3.5, 3.5, 0, 0]], dtype=np.float32)
    det = np.array([[0, 0, 1, 0]], dtype=np.float32)
    pix, c2, s2 = expand(bore, 1, det, 3, 4, 3)
    # sample 0: x = -0.5 (outside); 1: inside, pixel (1, 0); 2: orientation (0, 0) -> flagged
    assert list(pix) == [-1, 1 * 4 + 0, -1]
    assert c2[1] == 1.0 and s2[1] == 0.0
    pix_t, c_t, _ = expand(bore, 1, det, 3, 4, 3, polarised=False)
    assert c_t is None and list(pix_t) == [-1, 4, 1 * 4 + 3]


def test_gcp_system_matches_angle_system():
    """The oracle System fed the expansion's weights equals the System fed the angles they
    come from (the weights argument is the same A), up to the float32 weights' length
    (c^2 + s^2 = 1 within a few 1e-7)."""
    from oracle.gcp import expand
    from synth.boresight import make_boresight_problem
    from tests.helpers import lags_for
    from oracle.solver import System
    p = make_boresight_problem("gcp", 21, 8, 2, 700, 8, 3, 10, noise=(1.0, 3.0, 1.5),
                               interval_lengths=lambda rng, n: [300, 400])
    pix, c2, s2 = expand(p.boresight, p.bore_step, p.det, p.samples_per_det, p.width, p.height)
    lags = lags_for(p)
    S1 = System(pix, None, p.n_pix, 3, p.interval_offsets, p.interval_filter, lags, weights=(c2, s2))
    psi = 0.5 * np.arctan2(s2.astype(np.float64), c2.astype(np.float64))
    S2 = System(pix, psi, p.n_pix, 3, p.interval_offsets, p.interval_filter, lags)
    x = np.random.default_rng(0).standard_normal((S1.n_obs, 3))
    assert rel_rms(S1.H(x), S2.H(x)) < 1e-6
    assert S1.n_obs > 40 and not S1.excised.all()


# ------------------------------------------------------------------ extended pointing (Section 6)
def _ext_system(p, idx, n_extra, lags=None, **kw):
    from oracle.extended import ExtendedSystem
    return ExtendedSystem(p.pix, p.psi, p.n_pix, p.n_stokes, p.interval_offsets, p.interval_filter,
                          lags_for(p) if lags is None else lags, idx, n_extra, **kw)


def test_extended_without_extra_columns_is_the_plain_system():
    p = tiny_IQU(seed=51, n_per_det=400)
    S = system_for(p)
    E = _ext_system(p, np.full(p.n_samples, -1, np.int32), 3)
    x = np.random.default_rng(0).standard_normal((E.n_obs, 3))
    x[E.n_sky:] = 0.0
    assert np.allclose(E.H(x)[:E.n_sky], S.H(x[:E.n_sky]), rtol=1e-12, atol=1e-12)
    assert np.all(E.H(x)[E.n_sky:] == 0.0) and E.excised_extra.all()
    xe, _ = E.solve(p.d[0], rel_tol=1e-13, max_iter=400)
    xs, _ = S.solve(p.d[0], rel_tol=1e-13, max_iter=400)
    assert rel_rms(xe[:E.n_sky], xs) < 1e-10 and np.all(xe[E.n_sky:] == 0.0)


def test_extended_pcg_matches_dense_cholesky_and_is_symmetric():
    from synth.extended import baseline_index
    p = tiny_IQU(seed=52, n_per_det=300, n_lags=6)
    idx, n_extra = baseline_index(300, 4, 64)
    E = _ext_system(p, idx, n_extra)
    xd = E.dense_solve(p.d[0])
    xp, info = E.solve(p.d[0], rel_tol=1e-13, max_iter=2000)
    act = E.active()
    assert info["best_res"] < 1e-12
    assert rel_rms(xp[act], xd[act]) < 1e-9 and np.all(xp[~act] == 0.0)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal((2, E.n_obs, 3)) * act
    a, b = float(np.sum(y * E.H(x))), float(np.sum(x * E.H(y)))
    assert abs(a - b) <= 1e-12 * abs(a) and float(np.sum(x * E.H(x))) > 0


def test_extended_destriping_recovers_sky_and_offsets():
    """White noise (one lag, no FFT involved) and noiseless data d = A z + B o: the
    solution is the sky and the offsets (the reference baseline fixes the level)."""
    from synth.extended import add_extra_signal, baseline_index
    p = tiny_T(seed=53, n=1200, width=6, ivls=(500, 700), noiseless=True)
    idx, n_extra = baseline_index(1200, 1, 50)
    o = np.random.default_rng(2).normal(0.0, 3.0, n_extra)
    d = add_extra_signal(p.d[0], idx, o)
    white = np.array([[1.0]])
    E = _ext_system(p, idx, n_extra, lags=white, ninv="direct")
    x, info = E.solve(d, rel_tol=1e-14, max_iter=3000)
    z, oo, _ = E.split(x)
    keep = ~E.excised_sky
    assert rel_rms(z[keep, 0], p.sky[E.obs2glob[keep], 0]) < 1e-6       # d is float32
    assert rel_rms(oo, o) < 1e-6


def test_extended_binned_template_recovery():
    """A chopper-synchronous signal binned in angle (item 1 of Section 6) on top of an IQU
    sky, noiseless: both are recovered."""
    from synth.extended import add_extra_signal, chop_bins
    p = tiny_IQU(seed=54, n_per_det=1500, width=5, noiseless=True)
    idx, n_extra = chop_bins(p.n_samples, 9, 37.0, np.random.default_rng(3))
    amp = np.random.default_rng(4).normal(0.0, 2.0, n_extra)
    d = add_extra_signal(p.d[0], idx, amp)
    E = _ext_system(p, idx, n_extra)
    x, _ = E.solve(d, rel_tol=1e-14, max_iter=3000)
    z, oo, _ = E.split(x)
    keep = ~E.excised_sky
    for s in range(3):
        assert rel_rms(z[keep, s], p.sky[E.obs2glob[keep], s]) < 1e-5
    assert rel_rms(oo, amp) < 1e-5


def _hwp_case(seed, noiseless=True, n_per=1500):
    from synth.extended import add_hwp_signal, hwp_inputs
    p = tiny_IQU(seed=seed, n_per_det=n_per, width=5, noiseless=noiseless, n_ivl_lo=500, n_ivl_hi=1500)
    ang, tau, grp, n_groups = hwp_inputs(p.interval_offsets, p.fs, 1.3, np.random.default_rng(seed))
    b = np.random.default_rng(seed + 1).normal(0.0, 0.3, (n_groups, 32))
    d = add_hwp_signal(p.d[0], p.interval_offsets, ang, tau, grp, b)
    return p, (ang, tau, grp, n_groups), b, d


def test_extended_hwp_noiseless_recovery():
    """An injected half-wave-plate signal (Eqs. 41-42, synthesised as the real part of a
    complex-exponential sum) and an IQU sky, noiseless: both are recovered."""
    p, hwp, b, d = _hwp_case(61)
    E = _ext_system(p, np.full(p.n_samples, -1, np.int32), 1, hwp=hwp)
    x, info = E.solve(d, rel_tol=1e-14, max_iter=5000)
    z, _, bb = E.split(x)
    keep = ~E.excised_sky
    for s in range(3):
        assert rel_rms(z[keep, s], p.sky[E.obs2glob[keep], s]) < 1e-5
    assert rel_rms(bb, b) < 1e-5


def test_extended_hwp_dense_cholesky_symmetry_and_reduction():
    from synth.extended import baseline_index
    p, hwp, b, d = _hwp_case(62, noiseless=False, n_per=400)
    idx, n_extra = baseline_index(400, 4, 100)
    E = _ext_system(p, idx, n_extra, hwp=hwp)
    xd = E.dense_solve(d)
    xp, info = E.solve(d, rel_tol=1e-13, max_iter=5000)
    act = E.active()
    assert info["best_res"] < 1e-12 and rel_rms(xp[act], xd[act]) < 1e-8
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((2, E.n_obs, 3)) * act
    a, c = float(np.sum(y * E.H(x))), float(np.sum(x * E.H(y)))
    assert abs(a - c) <= 1e-12 * abs(a)
    # every group switched off: the system without the half-wave-plate block
    ang, tau, grp, ng = hwp
    E0 = _ext_system(p, idx, n_extra, hwp=(ang, tau, np.full_like(grp, -1), ng))
    E1 = _ext_system(p, idx, n_extra)
    x1 = rng.standard_normal((E1.n_obs, 3)) * E1.active()
    x0 = np.zeros((E0.n_obs, 3))
    x0[:E1.n_obs] = x1
    assert np.allclose(E0.H(x0)[:E1.n_obs], E1.H(x1), rtol=1e-12, atol=1e-12) and E0.excised_hwp.all()


def test_gcp_expansion_does_not_depend_on_the_chunking():
    """The expansion walks the samples in chunks; any chunk size gives the same pointing."""
    from oracle.gcp import expand, nodes_needed
    from synth.boresight import make_boresight_problem
    p = make_boresight_problem("ch", 22, 16, 3, 2000, 8, 3, 6, noise=(1.0, 2.0, 1.5), rot_period=1500)
    assert p.boresight.shape[0] == nodes_needed(p.samples_per_det, p.bore_step)
    a = expand(p.boresight, p.bore_step, p.det, p.samples_per_det, p.width, p.height)
    b = expand(p.boresight, p.bore_step, p.det, p.samples_per_det, p.width, p.height, chunk=37)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
