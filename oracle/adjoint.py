"""Gradients of a map loss through the solve (oracle, FP64).  Test infrastructure only.

The map m = H^-1 b with H = A^T N^-1 A and b = A^T N^-1 d (Section 4, Eq. 10).
The paper does not differentiate the solve; this is the implicit adjoint
written out.  Perturbing N^-1 and d:

    dm = H^-1 (A^T N^-1 dd + A^T dN^-1 (d - A m)),

so for a loss L(m) with g = dL/dm and the adjoint map lambda = H^-1 g (H is
self-adjoint, so one more solve with the same operator):

    dL/dd      = N^-1 A lambda
    dL/dN^-1   = (A lambda) (d - A m)^T   (restricted to the band of N^-1)

N^-1 is banded block Toeplitz (Section 5.2, Eq. 15), each lag f_k(tau) of
filter k appearing at every pair (t, t') of an interval using k with
|t - t'| = tau.  Hence

    dL/df_k(tau) = sum over intervals using k of
                   sum_{t, t' in interval, |t - t'| = tau} a_t r_t'
    with a = A lambda and r = d - A m (both orders of the pair for tau > 0).

Parameters (sigma, f_knee, alpha) of each filter follow by the chain rule
through the filter builder (oracle.noise.filter_lags with_grad).

Parity pinned by tests/test_oracle_pins.py::test_adjoint_* (central finite
differences through float64 solves in d, in the lags and in the PSD
parameters; exact linearity in d; invariance of the map under a common scale
of every sigma).
"""

from __future__ import annotations

import numpy as np

from . import noise as _noise


def lag_correlation(a, r, offsets, ivl_filter, n_filters, n_lags):
    """sum_{|t-t'|=tau, same interval} a_t r_t' per filter and lag, by direct sums."""
    out = np.zeros((n_filters, n_lags))
    for i in range(len(ivl_filter)):
        lo, hi = int(offsets[i]), int(offsets[i + 1])
        aa = np.asarray(a[lo:hi], dtype=np.float64)
        rr = np.asarray(r[lo:hi], dtype=np.float64)
        k = int(ivl_filter[i])
        out[k, 0] += float(aa @ rr)
        for tau in range(1, min(n_lags, hi - lo)):
            out[k, tau] += float(aa[:-tau] @ rr[tau:]) + float(aa[tau:] @ rr[:-tau])
    return out


def solve_backward(S, d, m, g, rel_tol=1e-13, max_iter=2000):
    """(dL/dd, dL/df [n_filters, n_lags], info) for the map m of data d and g = dL/dm.

    S is an oracle.solver.System (or a multires.MultiResSystem); m and g are
    [n_obs, n_s] over its observed pixels (slots).  g is zeroed at unknowns
    that do not exist (excised pixels): H has no row there.
    """
    g = np.asarray(g, dtype=np.float64).reshape(S.n_obs, S.n_s).copy()
    if hasattr(S, "active"):
        g[~S.active()] = 0.0
    else:
        g[S.excised] = 0.0
    lam, info = S.pcg(g, rel_tol=rel_tol, max_iter=max_iter)
    a = S.unpoint(lam)
    grad_d = S.ninv(a)
    r = np.asarray(d, dtype=np.float64) - S.unpoint(m)
    grad_f = lag_correlation(a, r, S.offsets, S.ivl_filter, S.lags.shape[0], S.n_c)
    return grad_d, grad_f, info


def params_gradient(grad_f, n_lags, fs, params):
    """Chain rule from lag gradients [n_filters, n_lags] to (sigma, f_knee, alpha) per filter."""
    out = np.zeros((len(params), 3))
    for k, (s, fk, al) in enumerate(params):
        _, dl = _noise.filter_lags(n_lags, fs, s, fk, al, with_grad=True)
        out[k] = dl @ grad_f[k]
    return out
