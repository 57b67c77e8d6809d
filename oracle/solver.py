"""The map-making system and its PCG solve (oracle, FP64).  Test infrastructure only.

Section 4, Eq. 10: H x = b with H = A^T N^-1 A and b = A^T N^-1 d; its
solution is the maximum-likelihood map of Section 3, Eq. 8.

Preconditioner (Section 5): MADpre's block form (A^T W^-1 A)^-1 with W^-1 the
diagonal of N^-1, so each sample weighs in with f(0) of its interval's
filter.  For IQU the blocks are the per-pixel 3 x 3 matrices; for T the
1 x 1 case, which differs from point Jacobi 1/hits only by the uniform
factor f(0) when there is one filter (PCG iterates are unchanged by a uniform
scale of the preconditioner).

Poorly constrained pixels (Section 4): the 3 x 3 block of A^T A of each IQU
pixel is examined; with hits < 3 or rcond = lambda_min / lambda_max below
``rcond_excise`` the pixel is excised, its samples' rows of A are set to zero
as after gap filling, and its map value is 0.  Pixels with rcond below
``rcond_fp64`` are only flagged (the GPU library keeps their block inverse in
float64).  The paper gives no thresholds; 1e-6 and 1e-2 are the defaults here.

PCG (Section 4; Section 5 termination): x_0 = 0; the standard preconditioned
conjugate-gradient recurrences; stop when the relative residual
||r_k|| / ||b|| (r_k the recursively updated residual) is at most the
tolerance, or after ``max_iter`` iterations; return the iterate with the
lowest relative residual seen so far (ties to the earlier one).

Dense path (Section 3 and 4, brute force for tiny inputs): A and N^-1 written
out as matrices, H formed explicitly and solved by Cholesky.
"""

from __future__ import annotations

import numpy as np

from . import noise as _noise
from . import pointing as _pt


class System:
    """A^T N^-1 A over the observed pixels of one pointing, in float64.

    Parameters mirror the library's plan: global pixel per sample (-1 =
    flagged), float32 angles (IQU only), interval offsets, the filter of each
    interval and the filter lags [n_filters, n_c].  ``ninv`` selects the FFT
    product of Section 5.2 ("fft", default, n_f from the paper's rule unless
    given) or the direct sum of Eq. 15 ("direct").
    """

    def __init__(self, pix, psi, n_pix, n_stokes, offsets, ivl_filter, lags,
                 rcond_excise=1e-6, rcond_fp64=1e-2, ninv="fft", n_f=None):
        self.n_s = int(n_stokes)
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.ivl_filter = np.asarray(ivl_filter, dtype=np.int64)
        self.lags = np.atleast_2d(np.asarray(lags, dtype=np.float64))
        self.n_c = self.lags.shape[1]
        self.obs2glob, self.glob2obs = _pt.observed_pixels(np.asarray(pix), int(n_pix))
        self.n_obs = int(self.obs2glob.size)
        pixl = _pt.local_pixels(np.asarray(pix), self.glob2obs)
        self.w = _pt.weights(psi, self.n_s)
        lengths = np.diff(self.offsets)
        f0 = np.repeat(self.lags[self.ivl_filter, 0], lengths)     # diag of N^-1 per sample
        self._classify(pixl, f0, rcond_excise, rcond_fp64)
        pixl = pixl.copy()
        keep = pixl >= 0
        pixl[keep & self.excised[np.where(keep, pixl, 0)]] = -1     # zero rows of excised pixels
        self.pixl = pixl
        if ninv == "direct":
            self.n_f = None
        else:
            longest = int(lengths.max()) if lengths.size else 1
            self.n_f = int(n_f) if n_f else _noise.fft_length(self.n_c, longest)
        self.ninv_mode = ninv

    # ---------------------------------------------------------------- set-up
    def _classify(self, pixl, f0, rcond_excise, rcond_fp64):
        n_obs, n_s = self.n_obs, self.n_s
        ok = pixl >= 0
        p = pixl[ok]
        self.hits = np.bincount(p, minlength=n_obs)
        if n_s == 1:
            wsum = np.bincount(p, weights=f0[ok], minlength=n_obs)
            self.blocks = wsum.reshape(n_obs, 1, 1)
            self.excised = self.hits == 0
            self.fp64 = np.zeros(n_obs, dtype=bool)
            self.rcond = np.ones(n_obs)
            with np.errstate(divide="ignore"):
                self.Pinv = np.where(self.excised, 0.0, 1.0 / wsum).reshape(n_obs, 1, 1)
            return
        w = self.w[ok]
        AtA = np.zeros((n_obs, 3, 3))
        AtWA = np.zeros((n_obs, 3, 3))
        for a in range(3):
            for b in range(3):
                AtA[:, a, b] = np.bincount(p, weights=w[:, a] * w[:, b], minlength=n_obs)
                AtWA[:, a, b] = np.bincount(p, weights=f0[ok] * w[:, a] * w[:, b], minlength=n_obs)
        ev = np.linalg.eigvalsh(AtA)                    # ascending
        with np.errstate(divide="ignore", invalid="ignore"):
            rc = np.where(ev[:, 2] > 0, ev[:, 0] / ev[:, 2], 0.0)
        self.rcond = rc
        self.excised = (self.hits < 3) | (rc < rcond_excise)
        self.fp64 = (~self.excised) & (rc < rcond_fp64)
        self.blocks = AtWA
        Pinv = np.zeros_like(AtWA)
        good = ~self.excised
        Pinv[good] = np.linalg.inv(AtWA[good])
        self.Pinv = Pinv

    # ---------------------------------------------------------------- operators
    def unpoint(self, x):
        return _pt.unpoint(np.asarray(x, dtype=np.float64).reshape(self.n_obs, self.n_s), self.pixl, self.w)

    def point(self, y):
        return _pt.point(y, self.pixl, self.w, self.n_obs, self.n_s)

    def ninv(self, y):
        if self.ninv_mode == "direct":
            return _noise.apply_ninv_direct(y, self.offsets, self.ivl_filter, self.lags)
        return _noise.apply_ninv_fft(y, self.offsets, self.ivl_filter, self.lags, self.n_f)

    def H(self, x):
        """H x = A^T N^-1 A x (Eq. 10)."""
        return self.point(self.ninv(self.unpoint(x)))

    def rhs(self, d):
        """b = A^T N^-1 d (Eq. 10)."""
        return self.point(self.ninv(np.asarray(d, dtype=np.float64)))

    def H_sampled(self, x, pixels):
        """(H x)_p for a few observed pixels p, each computed on its own from Eq. 15.

        For every sample t of pixel p: (N^-1 A x)_t = sum over |tau| < n_c inside
        t's interval of f(|tau|) (A x)_{t+tau}; then weight and sum into p.  Used
        to check full-size operator outputs one by one.
        """
        x = np.asarray(x, dtype=np.float64).reshape(self.n_obs, self.n_s)
        out = np.zeros((len(pixels), self.n_s))
        for k, p in enumerate(pixels):
            ts = np.flatnonzero(self.pixl == p)
            for t in ts:
                i = int(np.searchsorted(self.offsets, t, side="right") - 1)
                a, b = int(self.offsets[i]), int(self.offsets[i + 1])
                lo, hi = max(a, t - self.n_c + 1), min(b, t + self.n_c)
                sl = slice(lo, hi)
                pl = self.pixl[sl]
                ok = pl >= 0
                w = None if self.w is None else self.w[sl]
                ax = _pt.unpoint(x, pl, w)
                f = self.lags[self.ivl_filter[i]][np.abs(np.arange(lo, hi) - t)]
                v = float(np.sum(f[ok] * ax[ok]))
                if self.w is None:
                    out[k, 0] += v
                else:
                    out[k] += v * self.w[t]
        return out

    def precond(self, r):
        return np.einsum("pab,pb->pa", self.Pinv, r)

    # ---------------------------------------------------------------- solve
    def pcg(self, b, rel_tol=1e-6, max_iter=50, keep_history=False):
        """Preconditioned CG with x_0 = 0 and the lowest-residual output rule."""
        b = np.asarray(b, dtype=np.float64).reshape(self.n_obs, self.n_s)
        return pcg(self.H, self.precond, b, rel_tol, max_iter, keep_history)

    def solve(self, d, rel_tol=1e-6, max_iter=50, keep_history=False):
        return self.pcg(self.rhs(d), rel_tol, max_iter, keep_history)

    # ---------------------------------------------------------------- dense
    def dense_H(self):
        A = _pt.dense_pointing(self.pixl, self.w, self.n_obs, self.n_s)
        N = _noise.dense_ninv(self.offsets, self.ivl_filter, self.lags)
        return A, N, A.T @ N @ A

    def dense_solve(self, d):
        """Brute-force ML map (Eq. 8): explicit H, Cholesky, excised unknowns removed."""
        A, N, H = self.dense_H()
        b = A.T @ N @ np.asarray(d, dtype=np.float64)
        keep = np.repeat(~self.excised, self.n_s)
        x = np.zeros(self.n_obs * self.n_s)
        Hk = H[np.ix_(keep, keep)]
        L = np.linalg.cholesky(Hk)
        x[keep] = np.linalg.solve(L.T, np.linalg.solve(L, b[keep]))
        return x.reshape(self.n_obs, self.n_s)


def pcg(apply_H, apply_P, b, rel_tol, max_iter, keep_history=False):
    """Standard PCG on H x = b (x_0 = 0), returning the lowest-residual iterate.

    Returns (x_best, info) with info = dict(iters, best_iter, best_res,
    final_res, history [, iterates]).
    """
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = float(np.sqrt(np.sum(b * b)))
    info = dict(iters=0, best_iter=0, best_res=0.0 if bnorm == 0 else 1.0, final_res=0.0, history=[])
    if bnorm == 0.0:
        return x, info
    z = apply_P(r)
    p = z.copy()
    rz = float(np.sum(r * z))
    res = float(np.sqrt(np.sum(r * r))) / bnorm
    hist = [res]
    its = [x.copy()] if keep_history else None
    best_x, best_res, best_k = x.copy(), res, 0
    k = 0
    while res > rel_tol and k < max_iter:
        q = apply_H(p)
        alpha = rz / float(np.sum(p * q))
        x = x + alpha * p
        r = r - alpha * q
        k += 1
        res = float(np.sqrt(np.sum(r * r))) / bnorm
        hist.append(res)
        if keep_history:
            its.append(x.copy())
        if res < best_res:
            best_x, best_res, best_k = x.copy(), res, k
        if res <= rel_tol:
            break
        z = apply_P(r)
        rz_new = float(np.sum(r * z))
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    info = dict(iters=k, best_iter=best_k, best_res=best_res, final_res=res, history=hist)
    if keep_history:
        info["iterates"] = its
    return best_x, info
