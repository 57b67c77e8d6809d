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
                 rcond_excise=1e-6, rcond_fp64=1e-2, ninv="fft", n_f=None, weights=None):
        """weights (IQU, optional): (cos 2psi, sin 2psi) per sample given directly, e.g. by
        the expansion of compressed pointing (oracle.gcp); psi is then unused."""
        self.n_s = int(n_stokes)
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.ivl_filter = np.asarray(ivl_filter, dtype=np.int64)
        self.lags = np.atleast_2d(np.asarray(lags, dtype=np.float64))
        self.n_c = self.lags.shape[1]
        self.obs2glob, self.glob2obs = _pt.observed_pixels(np.asarray(pix), int(n_pix))
        self.n_obs = int(self.obs2glob.size)
        pixl = _pt.local_pixels(np.asarray(pix), self.glob2obs)
        if weights is not None and self.n_s == 3:
            c2, s2 = (np.asarray(v, dtype=np.float64) for v in weights)
            self.w = np.stack([np.ones_like(c2), c2, s2], axis=1)
        else:
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
        hits, AtA, AtWA = pixel_blocks(pixl, self.w, f0, self.n_obs, self.n_s)
        c = classify_blocks(hits, AtA, AtWA, rcond_excise, rcond_fp64)
        self.hits, self.blocks, self.rcond = hits, AtWA, c["rcond"]
        self.excised, self.fp64, self.Pinv = c["excised"], c["fp64"], c["Pinv"]

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

        Used to check full-size operator outputs one by one (see sampled_rows).
        """
        x = np.asarray(x, dtype=np.float64).reshape(self.n_obs, self.n_s)

        def ax(lo, hi):
            return _pt.unpoint(x, self.pixl[lo:hi], None if self.w is None else self.w[lo:hi])

        hits = [np.flatnonzero(self.pixl == p) for p in pixels]
        return sampled_rows(hits, ax, lambda ts: None if self.w is None else self.w[ts],
                            self.offsets, self.ivl_filter, self.lags, self.n_s)

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


def pixel_blocks(pixl, w, f0, n_obs, n_s, out=None):
    """Per pixel: hits, A^T A and A^T W^-1 A blocks [n_obs, n_s, n_s] (W^-1 = diag of N^-1).

    pixl: pixel of each sample (-1 = no row); w: row weights or None (T);
    f0: f(0) of each sample's filter.  With ``out`` = (hits, AtA, AtWA) the
    sums are added to it (chunked accumulation).
    """
    if out is None:
        out = (np.zeros(n_obs, dtype=np.int64), np.zeros((n_obs, n_s, n_s)), np.zeros((n_obs, n_s, n_s)))
    hits, AtA, AtWA = out
    ok = pixl >= 0
    p = pixl[ok]
    h = np.bincount(p, minlength=n_obs)
    hits += h
    f = f0[ok]
    if w is None:
        AtA[:, 0, 0] += h
        AtWA[:, 0, 0] += np.bincount(p, weights=f, minlength=n_obs)
        return out
    wk = w[ok]
    for a in range(n_s):
        for b in range(a, n_s):
            ww = wk[:, a] * wk[:, b]
            v = np.bincount(p, weights=ww, minlength=n_obs)
            vw = np.bincount(p, weights=f * ww, minlength=n_obs)
            AtA[:, a, b] += v
            AtWA[:, a, b] += vw
            if b != a:
                AtA[:, b, a] += v
                AtWA[:, b, a] += vw
    return out


def classify_blocks(hits, AtA, AtWA, rcond_excise, rcond_fp64):
    """Excision, float64 flags and block inverses of the preconditioner (Section 4, Section 5).

    T: a pixel is excised when unobserved; its preconditioner is 1 / (A^T W^-1 A).
    IQU: excised when hits < 3 or rcond(A^T A) = lambda_min / lambda_max < rcond_excise;
    flagged float64 when kept with rcond < rcond_fp64; preconditioner (A^T W^-1 A)^-1.
    """
    n_obs, n_s = AtA.shape[0], AtA.shape[1]
    if n_s == 1:
        wsum = AtWA[:, 0, 0]
        excised = hits == 0
        with np.errstate(divide="ignore"):
            Pinv = np.where(excised, 0.0, 1.0 / wsum).reshape(n_obs, 1, 1)
        return dict(excised=excised, fp64=np.zeros(n_obs, dtype=bool), rcond=np.ones(n_obs), Pinv=Pinv)
    ev = np.linalg.eigvalsh(AtA)                    # ascending
    with np.errstate(divide="ignore", invalid="ignore"):
        rc = np.where(ev[:, 2] > 0, ev[:, 0] / ev[:, 2], 0.0)
    excised = (hits < 3) | (rc < rcond_excise)
    fp64 = (~excised) & (rc < rcond_fp64)
    Pinv = np.zeros_like(AtWA)
    good = ~excised
    Pinv[good] = np.linalg.inv(AtWA[good])
    return dict(excised=excised, fp64=fp64, rcond=rc, Pinv=Pinv)


def sampled_rows(hits, values, w_at, offsets, ivl_filter, lags, n_s):
    """(A^T N^-1 y)_p for a few pixels, each from Eq. 15 on its own.

    hits[k]: the samples t of pixel k (rows of A that are not zero);
    values(lo, hi): y on samples lo .. hi-1; w_at(ts): the row weights of
    samples ts (None for T).  For every t: (N^-1 y)_t = sum over |tau| < n_c
    inside t's interval of f(|tau|) y_{t+tau}; then weight and sum into p.
    """
    n_c = lags.shape[1]
    out = np.zeros((len(hits), n_s))
    for k, ts in enumerate(hits):
        ts = np.asarray(ts, dtype=np.int64)
        wt = w_at(ts)
        for m, t in enumerate(ts):
            i = int(np.searchsorted(offsets, t, side="right") - 1)
            a, b = int(offsets[i]), int(offsets[i + 1])
            lo, hi = max(a, t - n_c + 1), min(b, t + n_c)
            f = lags[ivl_filter[i]][np.abs(np.arange(lo, hi) - t)]
            v = float(f @ np.asarray(values(lo, hi), dtype=np.float64))
            if wt is None:
                out[k, 0] += v
            else:
                out[k] += v * wt[m]
    return out


class StreamedSystem:
    """Sampled rows of H and b for pointing too large for System (same definitions).

    Keeps the caller's int32 pixels and float32 angles by reference and walks
    them in chunks: the observed-pixel bit array (Section 5.4), the per-pixel
    blocks and their classification (Section 4) are accumulated chunk by chunk,
    and rows of H x or b (Eq. 10) are evaluated one pixel at a time from Eq. 15.
    Nothing of size n_t is held in float64.
    """

    def __init__(self, pix, psi, n_pix, n_stokes, offsets, ivl_filter, lags,
                 rcond_excise=1e-6, rcond_fp64=1e-2, chunk=1 << 22):
        self.pix, self.psi = pix, psi
        self.n_s = int(n_stokes)
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.ivl_filter = np.asarray(ivl_filter, dtype=np.int64)
        self.lags = np.atleast_2d(np.asarray(lags, dtype=np.float64))
        self.n_c = self.lags.shape[1]
        self.chunk = int(chunk)
        n_t = int(pix.shape[0])
        self.n_t = n_t
        self.obs2glob, self.glob2obs = _pt.observed_pixels(pix, int(n_pix), chunk=self.chunk)
        self.n_obs = int(self.obs2glob.size)
        acc = None
        for lo in range(0, n_t, self.chunk):
            hi = min(n_t, lo + self.chunk)
            pl, w, f0 = self._rows(lo, hi, excise=False)
            acc = pixel_blocks(pl, w, f0, self.n_obs, self.n_s, out=acc)
        if acc is None:
            acc = pixel_blocks(np.zeros(0, np.int64), None if self.n_s == 1 else np.zeros((0, 3)),
                               np.zeros(0), self.n_obs, self.n_s)
        self.hits = acc[0]
        c = classify_blocks(*acc, rcond_excise, rcond_fp64)
        self.excised, self.fp64, self.rcond, self.Pinv = c["excised"], c["fp64"], c["rcond"], c["Pinv"]

    def _rows(self, lo, hi, excise=True):
        """Observed pixel (excised -> -1 when ``excise``), weights and f(0) of samples lo .. hi-1."""
        pl = _pt.local_pixels(np.asarray(self.pix[lo:hi]), self.glob2obs)
        if excise:
            ok = pl >= 0
            pl[ok & self.excised[np.where(ok, pl, 0)]] = -1
        w = _pt.weights(None if self.psi is None else self.psi[lo:hi], self.n_s)
        i0 = int(np.searchsorted(self.offsets, lo, side="right") - 1)
        i1 = int(np.searchsorted(self.offsets, hi - 1, side="right") - 1)
        f0 = np.empty(hi - lo)
        for i in range(i0, i1 + 1):
            a, b = max(lo, int(self.offsets[i])), min(hi, int(self.offsets[i + 1]))
            f0[a - lo:b - lo] = self.lags[self.ivl_filter[i], 0]
        return pl, w, f0

    def hits_of(self, pixels):
        """Samples of each observed pixel in ``pixels`` (empty for excised pixels)."""
        sel = np.full(self.n_obs, -1, dtype=np.int64)
        sel[np.asarray(pixels, dtype=np.int64)] = np.arange(len(pixels))
        found = [[] for _ in pixels]
        for lo in range(0, self.n_t, self.chunk):
            hi = min(self.n_t, lo + self.chunk)
            pl = _pt.local_pixels(np.asarray(self.pix[lo:hi]), self.glob2obs)
            k = np.where(pl >= 0, sel[np.where(pl >= 0, pl, 0)], -1)
            for t in np.flatnonzero(k >= 0):
                found[k[t]].append(lo + t)
        return [np.asarray(f if not self.excised[p] else [], dtype=np.int64) for f, p in zip(found, pixels)]

    def _w_at(self, ts):
        return None if self.n_s == 1 else _pt.weights(np.asarray(self.psi)[ts], self.n_s)

    def H_sampled(self, x, pixels, hits=None):
        """(H x)_p for observed pixels p (x over the observed pixels, [n_obs, n_s])."""
        x = np.asarray(x, dtype=np.float64).reshape(self.n_obs, self.n_s)
        hits = self.hits_of(pixels) if hits is None else hits

        def ax(lo, hi):
            pl, w, _ = self._rows(lo, hi)
            return _pt.unpoint(x, pl, w)

        return sampled_rows(hits, ax, self._w_at, self.offsets, self.ivl_filter, self.lags, self.n_s)

    def rhs_sampled(self, d, pixels, hits=None):
        """b_p = (A^T N^-1 d)_p for observed pixels p."""
        hits = self.hits_of(pixels) if hits is None else hits
        return sampled_rows(hits, lambda lo, hi: d[lo:hi], self._w_at, self.offsets, self.ivl_filter,
                            self.lags, self.n_s)


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
