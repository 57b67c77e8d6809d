"""Multi-resolution Stokes maps (oracle, FP64).  Test infrastructure only.

Section 6 (item 4): MADmap makes no assumption about the pixelisation, so the
Stokes parameters may live on different pixels; the intensity is typically
pixelised more finely than Q and U.  Each sample t then has an I pixel p_t
and a polarisation pixel q_t, and its row of A is

    y_t = i[p_t] + cos 2psi_t q[q_t] + sin 2psi_t u[q_t]

(the weights of Section 3, Eqs. 2-4, with the relabelling used throughout the
library).  H = A^T N^-1 A and b = A^T N^-1 d as in Eq. 10.

Layout ("slots"): vectors are [n_slots, 3] with n_slots = max(observed I
pixels, observed QU pixels); slot k holds I of observed I pixel k and Q, U of
observed QU pixel k, so I and QU of one slot are unrelated.  Entries past
either count are unused (always 0).

Readings where the paper is silent:
* Preconditioner (Section 5, MADpre): the block diagonal of A^T W^-1 A with
  the pixelisation's own blocks: 1 x 1 for each I pixel, 2 x 2 (Q, U) for each
  polarisation pixel; the I-QU couplings, which join different pixels, are
  dropped.
* Poorly constrained pixels (Section 4): a polarisation pixel is excised when
  it has fewer than 2 hits or rcond of its 2 x 2 block of A^T A is below the
  threshold; the rows of its samples are then zero (gap filling), and an I
  pixel left without rows is excised too.  Samples flagged in either
  pixelisation (-1) have zero rows.

Pinned by tests/test_oracle_pins.py::test_multires_* (the reduction to the
single-resolution system when q = p, dense Cholesky, noiseless recovery of a
sky that is constant within polarisation pixels, symmetry).
"""

from __future__ import annotations

import numpy as np

from . import noise as _noise
from . import pointing as _pt
from .solver import pcg as _pcg


class MultiResSystem:
    def __init__(self, pix, pix_pol, psi, n_pix, n_pix_pol, offsets, ivl_filter, lags,
                 rcond_excise=1e-6, rcond_fp64=1e-2, ninv="fft", n_f=None):
        pix = np.asarray(pix)
        pix_pol = np.asarray(pix_pol)
        self.n_s = 3
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.ivl_filter = np.asarray(ivl_filter, dtype=np.int64)
        self.lags = np.atleast_2d(np.asarray(lags, dtype=np.float64))
        self.n_c = self.lags.shape[1]
        both = (pix >= 0) & (pix_pol >= 0)
        self.obs2glob, self.glob2obs = _pt.observed_pixels(np.where(both, pix, -1), int(n_pix))
        self.obs2glob_pol, self.glob2obs_pol = _pt.observed_pixels(np.where(both, pix_pol, -1), int(n_pix_pol))
        self.n_obs_i, self.n_obs_pol = int(self.obs2glob.size), int(self.obs2glob_pol.size)
        self.n_obs = max(self.n_obs_i, self.n_obs_pol)
        pi = _pt.local_pixels(np.where(both, pix, -1), self.glob2obs)
        pq = _pt.local_pixels(np.where(both, pix_pol, -1), self.glob2obs_pol)
        two = 2.0 * np.asarray(psi, dtype=np.float64)
        self.c, self.s = np.cos(two), np.sin(two)
        lengths = np.diff(self.offsets)
        f0 = np.repeat(self.lags[self.ivl_filter, 0], lengths)
        n = self.n_obs
        # polarisation blocks and their classification
        ok = pq >= 0
        q = pq[ok]
        cc, cs, ss, w = self.c[ok] ** 2, self.c[ok] * self.s[ok], self.s[ok] ** 2, f0[ok]
        hits_pol = np.bincount(q, minlength=n)
        AtA = np.zeros((n, 2, 2))
        AtWA = np.zeros((n, 2, 2))
        for (a, b), v in (((0, 0), cc), ((0, 1), cs), ((1, 1), ss)):
            AtA[:, a, b] = np.bincount(q, weights=v, minlength=n)
            AtWA[:, a, b] = np.bincount(q, weights=w * v, minlength=n)
        AtA[:, 1, 0], AtWA[:, 1, 0] = AtA[:, 0, 1], AtWA[:, 0, 1]
        ev = np.linalg.eigvalsh(AtA)
        with np.errstate(divide="ignore", invalid="ignore"):
            rc = np.where(ev[:, 1] > 0, ev[:, 0] / ev[:, 1], 0.0)
        ex_pol = (hits_pol < 2) | (rc < rcond_excise)
        ex_pol[self.n_obs_pol:] = True
        self.rcond_pol = rc
        self.fp64 = (~ex_pol) & (rc < rcond_fp64)
        # gap filling: rows of excised polarisation pixels are zero
        drop = (pq < 0) | ex_pol[np.where(pq >= 0, pq, 0)]
        pi = np.where(drop, -1, pi)
        pq = np.where(drop, -1, pq)
        self.pi, self.pq = pi, pq
        # intensity blocks from the remaining rows
        oki = pi >= 0
        hits_i = np.bincount(pi[oki], minlength=n)
        aI = np.bincount(pi[oki], weights=f0[oki], minlength=n)
        ex_i = hits_i == 0
        ex_i[self.n_obs_i:] = True
        self.excised, self.excised_pol = ex_i, ex_pol
        self.hits, self.hits_pol = hits_i, hits_pol
        Pinv = np.zeros((n, 3, 3))
        with np.errstate(divide="ignore"):
            Pinv[:, 0, 0] = np.where(ex_i, 0.0, 1.0 / np.where(ex_i, 1.0, aI))
        good = ~ex_pol
        Pinv[good, 1:, 1:] = np.linalg.inv(AtWA[good])
        self.Pinv = Pinv
        if ninv == "direct":
            self.n_f = None
        else:
            longest = int(lengths.max()) if lengths.size else 1
            self.n_f = int(n_f) if n_f else _noise.fft_length(self.n_c, longest)
        self.ninv_mode = ninv

    def active(self):
        """[n_slots, 3] mask of the unknowns that exist (not excised, within the counts)."""
        m = np.zeros((self.n_obs, 3), dtype=bool)
        m[:, 0] = ~self.excised
        m[:, 1] = m[:, 2] = ~self.excised_pol
        return m

    def unpoint(self, x):
        x = np.asarray(x, dtype=np.float64).reshape(self.n_obs, 3)
        ok = self.pi >= 0
        i, q = np.where(ok, self.pi, 0), np.where(ok, self.pq, 0)
        y = x[i, 0] + self.c * x[q, 1] + self.s * x[q, 2]
        return np.where(ok, y, 0.0)

    def point(self, y):
        ok = self.pi >= 0
        out = np.zeros((self.n_obs, 3))
        out[:, 0] = np.bincount(self.pi[ok], weights=y[ok], minlength=self.n_obs)
        out[:, 1] = np.bincount(self.pq[ok], weights=(y * self.c)[ok], minlength=self.n_obs)
        out[:, 2] = np.bincount(self.pq[ok], weights=(y * self.s)[ok], minlength=self.n_obs)
        return out

    def ninv(self, y):
        if self.ninv_mode == "direct":
            return _noise.apply_ninv_direct(y, self.offsets, self.ivl_filter, self.lags)
        return _noise.apply_ninv_fft(y, self.offsets, self.ivl_filter, self.lags, self.n_f)

    def H(self, x):
        return self.point(self.ninv(self.unpoint(x)))

    def rhs(self, d):
        return self.point(self.ninv(np.asarray(d, dtype=np.float64)))

    def precond(self, r):
        return np.einsum("pab,pb->pa", self.Pinv, r)

    def pcg(self, b, rel_tol=1e-6, max_iter=50, keep_history=False):
        b = np.asarray(b, dtype=np.float64).reshape(self.n_obs, 3)
        return _pcg(self.H, self.precond, b, rel_tol, max_iter, keep_history)

    def solve(self, d, rel_tol=1e-6, max_iter=50, keep_history=False):
        return self.pcg(self.rhs(d), rel_tol, max_iter, keep_history)

    def dense_H(self):
        n_t = self.pi.shape[0]
        A = np.zeros((n_t, self.n_obs * 3))
        for t in range(n_t):
            if self.pi[t] < 0:
                continue
            A[t, 3 * self.pi[t]] = 1.0
            A[t, 3 * self.pq[t] + 1] = self.c[t]
            A[t, 3 * self.pq[t] + 2] = self.s[t]
        N = _noise.dense_ninv(self.offsets, self.ivl_filter, self.lags)
        return A, N, A.T @ N @ A

    def dense_solve(self, d):
        """Brute-force ML map (Section 3, Eq. 8) over the active unknowns, by Cholesky."""
        A, N, H = self.dense_H()
        b = A.T @ N @ np.asarray(d, dtype=np.float64)
        keep = self.active().reshape(-1)
        x = np.zeros(self.n_obs * 3)
        L = np.linalg.cholesky(H[np.ix_(keep, keep)])
        x[keep] = np.linalg.solve(L.T, np.linalg.solve(L, b[keep]))
        return x.reshape(self.n_obs, 3)
