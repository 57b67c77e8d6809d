"""Extended pointing: destriping offsets and binned synchronous templates
(oracle, FP64).  Test infrastructure only.

Section 6 (items 1 and 3): the data model gains a term B o, d = A z + B o + n,
and the map vector and pointing matrix are extended to [z; o] and [A B]
(Eqs. 39-40), so the same PCG solves for both.  Here B has one unit entry per
sample: column e_t = ``extra_index[t]`` (-1: none).  That covers

* destriping offsets (item 3): e_t = the baseline interval of sample t, with
  N white (one filter lag, so no FFT is involved);
* non-parametric synchronous signals (item 1): e_t = the bin of the sample's
  synchronous parameter (e.g. a chopper angle);

and, for the parametric half-wave-plate signal of item 2 (Eqs. 41-42), a
dense block C of 32 columns per group of intervals: with the polariser angle
w_t and the time variable tau_t of sample t, C_{t,k} = cos k w_t,
C_{t,8+k} = tau_t cos k w_t, C_{t,16+k} = sin k w_t, C_{t,24+k} = tau_t sin k w_t
for k = 1..8 (the paper's column order).

Readings where the paper is silent:
* A sample that is flagged (pixel -1) or whose sky pixel is excised has a zero
  row in both blocks (gap filling, Section 4).
* The sky pixels' preconditioner blocks and their excision come from the sky
  block A alone (as without extra columns); each extra column's block is the
  scalar 1 / (B^T W^-1 B), W^-1 = diag(N^-1); an extra column without samples
  is excised.
* The layout: vectors are [n_obs + n_extra, n_s]: the sky rows, then one row
  per extra column holding its amplitude in slot 0 (its other slots are
  unused and stay 0).
* The system must be non-singular: offsets that cover every sample are
  degenerate with a constant I map, so the caller gives one baseline no
  offset (extra index -1), as destripers fix one offset.
* Half-wave-plate parameters: each interval belongs to a group (-1: none)
  with its own 32 parameters; tau_t is supplied by the caller (its origin and
  unit are the caller's choice); the preconditioner of each parameter is the
  scalar 1 / sum_t f(0) C_{t,i}^2 (the paper gives none for templates; the
  32 x 32 block is not formed); a parameter with a zero sum is excised.
  Their rows follow the extra columns' rows, one row per parameter (slot 0).

Pinned by tests/test_oracle_pins.py::test_extended_* (reduction to the plain
system without extra columns, dense Cholesky and symmetry, noiseless recovery
of sky and offsets with white noise, recovery of a binned template).
"""

from __future__ import annotations

import numpy as np

from . import noise as _noise
from .solver import System, pcg as _pcg


class ExtendedSystem:
    def __init__(self, pix, psi, n_pix, n_stokes, offsets, ivl_filter, lags, extra_index, n_extra,
                 rcond_excise=1e-6, rcond_fp64=1e-2, ninv="fft", n_f=None, weights=None, hwp=None):
        """hwp (optional): (angle float32 [n_t], tau float32 [n_t], group of each interval [n_ivl],
        n_groups) for the 32-parameter half-wave-plate model."""
        self.sky = System(pix, psi, n_pix, n_stokes, offsets, ivl_filter, lags, rcond_excise=rcond_excise,
                          rcond_fp64=rcond_fp64, ninv=ninv, n_f=n_f, weights=weights)
        S = self.sky
        self.n_s = S.n_s
        self.n_sky = S.n_obs
        self.n_extra = int(n_extra)
        self.n_groups = int(hwp[3]) if hwp is not None else 0
        self.n_hwp = 32 * self.n_groups
        self.n_obs = self.n_sky + self.n_extra + self.n_hwp
        self.obs2glob, self.excised_sky = S.obs2glob, S.excised
        e = np.asarray(extra_index, dtype=np.int64)
        # rows that are zero in A (flagged or excised sky pixel) are zero in B too
        self.ex = np.where((S.pixl >= 0) & (e >= 0), e, -1)
        lengths = np.diff(S.offsets)
        f0 = np.repeat(S.lags[S.ivl_filter, 0], lengths)
        ok = self.ex >= 0
        self.hits_extra = np.bincount(self.ex[ok], minlength=self.n_extra)
        wsum = np.bincount(self.ex[ok], weights=f0[ok], minlength=self.n_extra)
        self.excised_extra = self.hits_extra == 0
        with np.errstate(divide="ignore"):
            self.p_extra = np.where(self.excised_extra, 0.0, 1.0 / np.where(self.excised_extra, 1.0, wsum))
        # half-wave-plate block: group of every sample (-1 where its row is zero) and C
        if self.n_groups:
            ang, tau, grp, _ = hwp
            g = np.repeat(np.asarray(grp, dtype=np.int64), lengths)
            self.hg = np.where(S.pixl >= 0, g, -1)
            self.C = hwp_columns(ang, tau)                       # [n_t, 32] float64
            okh = self.hg >= 0
            csum = np.zeros((self.n_groups, 32))
            for i in range(32):
                csum[:, i] = np.bincount(self.hg[okh], weights=f0[okh] * self.C[okh, i] ** 2,
                                         minlength=self.n_groups)
            csum = csum.reshape(-1)
            self.excised_hwp = ~(csum > 0)
            with np.errstate(divide="ignore"):
                self.p_hwp = np.where(self.excised_hwp, 0.0, 1.0 / np.where(self.excised_hwp, 1.0, csum))
        else:
            self.hg = np.full(e.shape[0], -1, dtype=np.int64)
            self.C = None
            self.excised_hwp = np.zeros(0, dtype=bool)
            self.p_hwp = np.zeros(0)

    # the noise description (as the plain system's)
    offsets = property(lambda self: self.sky.offsets)
    ivl_filter = property(lambda self: self.sky.ivl_filter)
    lags = property(lambda self: self.sky.lags)
    n_c = property(lambda self: self.sky.n_c)

    # ---------------------------------------------------------------- layout
    def active(self):
        """[n_obs + n_extra, n_s] mask of the unknowns that exist."""
        m = np.zeros((self.n_obs, self.n_s), dtype=bool)
        m[:self.n_sky] = ~self.excised_sky[:, None]
        m[self.n_sky:self.n_sky + self.n_extra, 0] = ~self.excised_extra
        m[self.n_sky + self.n_extra:, 0] = ~self.excised_hwp
        return m

    def split(self, x):
        """(sky [n_sky, n_s], extra amplitudes [n_extra], half-wave-plate parameters [n_groups, 32])."""
        x = np.asarray(x, dtype=np.float64).reshape(self.n_obs, self.n_s)
        e0 = self.n_sky + self.n_extra
        return x[:self.n_sky], x[self.n_sky:e0, 0], x[e0:, 0].reshape(self.n_groups, 32)

    # ---------------------------------------------------------------- operators
    def unpoint(self, x):
        z, o, b = self.split(x)
        y = self.sky.unpoint(z)
        ok = self.ex >= 0
        y[ok] += o[self.ex[ok]]
        if self.n_groups:
            okh = self.hg >= 0
            y[okh] += np.einsum("ti,ti->t", self.C[okh], b[self.hg[okh]])
        return y

    def point(self, y):
        y = np.asarray(y, dtype=np.float64)
        out = np.zeros((self.n_obs, self.n_s))
        out[:self.n_sky] = self.sky.point(y)
        ok = self.ex >= 0
        e0 = self.n_sky + self.n_extra
        out[self.n_sky:e0, 0] = np.bincount(self.ex[ok], weights=y[ok], minlength=self.n_extra)
        if self.n_groups:
            okh = self.hg >= 0
            hb = np.zeros((self.n_groups, 32))
            for i in range(32):
                hb[:, i] = np.bincount(self.hg[okh], weights=y[okh] * self.C[okh, i], minlength=self.n_groups)
            out[e0:, 0] = hb.reshape(-1)
        return out

    def ninv(self, y):
        return self.sky.ninv(y)

    def H(self, x):
        """[A B]^T N^-1 [A B] x (Eq. 10 with the extended pointing of Eq. 40)."""
        return self.point(self.ninv(self.unpoint(x)))

    def rhs(self, d):
        return self.point(self.ninv(np.asarray(d, dtype=np.float64)))

    def precond(self, r):
        r = np.asarray(r, dtype=np.float64).reshape(self.n_obs, self.n_s)
        out = np.zeros_like(r)
        e0 = self.n_sky + self.n_extra
        out[:self.n_sky] = self.sky.precond(r[:self.n_sky])
        out[self.n_sky:e0, 0] = self.p_extra * r[self.n_sky:e0, 0]
        out[e0:, 0] = self.p_hwp * r[e0:, 0]
        return out

    def pcg(self, b, rel_tol=1e-6, max_iter=50, keep_history=False):
        b = np.asarray(b, dtype=np.float64).reshape(self.n_obs, self.n_s)
        return _pcg(self.H, self.precond, b, rel_tol, max_iter, keep_history)

    def solve(self, d, rel_tol=1e-6, max_iter=50, keep_history=False):
        return self.pcg(self.rhs(d), rel_tol, max_iter, keep_history)

    # ---------------------------------------------------------------- dense
    def dense_H(self):
        n_t = self.ex.shape[0]
        A = np.zeros((n_t, self.n_obs * self.n_s))
        S = self.sky
        for t in range(n_t):
            p = S.pixl[t]
            if p < 0:
                continue
            if S.w is None:
                A[t, p] = 1.0
            else:
                A[t, p * self.n_s:(p + 1) * self.n_s] = S.w[t]
            if self.ex[t] >= 0:
                A[t, (self.n_sky + self.ex[t]) * self.n_s] = 1.0
            if self.hg[t] >= 0:
                base = self.n_sky + self.n_extra + 32 * self.hg[t]
                A[t, (base + np.arange(32)) * self.n_s] = self.C[t]
        N = _noise.dense_ninv(S.offsets, S.ivl_filter, S.lags)
        return A, N, A.T @ N @ A

    def dense_solve(self, d):
        """Brute-force ML solution of the extended system over its active unknowns, by Cholesky."""
        A, N, H = self.dense_H()
        b = A.T @ N @ np.asarray(d, dtype=np.float64)
        keep = self.active().reshape(-1)
        x = np.zeros(self.n_obs * self.n_s)
        L = np.linalg.cholesky(H[np.ix_(keep, keep)])
        x[keep] = np.linalg.solve(L.T, np.linalg.solve(L, b[keep]))
        return x.reshape(self.n_obs, self.n_s)


def hwp_columns(angle, tau):
    """The 32 columns of Eq. 42 for every sample, float64 from the float32 inputs."""
    w = np.asarray(angle, dtype=np.float32).astype(np.float64)
    t = np.asarray(tau, dtype=np.float32).astype(np.float64)
    k = np.arange(1, 9)
    c, s = np.cos(np.outer(w, k)), np.sin(np.outer(w, k))
    return np.concatenate([c, t[:, None] * c, s, t[:, None] * s], axis=1)
