"""Pointing matrix A and pixel indexing (oracle, FP64).  Test infrastructure only.

Section 3 (Eq. 3): for temperature, row t of A holds a single unit weight in
the column of the pixel observed at sample t.  Section 3 (Eq. 4) gives the
polarised row as one weight per Stokes parameter.  The paper's row is
(1/2)[i + q sin 2a + u cos 2a]; this library uses the weights
(1, cos 2 psi, sin 2 psi) for (I, Q, U), an exact linear relabelling
(I, Q, U) = (i/2, u/2, q/2) of the paper's Stokes vector (pinned by
tests/test_oracle_pins.py::test_polarisation_relabelling).

Section 5.4: pixels are re-indexed from the global scheme to the observed
scheme (only pixels hit by at least one sample).  The paper builds the map
with an n_z-bit array, one bit per global pixel, set when the pixel is seen;
the observed index of a pixel is its rank among the set bits in ascending
global order.  Rows of flagged samples (pixel -1) and of samples of excised
pixels are zero (Section 4, gap filling: "rows ... set to zero").
"""

from __future__ import annotations

import numpy as np


def observed_pixels(pix: np.ndarray, n_pix: int, chunk: int | None = None):
    """Global -> observed re-indexing through the n_z-bit array of Section 5.4.

    Returns (obs2glob int64 [n_obs] ascending, glob2obs int64 [n_pix] with -1
    for unobserved pixels).  ``chunk`` sets the bits from that many samples at
    a time (for pointing too large to copy whole).  Parity pinned by
    test_observed_pixels_bruteforce.
    """
    bits = np.zeros(n_pix, dtype=bool)          # the n_z-bit array
    n_t = int(pix.shape[0])
    step = n_t if not chunk else int(chunk)
    for lo in range(0, n_t, max(step, 1)):
        c = np.asarray(pix[lo:lo + step])
        bits[c[c >= 0].astype(np.int64)] = True
    obs2glob = np.flatnonzero(bits)             # set bits in ascending global order
    glob2obs = np.full(n_pix, -1, dtype=np.int64)
    glob2obs[obs2glob] = np.arange(obs2glob.size)
    return obs2glob, glob2obs


def local_pixels(pix: np.ndarray, glob2obs: np.ndarray) -> np.ndarray:
    """Observed index of every sample (-1 for flagged samples)."""
    out = np.full(pix.shape[0], -1, dtype=np.int64)
    ok = pix >= 0
    out[ok] = glob2obs[pix[ok]]
    return out


def weights(psi, n_stokes: int) -> np.ndarray:
    """Row weights w_t = (1,) for T or (1, cos 2psi, sin 2psi) for IQU, in float64.

    The angle is promoted from its stored float32 value before the
    trigonometry, so both sides of a parity test see the same angle.
    """
    if n_stokes == 1:
        return None
    two = 2.0 * np.asarray(psi, dtype=np.float64)
    return np.stack([np.ones_like(two), np.cos(two), np.sin(two)], axis=1)


def unpoint(x: np.ndarray, pixl: np.ndarray, w: np.ndarray | None) -> np.ndarray:
    """y = A x  (Section 3, Eq. 2: the signal part of the timestream).

    x is [n_obs, n_s]; pixl the observed pixel of each sample (-1 = zero row).
    """
    ok = pixl >= 0
    p = np.where(ok, pixl, 0)
    if w is None:
        y = x[p, 0].astype(np.float64)
    else:
        y = np.einsum("ts,ts->t", x[p, :], w)
    y[~ok] = 0.0
    return y


def point(y: np.ndarray, pixl: np.ndarray, w: np.ndarray | None, n_obs: int, n_s: int) -> np.ndarray:
    """z = A^T y: sum of weighted samples into their pixels (fixed index order)."""
    ok = pixl >= 0
    p = pixl[ok]
    out = np.zeros((n_obs, n_s))
    if w is None:
        out[:, 0] = np.bincount(p, weights=y[ok], minlength=n_obs)
    else:
        for s in range(n_s):
            out[:, s] = np.bincount(p, weights=y[ok] * w[ok, s], minlength=n_obs)
    return out


def dense_pointing(pixl: np.ndarray, w: np.ndarray | None, n_obs: int, n_s: int) -> np.ndarray:
    """Explicit A as a dense [n_t, n_obs * n_s] matrix (tiny problems only)."""
    n_t = pixl.shape[0]
    A = np.zeros((n_t, n_obs * n_s))
    for t in range(n_t):
        p = pixl[t]
        if p < 0:
            continue
        if w is None:
            A[t, p] = 1.0
        else:
            A[t, p * n_s:(p + 1) * n_s] = w[t]
    return A
