"""Noise model and inverse-noise weighting N^-1 (oracle, FP64).  Test infrastructure only.

* Noise PSD, Section 4 Eq. 13: p(f) = sigma^2 [1 + (f_k / f)^alpha].
* N^-1 is block diagonal, one block per stationary interval, each block a
  banded Toeplitz matrix: N^-1_{t,t'} = f(|t - t'|) for |t - t'| < n_c and 0
  otherwise (Section 5.2, Eq. 15).  Lags tau = 0 .. n_c - 1 (the band edge
  of Eq. 15 is taken as the definition; Eqs. 19-20 write |i - j| > n_c).
* The product with one block is computed exactly by embedding the band in a
  circulant two bandwidths larger, zero-padding the input by one bandwidth at
  each end and trimming one bandwidth from each end of the result; a long
  interval is cut into overlapping FFT blocks that each yield n_f - 2 n_c
  exact outputs (Section 5.2, Eqs. 16-22).  ``apply_ninv_direct`` computes
  the same product straight from Eq. 15 and is the brute-force check.
* FFT length: h(n_f) = n_f ln n_f / (n_f - 2 n_c) (Eq. 23), its derivative
  (Eq. 24), the critical point n_f - 2 n_c (1 + ln n_f) = 0 (Eq. 26) shown to
  be a minimum in Appendix A, and the power-of-two rule of Section 5.2.

Filter lags from the PSD.  The paper states that filters are computed from
parametric noise at run time but gives no formula.  Reading used here: sample
1/p on the L = 4 n_c point frequency grid nu_j = min(j, L - j) f_s / L, give
the zero-frequency bin the value of the first non-zero bin (detectors have
finite power at f = 0, Section 4 footnote), inverse-DFT to lags c_tau, and
taper with a Bartlett window w_tau = 1 - tau / n_c.  The tapered band is then
a Fejer-kernel average of a positive spectrum, so every Toeplitz block is
positive definite, which Section 3 requires for an unbiased map.
"""

from __future__ import annotations

import math

import numpy as np


# ------------------------------------------------------------------ PSD and lags
def psd(nu, sigma, fknee, alpha):
    """Eq. 13: p(f) = sigma^2 [1 + (f_k / f)^alpha]."""
    nu = np.asarray(nu, dtype=np.float64)
    return sigma * sigma * (1.0 + (fknee / nu) ** alpha)


def _grid(n_lags: int, fs: float):
    L = 4 * n_lags
    j = np.arange(L)
    nu = np.minimum(j, L - j).astype(np.float64) * fs / L
    nu[0] = nu[1]
    return L, nu


def filter_lags(n_lags: int, fs: float, sigma: float, fknee: float, alpha: float,
                with_grad: bool = False):
    """Inverse-noise filter f(0 .. n_c-1) for one stationary interval.

    Returns f (float64 [n_lags]); with ``with_grad`` also df/d(sigma, f_k,
    alpha) as float64 [3, n_lags].  Parity pinned by test_filter_* (white-noise
    limit, the alpha = 2 Lorentzian closed form, 1/sigma^2 scaling, positive
    definiteness, finite differences).
    """
    L, nu = _grid(n_lags, fs)
    q = 1.0 / psd(nu, sigma, fknee, alpha)
    taper = 1.0 - np.arange(n_lags, dtype=np.float64) / n_lags
    # c_tau = (1/L) sum_j q_j cos(2 pi j tau / L); q is even in j so the DFT is real.
    c = np.real(np.fft.ifft(q))[:n_lags]
    f = taper * c
    if not with_grad:
        return f
    r = (fknee / nu) ** alpha
    dq = np.empty((3, L))
    dq[0] = -2.0 * q / sigma
    dq[1] = -q * q * sigma * sigma * alpha * r / fknee
    dq[2] = -q * q * sigma * sigma * r * np.log(fknee / nu)
    g = taper[None, :] * np.real(np.fft.ifft(dq, axis=1))[:, :n_lags]
    return f, g


def toeplitz_symbol(f: np.ndarray, n_grid: int) -> np.ndarray:
    """Symbol S(theta) = f0 + 2 sum_tau f_tau cos(tau theta) on n_grid angles in [0, pi]."""
    th = np.linspace(0.0, np.pi, n_grid)
    tau = np.arange(1, f.shape[0])
    return f[0] + 2.0 * (np.cos(np.outer(th, tau)) @ f[1:])


# ------------------------------------------------------------------ N^-1 products
def apply_ninv_direct(y: np.ndarray, offsets: np.ndarray, ivl_filter: np.ndarray,
                      lags: np.ndarray) -> np.ndarray:
    """w = N^-1 y straight from Eq. 15, interval by interval, O(n n_c)."""
    out = np.zeros_like(y, dtype=np.float64)
    n_c = lags.shape[1]
    for i in range(ivl_filter.shape[0]):
        a, b = int(offsets[i]), int(offsets[i + 1])
        seg = np.asarray(y[a:b], dtype=np.float64)
        f = lags[ivl_filter[i]]
        w = f[0] * seg
        for tau in range(1, min(n_c, b - a)):
            w[tau:] += f[tau] * seg[:-tau]
            w[:-tau] += f[tau] * seg[tau:]
        out[a:b] = w
    return out


def circulant_spectrum(f: np.ndarray, n_f: int) -> np.ndarray:
    """DFT of the first column of the n_f x n_f circulant holding the band (Eqs. 16-18)."""
    n_c = f.shape[0]
    col = np.zeros(n_f)
    col[:n_c] = f
    col[n_f - n_c + 1:] = f[1:][::-1]
    return np.fft.rfft(col)


def apply_ninv_fft(y: np.ndarray, offsets: np.ndarray, ivl_filter: np.ndarray,
                   lags: np.ndarray, n_f: int) -> np.ndarray:
    """w = N^-1 y by circulant embedding and overlapping FFT blocks (Section 5.2).

    Each interval is padded with n_c zeros at both ends; block j multiplies the
    n_f samples starting at j (n_f - 2 n_c) of the padded interval by the
    circulant and keeps the n_f - 2 n_c central outputs.  Exact (Eq. 21 with the
    offset b = n_c); pinned against ``apply_ninv_direct`` and the dense matrix.
    """
    n_c = lags.shape[1]
    if n_f <= 2 * n_c:
        raise ValueError("n_f must exceed 2 n_c")
    U = n_f - 2 * n_c
    spectra = {}
    out = np.zeros_like(y, dtype=np.float64)
    for i in range(ivl_filter.shape[0]):
        a, b = int(offsets[i]), int(offsets[i + 1])
        n = b - a
        k = int(ivl_filter[i])
        if k not in spectra:
            spectra[k] = circulant_spectrum(lags[k], n_f)
        F = spectra[k]
        n_blocks = -(-n // U)
        pad = np.zeros(n_blocks * U + 2 * n_c)
        pad[n_c:n_c + n] = y[a:b]
        w = np.empty(n_blocks * U)
        for j in range(n_blocks):
            win = pad[j * U:j * U + n_f]
            w[j * U:(j + 1) * U] = np.fft.irfft(np.fft.rfft(win) * F, n_f)[n_c:n_c + U]
        out[a:b] = w[:n]
    return out


def dense_ninv(offsets: np.ndarray, ivl_filter: np.ndarray, lags: np.ndarray) -> np.ndarray:
    """Explicit block-diagonal banded Toeplitz N^-1 of Eq. 15 (tiny problems only)."""
    n_t = int(offsets[-1])
    n_c = lags.shape[1]
    M = np.zeros((n_t, n_t))
    for i in range(ivl_filter.shape[0]):
        a, b = int(offsets[i]), int(offsets[i + 1])
        f = lags[ivl_filter[i]]
        for t in range(a, b):
            for tp in range(a, b):
                if abs(t - tp) < n_c:
                    M[t, tp] = f[abs(t - tp)]
    return M


# ------------------------------------------------------------------ FFT length
def h(n_f, n_c):
    """Eq. 23: cost per exact output, up to constants."""
    return n_f * math.log(n_f) / (n_f - 2 * n_c)


def hprime(n_f, n_c):
    """Eq. 24."""
    return (1.0 + math.log(n_f)) / (n_f - 2 * n_c) - n_f * math.log(n_f) / (n_f - 2 * n_c) ** 2


def hsecond(n_f, n_c):
    """Eq. 25."""
    d = n_f - 2 * n_c
    return 2 * n_f * math.log(n_f) / d ** 3 - 2 * (1 + math.log(n_f)) / d ** 2 + 1.0 / (n_f * d)


def optimal_nf(n_c: int) -> float:
    """Root of n_f - 2 n_c (1 + ln n_f) = 0 above 2 n_c (Eq. 26), by bisection."""
    g = lambda x: x - 2.0 * n_c * (1.0 + math.log(x))  # noqa: E731
    lo, hi = 2.0 * n_c, 4.0 * n_c
    while g(hi) < 0:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) < 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def fft_length(n_c: int, longest: int) -> int:
    """Power-of-two FFT length of Section 5.2.

    Start from the smallest power of two larger than the longest interval (and
    larger than 2 n_c, or no output would be exact).  While h' is positive, halve,
    stopping before a length whose h' is negative or which no longer exceeds 2 n_c.
    """
    n_f = 1
    while n_f <= longest:
        n_f *= 2
    while n_f <= 2 * n_c:
        n_f *= 2
    if hprime(n_f, n_c) > 0:
        while n_f // 2 > 2 * n_c and hprime(n_f // 2, n_c) >= 0:
            n_f //= 2
    return n_f
