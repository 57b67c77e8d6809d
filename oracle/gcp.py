"""Pointing expanded from compressed boresight pointing (oracle).  Test infrastructure only.

Section 5.3: instead of storing a pixel index and weight for every detector
sample, the pointing is held in a compressed form sampled at a constant,
lower rate, and the sparse rows of A are produced when needed: the
boresight pointing is interpolated to the detector sample rate, rotated to
each detector's offset from the boresight, discretised into a pixel index,
and given the detector's polarisation weights.  The paper leaves the
representation experiment-specific; the one used here (written out so the
GPU library and this oracle make the same integer decisions) is:

* boresight node u (u = 0 .. n_bore-1) at detector sample j = u * step holds
  float32 (x_u, y_u, c_u, s_u): position on a flat W x H pixel grid in pixel
  units and the boresight orientation as (cos, sin);
* detector d holds float32 (dx_d, dy_d, cd_d, sd_d): its offset in the focal
  plane and its polariser orientation relative to the boresight;
* sample t = d * n_per_det + j of detector d: with u = j div step and
  f = (j mod step) / step, every node quantity q is interpolated linearly,
  q = q_u + f (q_{u+1} - q_u); the detector sits at
  X = x + (c dx - s dy), Y = y + (s dx + c dy); its pixel is
  floor(Y) * W + floor(X) when 0 <= X < W and 0 <= Y < H, else the sample is
  flagged (-1);
* polarisation (IQU): the detector's orientation is (C, S) =
  (c cd - s sd, s cd + c sd) (angle addition); with n = C^2 + S^2 its weights
  are cos 2psi = (C^2 - S^2) / n and sin 2psi = 2 C S / n (double angle,
  normalised because interpolated (c, s) are not of unit length).  A sample
  with n = 0 is flagged.

Every step is one float32 operation rounded to nearest, in the order written
above (no fused multiply-add), so the pixel decisions are bit-exact between
this oracle and the GPU.  The weights feed oracle.solver.System through its
``weights`` argument.

Pinned by tests/test_oracle_pins.py::test_gcp_* (exact dyadic cases against
rational arithmetic, angle addition against the trigonometric functions,
agreement with the float64 position away from pixel edges, flags).
"""

from __future__ import annotations

import numpy as np

F32 = np.float32


def expand(boresight, step, det, n_per_det, width, height, polarised=True, chunk=1 << 22):
    """(pix int64 [n_t], cos2psi float32 [n_t] or None, sin2psi float32 [n_t] or None).

    boresight float32 [n_bore, 4]; det float32 [n_det, 4]; n_t = n_det * n_per_det.
    """
    bore = np.asarray(boresight, dtype=F32)
    det = np.asarray(det, dtype=F32)
    n_det = det.shape[0]
    n_t = n_det * int(n_per_det)
    pix = np.empty(n_t, dtype=np.int64)
    c2 = np.empty(n_t, dtype=F32) if polarised else None
    s2 = np.empty(n_t, dtype=F32) if polarised else None
    stepf = F32(step)
    for d in range(n_det):
        dx, dy, cd, sd = (F32(v) for v in det[d])
        for j0 in range(0, int(n_per_det), chunk):
            j = np.arange(j0, min(int(n_per_det), j0 + chunk), dtype=np.int64)
            u = j // step
            f = (j - u * step).astype(F32) / stepf
            lo, hi = bore[u], bore[u + 1]
            q = lo + f[:, None] * (hi - lo)                       # interpolated (x, y, c, s)
            x, y, c, s = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
            X = x + (c * dx - s * dy)
            Y = y + (s * dx + c * dy)
            ix, iy = np.floor(X), np.floor(Y)
            ok = (ix >= 0) & (ix < width) & (iy >= 0) & (iy < height)
            p = np.where(ok, iy.astype(np.int64) * width + ix.astype(np.int64), -1)
            sl = slice(d * int(n_per_det) + j0, d * int(n_per_det) + j0 + j.size)
            if polarised:
                C = c * cd - s * sd
                S = s * cd + c * sd
                cc, ss = C * C, S * S
                n = cc + ss
                good = n > 0
                cs = C * S
                with np.errstate(divide="ignore", invalid="ignore"):
                    c2[sl] = np.where(good, (cc - ss) / n, F32(0))
                    s2[sl] = np.where(good, (cs + cs) / n, F32(0))
                p = np.where(good, p, -1)
            pix[sl] = p
    return pix, c2, s2


def nodes_needed(n_per_det, step):
    """Boresight nodes an expansion of n_per_det samples reads (node u + 1 of the last sample)."""
    return (int(n_per_det) - 1) // int(step) + 2 if n_per_det > 0 else 0
