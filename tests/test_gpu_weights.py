"""The float32 operator's polarisation weights against exact ones.

Section 3, Eq. 4 (relabelled): each IQU sample has the weights (1, cos 2psi,
sin 2psi).  The float32 kernels reduce 2 psi to [-pi, pi] by Cody and Waite's
two-part subtraction of 2 pi and then use the hardware sine and cosine
approximations.  Error budget against the exact weights of the float32 angle:
the reduction carries at most two roundings of a number below pi (2 x 1.2e-7)
and the approximations are within 4e-7 on [-pi, pi], so 1e-6 absolute bounds
the total.  The float64 kernels' weights are correctly rounded sincos of
2 (double) psi and must agree with float64 numpy to a few ulp.
"""

from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

FP32_WEIGHT_BOUND = 1e-6


def _angles():
    rng = np.random.default_rng(12)
    k = np.arange(-64, 65)
    edges = np.concatenate([k * np.pi / 4, k * np.pi / 4 + 1e-7, k * np.pi / 4 - 1e-7])
    return np.concatenate([
        rng.uniform(-np.pi, np.pi, 200_000),          # the all-sky generator's range
        rng.uniform(-20.0, 20.0, 200_000),            # detector angle plus twice the half-wave plate
        rng.uniform(-1000.0, 1000.0, 100_000),        # far from the origin
        edges,
    ]).astype(np.float32)


def test_fp32_weights_within_bound_of_exact():
    import torch
    import paper_0906_1775_gb300 as mm
    psi = _angles()
    c, s = mm.madmap_polarisation_weights(torch.from_numpy(psi).cuda(), "fp32")
    c, s = c.cpu().numpy().astype(np.float64), s.cpu().numpy().astype(np.float64)
    x = 2.0 * psi.astype(np.float64)
    err = max(np.abs(c - np.cos(x)).max(), np.abs(s - np.sin(x)).max())
    assert err < FP32_WEIGHT_BOUND, err
    # the full-precision float32 library functions on the same angles
    xt = torch.from_numpy(psi).cuda() * 2.0
    cf, sf = torch.cos(xt).cpu().numpy(), torch.sin(xt).cpu().numpy()
    assert max(np.abs(c - cf).max(), np.abs(s - sf).max()) < FP32_WEIGHT_BOUND
    # the weights stay on the unit circle
    assert np.abs(c * c + s * s - 1.0).max() < 2 * FP32_WEIGHT_BOUND


def test_fp64_weights_are_correctly_rounded_sincos():
    import torch
    import paper_0906_1775_gb300 as mm
    psi = _angles()
    c, s = mm.madmap_polarisation_weights(torch.from_numpy(psi).cuda(), "fp64")
    x = 2.0 * psi.astype(np.float64)
    assert np.abs(c.cpu().numpy() - np.cos(x)).max() < 1e-15
    assert np.abs(s.cpu().numpy() - np.sin(x)).max() < 1e-15
