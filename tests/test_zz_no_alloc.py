"""The allocation-free noise weighting against the plan-based one.

madmap_apply_ninv_noalloc exists for callers that cannot allocate device
memory when they need N^-1 y (an allocator that forbids new allocations after
start-up, a real-time loop that must not stall in cudaMalloc, host code
without its own CUDA memory management).  It keeps everything it derives in a
fixed device array, so these tests check that it gives the same weighted
timestreams as madmap_apply_ninv over a plan, on two calls in a row (the
second call must not see leftovers of the first), and that sizes beyond the
fixed array are refused with a clear error.  This file is collected last.
"""

from __future__ import annotations

import numpy as np
import pytest

from tests.gpu_helpers import cuda, dominant_lags, host, make_plan
from tests.helpers import rel_rms, tiny_IQU

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-11, "fp32": 2e-5}   # the operator tolerances of the parity tests


def _problem():
    return tiny_IQU(seed=41, n_per_det=3000, n_lags=40, n_ivl_lo=30, n_ivl_hi=2500)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_weighting_matches_plan_weighting_twice(prec):
    import torch
    import paper_0906_1775_gb300 as mm
    p = _problem()
    lags = dominant_lags(p.n_filters, p.n_lags, seed=17)
    plan = make_plan(p, lags=lags)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(5)
    for call in range(2):
        y = cuda(rng.standard_normal(p.n_samples) * (1 + 10 * call), dt)
        ref = host(plan.apply_ninv(y, precision=prec))[0]
        w = torch.full_like(y, float("nan"))
        mm.madmap_apply_ninv_noalloc(prec, p.n_samples, p.interval_offsets, p.interval_filter, lags,
                                     y.data_ptr(), w.data_ptr())
        torch.cuda.synchronize()
        assert rel_rms(host(w), ref) < TOL[prec], (call, prec)


def test_noalloc_weighting_refuses_sizes_beyond_its_array():
    import torch
    import paper_0906_1775_gb300 as mm
    n = 1000
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(y)
    too_many_lags = np.zeros((1, (1 << 15) + 1))
    too_many_lags[0, 0] = 1.0
    with pytest.raises(mm.MadmapError) as e:
        mm.madmap_apply_ninv_noalloc("fp64", n, np.array([0, n]), np.array([0]), too_many_lags,
                                     y.data_ptr(), w.data_ptr())
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG and "MADMAP_NOALLOC_MAX_LAGS" in str(e.value)
    many_filters = np.zeros((80, 1 << 15))
    many_filters[:, 0] = 1.0
    with pytest.raises(mm.MadmapError) as e:
        mm.madmap_apply_ninv_noalloc("fp64", n, np.array([0, n]), np.array([0]), many_filters,
                                     y.data_ptr(), w.data_ptr())
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG and "MADMAP_NOALLOC_SCRATCH_BYTES" in str(e.value)
