"""The allocation-free noise weighting against the oracle.

madmap_apply_ninv_noalloc exists for callers that cannot allocate device
memory when they need N^-1 y (an allocator that forbids new allocations after
start-up, a real-time loop that must not stall in cudaMalloc, host code
without its own CUDA memory management).  It keeps everything it derives in a
fixed device array.  These tests check, through the C ABI, that:

* it gives the weighted timestreams of the FP64 oracle (Eq. 15 direct sums on
  a small ragged case; the oracle's overlap-save product, pinned against the
  direct sums, on a case whose windows need several chunks of the array), on
  two calls in a row (the second call must not see leftovers of the first),
  and the same result as madmap_apply_ninv over a plan;
* a call allocates nothing: free device memory is unchanged across a call,
  and the call launches whole three-kernel chunks only;
* sizes beyond the fixed array are refused with a clear error, and so is a
  call made while its stream is being captured into a CUDA graph.

This file is collected last, so a run that stops at the first failure has
already run every other test.
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


def _noalloc(prec, n, off, filt, lags, y, w, stream=None):
    import paper_0906_1775_gb300 as mm
    mm.madmap_apply_ninv_noalloc(prec, n, off, filt, lags, y.data_ptr(), w.data_ptr(), stream=stream)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_weighting_matches_oracle_twice(prec):
    import torch
    from oracle.noise import apply_ninv_direct
    p = _problem()
    lags = dominant_lags(p.n_filters, p.n_lags, seed=17)
    plan = make_plan(p, lags=lags)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(5)
    for call in range(2):
        yh = rng.standard_normal(p.n_samples) * (1 + 10 * call)
        if prec == "fp32":
            yh = yh.astype(np.float32).astype(np.float64)
        y = cuda(yh, dt)
        ref = apply_ninv_direct(yh, p.interval_offsets, p.interval_filter, lags)
        w = torch.full_like(y, float("nan"))
        _noalloc(prec, p.n_samples, p.interval_offsets, p.interval_filter, lags, y, w)
        torch.cuda.synchronize()
        assert rel_rms(host(w), ref) < TOL[prec], (call, prec)
        planned = host(plan.apply_ninv(y, precision=prec))[0]
        assert rel_rms(host(w), planned) < TOL[prec], (call, prec)


def test_noalloc_weighting_several_chunks_allocates_nothing():
    """Windows of 2^14 samples (n_lags = 2^12) over 3.2e6 samples: about 190
    window pairs, more than one chunk of the fixed array holds, so the
    multi-chunk launch path runs."""
    import torch
    import paper_0906_1775_gb300 as mm
    from oracle.noise import apply_ninv_fft
    n_lags, n = 1 << 12, 3_200_000
    rng = np.random.default_rng(11)
    cuts = np.sort(rng.choice(np.arange(1, n), 9, replace=False))
    off = np.concatenate([[0], cuts, [n]]).astype(np.int64)
    filt = (np.arange(10) % 2).astype(np.int32)
    lags = dominant_lags(2, n_lags, seed=23)
    yh = rng.standard_normal(n)
    y = cuda(yh, torch.float64)
    ref = apply_ninv_fft(yh, off, filt, lags, 1 << 15)
    w = torch.empty_like(y)
    _noalloc("fp64", n, off, filt, lags, y, w)          # first call on this device: module loading, if any
    torch.cuda.synchronize()
    assert rel_rms(host(w), ref) < TOL["fp64"]
    w.fill_(float("nan"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    k0 = mm.madmap_kernel_launch_count()
    _noalloc("fp64", n, off, filt, lags, y, w)
    torch.cuda.synchronize()
    k1 = mm.madmap_kernel_launch_count()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert (k1 - k0) % 3 == 0 and k1 - k0 >= 6, k1 - k0      # whole chunks of three kernels, at least two
    assert rel_rms(host(w), ref) < TOL["fp64"]


def test_noalloc_weighting_refuses_stream_capture():
    import torch
    import paper_0906_1775_gb300 as mm
    n = 1000
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(y)
    lags = dominant_lags(1, 8, seed=3)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    caught = None
    with torch.cuda.graph(g, stream=s):
        try:
            _noalloc("fp64", n, np.array([0, n]), np.array([0]), lags, y, w, stream=s)
        except mm.MadmapError as e:
            caught = e
    assert caught is not None and caught.status == mm._lib.MADMAP_ERR_INVALID_ARG
    assert "capture" in str(caught)
    # outside a capture the same call runs
    _noalloc("fp64", n, np.array([0, n]), np.array([0]), lags, y, w)
    torch.cuda.synchronize()


def test_noalloc_weighting_refuses_sizes_beyond_its_array():
    import torch
    import paper_0906_1775_gb300 as mm
    n = 1000
    y = torch.zeros(n, dtype=torch.float64, device="cuda")
    w = torch.zeros_like(y)
    too_many_lags = np.zeros((1, (1 << 15) + 1))
    too_many_lags[0, 0] = 1.0
    with pytest.raises(mm.MadmapError) as e:
        _noalloc("fp64", n, np.array([0, n]), np.array([0]), too_many_lags, y, w)
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG and "MADMAP_NOALLOC_MAX_LAGS" in str(e.value)
    many_filters = np.zeros((80, 1 << 15))
    many_filters[:, 0] = 1.0
    with pytest.raises(mm.MadmapError) as e:
        _noalloc("fp64", n, np.array([0, n]), np.array([0]), many_filters, y, w)
    assert e.value.status == mm._lib.MADMAP_ERR_INVALID_ARG and "MADMAP_NOALLOC_SCRATCH_BYTES" in str(e.value)
