"""Argument checks of madmap_plan_create that run on the host before any device
work (no GPU needed): each malformed description returns MADMAP_ERR_INVALID_ARG
with a message, and no plan."""

from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

FAKE_DEV = 0x1000   # never dereferenced: every case fails before device memory is read


def _lib():
    import os
    import paper_0906_1775_gb300 as mm
    from paper_0906_1775_gb300 import build
    if not os.path.exists(mm.library_path()):
        build.build()
    return mm


def _desc(mm, keep, **kw):
    L = mm._lib
    off = np.array([0, 600, 1000], dtype=np.int64)
    filt = np.array([0, 0], dtype=np.int32)
    lags = np.array([[1.0, 0.2, 0.05]])
    keep.extend([off, filt, lags])
    d = L.madmap_plan_desc()
    d.n_stokes, d.n_samples, d.n_pix = 3, 1000, 64
    d.pix, d.psi = FAKE_DEV, FAKE_DEV
    d.n_intervals = 2
    d.interval_offsets, d.interval_filter = off.ctypes.data, filt.ctypes.data
    d.n_filters, d.n_lags = 1, 3
    d.filter_lags = lags.ctypes.data
    for k, v in kw.items():
        if isinstance(v, np.ndarray):
            keep.append(v)
            v = v.ctypes.data
        setattr(d, k, v)
    return d


CASES = {
    "n_stokes": dict(n_stokes=2),
    "n_pix": dict(n_pix=0),
    "psi_for_T": dict(n_stokes=1),
    "offsets_end": dict(interval_offsets=np.array([0, 600, 999], dtype=np.int64)),
    "offsets_order": dict(interval_offsets=np.array([0, 700, 600, 1000], dtype=np.int64), n_intervals=3,
                          interval_filter=np.zeros(3, np.int32)),
    "filter_range": dict(interval_filter=np.array([0, 1], dtype=np.int32)),
    "lags_finite": dict(filter_lags=np.array([[1.0, np.nan, 0.0]])),
    "fft_len": dict(fft_len=1000),
    "pix_pol_T": dict(n_stokes=1, psi=None, pix_pol=FAKE_DEV, n_pix_pol=16),
    "extra_with_pol": dict(extra_index=FAKE_DEV, n_extra=4, pix_pol=FAKE_DEV, n_pix_pol=16),
    "extra_count": dict(extra_index=FAKE_DEV, n_extra=0),
    "hwp_without_tau": dict(hwp_angle=FAKE_DEV, n_hwp_groups=1,
                            interval_hwp_group=np.array([0, 0], dtype=np.int32)),
    "hwp_group_range": dict(hwp_angle=FAKE_DEV, hwp_tau=FAKE_DEV, n_hwp_groups=1,
                            interval_hwp_group=np.array([0, 1], dtype=np.int32)),
    "boresight_with_pix": dict(boresight=FAKE_DEV, n_bore=600, bore_step=2, n_det=2,
                               det_pointing=np.zeros((2, 4), np.float32), grid_width=8, grid_height=8),
    "boresight_nodes": dict(pix=None, psi=None, boresight=FAKE_DEV, n_bore=10, bore_step=2, n_det=2,
                            det_pointing=np.zeros((2, 4), np.float32), grid_width=8, grid_height=8),
    "boresight_grid": dict(pix=None, psi=None, boresight=FAKE_DEV, n_bore=300, bore_step=2, n_det=2,
                           det_pointing=np.zeros((2, 4), np.float32), grid_width=8, grid_height=7),
    "boresight_det_finite": dict(pix=None, psi=None, boresight=FAKE_DEV, n_bore=300, bore_step=2, n_det=2,
                                 det_pointing=np.array([[0, 0, 1, 0], [np.inf, 0, 1, 0]], np.float32),
                                 grid_width=8, grid_height=8),
    "boresight_interval_spans_detectors": dict(pix=None, psi=None, boresight=FAKE_DEV, n_bore=300, bore_step=2,
                                               n_det=2, det_pointing=np.zeros((2, 4), np.float32),
                                               grid_width=8, grid_height=8),
    "deterministic_extended": dict(deterministic=1, extra_index=FAKE_DEV, n_extra=4),
    "deterministic_multires": dict(deterministic=1, pix_pol=FAKE_DEV, n_pix_pol=16),
    "sharded_multires": dict(allreduce="reducer", pix_pol=FAKE_DEV, n_pix_pol=16),
    "sharded_extended": dict(allreduce="reducer", extra_index=FAKE_DEV, n_extra=4),
    "scatter_runs_high": dict(scatter_runs=2),
    "scatter_runs_low": dict(scatter_runs=-2),
    "fft_split": dict(fft_split=2),
}


def _reducer(mm, keep):
    fn = mm._lib.REDUCE_FN(lambda buf, count, dtype, stream, user: 0)
    keep.append(fn)
    return fn


@pytest.mark.parametrize("case", list(CASES))
def test_malformed_description_is_rejected_on_the_host(case):
    mm = _lib()
    keep = []
    kw = dict(CASES[case])
    if kw.get("allreduce") == "reducer":
        kw["allreduce"] = _reducer(mm, keep)
    d = _desc(mm, keep, **kw)
    h = C.c_void_p()
    st = mm.load().madmap_plan_create(C.byref(d), None, C.byref(h))
    msg = mm.madmap_last_error()
    assert st == mm._lib.MADMAP_ERR_INVALID_ARG, (case, st, msg)
    assert not h.value
    assert KEYWORD.get(case, "") in msg, (case, msg)


KEYWORD = {
    "n_stokes": "n_stokes", "n_pix": "n_pix", "psi_for_T": "psi", "offsets_end": "interval_offsets",
    "offsets_order": "non-decreasing", "filter_range": "interval_filter", "lags_finite": "finite",
    "fft_len": "fft_len", "pix_pol_T": "pix_pol", "extra_with_pol": "extra_index", "extra_count": "n_extra",
    "hwp_without_tau": "hwp_tau", "hwp_group_range": "interval_hwp_group", "boresight_with_pix": "must be NULL",
    "boresight_nodes": "n_bore", "boresight_grid": "grid_width", "boresight_det_finite": "det_pointing",
    "boresight_interval_spans_detectors": "spans two detectors",
    "deterministic_extended": "deterministic", "deterministic_multires": "deterministic",
    "sharded_multires": "sharded", "sharded_extended": "sharded",
    "scatter_runs_high": "scatter_runs", "scatter_runs_low": "scatter_runs", "fft_split": "fft_split",
}


@pytest.mark.parametrize("case", ["precision", "offsets", "filter", "lags", "too_many_lags"])
def test_noalloc_weighting_checks_its_arguments_on_the_host(case):
    mm = _lib()
    L = mm.load()
    off = np.array([0, 500, 1000], dtype=np.int64)
    filt = np.array([0, 0], dtype=np.int32)
    lags = np.array([[1.0, 0.1]])
    prec, n_lags = mm._lib.MADMAP_FP64, 2
    if case == "precision":
        prec = mm._lib.MADMAP_MIXED
    elif case == "offsets":
        off = np.array([0, 500, 999], dtype=np.int64)
    elif case == "filter":
        filt = np.array([0, 3], dtype=np.int32)
    elif case == "lags":
        lags = np.array([[1.0, np.inf]])
    else:
        n_lags = (1 << 15) + 1
        lags = np.ones((1, n_lags))
    st = L.madmap_apply_ninv_noalloc(prec, 1000, 2, off.ctypes.data, filt.ctypes.data, 1, n_lags, lags.ctypes.data,
                                     FAKE_DEV, FAKE_DEV, None)
    assert st == mm._lib.MADMAP_ERR_INVALID_ARG, (case, st, mm.madmap_last_error())
    assert "apply_ninv_noalloc" in mm.madmap_last_error()
