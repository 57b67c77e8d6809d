"""Python binding of libmadmap: the MADmap PCG map-making solve on GB300.

Thin marshalling over the C ABI declared in ``include/madmap.h``: tensors are
passed as device pointers on the caller's current CUDA stream; every step of
the computation runs in the library's CUDA kernels.  PyTorch is used only for
device memory and streams.

    plan = Plan(pix, psi, n_pix, interval_offsets, interval_filter, filter_lags)
    m, info = plan.solve(d, precision="mixed", rel_tol=1e-6)
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _lib
from ._lib import (MADMAP_DF64, MADMAP_FP32, MADMAP_FP64, MADMAP_MIXED, MadmapError, check, load)  # noqa: F401

__all__ = ["Plan", "noise_filter", "paper_fft_length", "MadmapError", "load", "library_path",
           "madmap_partition_intervals", "partition_intervals", "shard_range", "torch_allreduce",
           "madmap_plan_create", "madmap_plan_destroy", "madmap_plan_get_stats", "madmap_plan_observed",
           "madmap_plan_observed_pol", "madmap_plan_expand_pointing",
           "madmap_plan_set_filters", "madmap_apply_ATNA", "madmap_rhs", "madmap_apply_ninv", "madmap_solve",
           "madmap_solve_batched", "madmap_solve_backward", "madmap_noise_filter_vjp", "MadmapSolve",
           "madmap_noise_filter", "madmap_paper_fft_length", "madmap_last_error", "madmap_kernel_launch_count",
           "madmap_time_operator", "madmap_polarisation_weights", "madmap_apply_ninv_noalloc",
           "madmap_solve_resume", "save_checkpoint", "load_checkpoint"]

_PREC = {"fp64": MADMAP_FP64, "mixed": MADMAP_MIXED, "fp32": MADMAP_FP32, "df64": MADMAP_DF64,
         MADMAP_FP64: MADMAP_FP64, MADMAP_MIXED: MADMAP_MIXED, MADMAP_FP32: MADMAP_FP32, MADMAP_DF64: MADMAP_DF64}


def library_path() -> str:
    return _lib.LIB_PATH


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return int(s.cuda_stream)


def _dev_ptr(t, dtype, what):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


# ----------------------------------------------------------------- C-ABI names
def madmap_plan_create(desc, stream=None):
    h = C.c_void_p()
    check(load().madmap_plan_create(C.byref(desc), C.c_void_p(_stream_ptr(stream)), C.byref(h)),
          "madmap_plan_create")
    return h


def madmap_plan_destroy(h):
    check(load().madmap_plan_destroy(h), "madmap_plan_destroy")


def madmap_partition_intervals(interval_offsets, n_ranks) -> np.ndarray:
    """First interval of each rank (int32 [n_ranks + 1]) under the concatenated
    distribution of Section 5.1 (whole intervals, balanced by sample count)."""
    off = np.ascontiguousarray(interval_offsets, dtype=np.int64)
    first = np.zeros(int(n_ranks) + 1, dtype=np.int32)
    check(load().madmap_partition_intervals(int(off.shape[0]) - 1, off.ctypes.data, int(n_ranks),
                                            first.ctypes.data), "madmap_partition_intervals")
    return first


partition_intervals = madmap_partition_intervals


def shard_range(interval_offsets, n_ranks, rank):
    """(first interval, end interval, first sample, end sample) of one rank's share."""
    first = madmap_partition_intervals(interval_offsets, n_ranks)
    off = np.asarray(interval_offsets, dtype=np.int64)
    i0, i1 = int(first[rank]), int(first[rank + 1])
    return i0, i1, int(off[i0]), int(off[i1])


class _DeviceArray:
    """A raw device buffer seen through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


_REDUCE_TYPES = {_lib.MADMAP_REDUCE_F64: "<f8", _lib.MADMAP_REDUCE_F32: "<f4", _lib.MADMAP_REDUCE_I32: "<i4"}


def torch_allreduce(group=None):
    """A madmap_reduce_fn over torch.distributed (sum over the ranks of `group`).

    NCCL process groups sum the device buffer in place, ordered on the library's
    stream; other backends (gloo) copy it to host memory, sum there and copy it
    back before returning.  Pass the result as Plan(..., allreduce=...)."""
    import torch.distributed as dist
    torch = _torch()
    nccl = dist.get_backend(group) == "nccl"

    def reduce(ptr, count, dtype, stream):
        t = torch.as_tensor(_DeviceArray(ptr, count, _REDUCE_TYPES[dtype]), device="cuda")
        es = torch.cuda.ExternalStream(int(stream)) if stream else torch.cuda.default_stream()
        with torch.cuda.stream(es):
            if nccl:
                dist.all_reduce(t, group=group)
            else:
                es.synchronize()
                h = t.cpu()
                dist.all_reduce(h, group=group)
                t.copy_(h)
    return reduce


def _reduce_callback(fn):
    """ctypes wrapper of a Python reducer fn(ptr, count, dtype, stream_ptr); exceptions
    become a non-zero status (the library call then fails with ERR_INTERNAL)."""
    def cb(buf, count, dtype, stream, _user):
        try:
            fn(buf or 0, count, dtype, stream or 0)
            return 0
        except Exception as e:  # pragma: no cover - reported through the status
            cb.error = e
            return 1
    cb.error = None
    return _lib.REDUCE_FN(cb), cb


def madmap_plan_get_stats(h) -> dict:
    s = _lib.madmap_plan_stats()
    check(load().madmap_plan_get_stats(h, C.byref(s)), "madmap_plan_get_stats")
    out = {k: getattr(s, k) for k, _ in s._fields_ if not k.startswith("tuned_")}
    out["tuned"] = [(int(s.tuned_fft_len[k]), int(s.tuned_tiles_per_chunk[k]), float(s.tuned_ms[k]),
                     int(s.tuned_runs[k]), int(s.tuned_n2[k])) for k in range(s.n_tuned)]
    return out


def madmap_plan_observed(h, obs2glob_ptr=None, excised_ptr=None, stream=None) -> int:
    n = C.c_int32()
    check(load().madmap_plan_observed(h, C.byref(n), obs2glob_ptr, excised_ptr,
                                      C.c_void_p(_stream_ptr(stream) if (obs2glob_ptr or excised_ptr) else 0)),
          "madmap_plan_observed")
    return n.value


def madmap_plan_observed_pol(h, obs2glob_pol_ptr=None, excised_pol_ptr=None, stream=None) -> int:
    n = C.c_int32()
    check(load().madmap_plan_observed_pol(h, C.byref(n), obs2glob_pol_ptr, excised_pol_ptr,
                                          C.c_void_p(_stream_ptr(stream) if (obs2glob_pol_ptr or excised_pol_ptr)
                                                     else 0)),
          "madmap_plan_observed_pol")
    return n.value


def madmap_plan_expand_pointing(h, pix_ptr=None, cos2psi_ptr=None, sin2psi_ptr=None, stream=None):
    check(load().madmap_plan_expand_pointing(h, pix_ptr, cos2psi_ptr, sin2psi_ptr, C.c_void_p(_stream_ptr(stream))),
          "madmap_plan_expand_pointing")


def madmap_plan_set_filters(h, lags: np.ndarray, stream=None):
    lags = np.ascontiguousarray(lags, dtype=np.float64)
    check(load().madmap_plan_set_filters(h, lags.ctypes.data, C.c_void_p(_stream_ptr(stream))),
          "madmap_plan_set_filters")


def madmap_apply_ATNA(h, precision, n_rhs, x_ptr, y_ptr, stream=None):
    check(load().madmap_apply_ATNA(h, precision, n_rhs, x_ptr, y_ptr, C.c_void_p(_stream_ptr(stream))),
          "madmap_apply_ATNA")


def madmap_rhs(h, precision, n_rhs, d_ptr, b_ptr, stream=None):
    check(load().madmap_rhs(h, precision, n_rhs, d_ptr, b_ptr, C.c_void_p(_stream_ptr(stream))), "madmap_rhs")


def madmap_apply_ninv(h, precision, n_rhs, y_ptr, w_ptr, stream=None):
    check(load().madmap_apply_ninv(h, precision, n_rhs, y_ptr, w_ptr, C.c_void_p(_stream_ptr(stream))),
          "madmap_apply_ninv")


def madmap_solve(h, d_ptr, m_ptr, opts, stream=None):
    info = _lib.madmap_solve_info()
    st = load().madmap_solve(h, d_ptr, m_ptr, C.byref(opts), C.byref(info), C.c_void_p(_stream_ptr(stream)))
    check(st, "madmap_solve", allow_warn=True)
    return info


def madmap_solve_resume(h, state, m_ptr, opts, stream=None):
    """state: a filled _lib.madmap_checkpoint (host maps)."""
    info = _lib.madmap_solve_info()
    st = load().madmap_solve_resume(h, C.byref(state), m_ptr, C.byref(opts), C.byref(info),
                                    C.c_void_p(_stream_ptr(stream)))
    check(st, "madmap_solve_resume", allow_warn=True)
    return info


# ----------------------------------------------------------------- checkpoints
_CKPT_MAPS = ("x", "r", "z", "p", "x_best")
_CKPT_SCALARS = ("n_obs", "n_stokes", "iters", "best_iter", "rz", "bnorm", "rel_res", "best_rel_res")


class _CheckpointBuffers:
    """Host buffers a solve writes its checkpoints into, and the C callback that hands
    each one to a Python function as a dict of numpy copies."""

    def __init__(self, n_obs, n_stokes, on_checkpoint):
        self.maps = {k: np.zeros((max(n_obs, 1), n_stokes)) for k in _CKPT_MAPS}
        self.c = _lib.madmap_checkpoint()
        for k in _CKPT_MAPS:
            setattr(self.c, k, self.maps[k].ctypes.data)
        self.user = on_checkpoint
        self.error = None

        def fn(ptr, _user):
            try:
                state = checkpoint_state(ptr.contents, self.maps)
                return 1 if (self.user is not None and self.user(state)) else 0
            except BaseException as e:  # keep the exception for the caller; stop the solve
                self.error = e
                return 1
        self.fn = _lib.CHECKPOINT_FN(fn)


def checkpoint_state(c, maps=None):
    """Dict of a madmap_checkpoint: its six scalars, the layout and copies of its five maps."""
    out = {k: getattr(c, k) for k in _CKPT_SCALARS}
    n, ns = int(c.n_obs), int(c.n_stokes)
    for k in _CKPT_MAPS:
        if maps is not None:
            out[k] = maps[k][:n].copy()
        else:
            out[k] = np.ctypeslib.as_array(C.cast(getattr(c, k), C.POINTER(C.c_double)), shape=(n, ns)).copy()
    return out


def save_checkpoint(path, state):
    """Write a checkpoint dict to an .npz file (the paper keeps its checkpoints on disk)."""
    np.savez(path, **{k: np.asarray(v) for k, v in state.items()})


def load_checkpoint(path):
    z = np.load(path)
    out = {k: z[k] for k in _CKPT_MAPS}
    for k in _CKPT_SCALARS:
        v = z[k]
        out[k] = int(v) if k in ("n_obs", "n_stokes", "iters", "best_iter") else float(v)
    return out


def madmap_solve_batched(h, n_rhs, d_ptr, m_ptr, opts, stream=None):
    infos = (_lib.madmap_solve_info * n_rhs)()
    st = load().madmap_solve_batched(h, int(n_rhs), d_ptr, m_ptr, C.byref(opts), infos, C.c_void_p(_stream_ptr(stream)))
    check(st, "madmap_solve_batched", allow_warn=True)
    return infos


def madmap_solve_backward(h, d_ptr, m_ptr, gm_ptr, gd_ptr, gl_ptr, opts, stream=None):
    info = _lib.madmap_solve_info()
    st = load().madmap_solve_backward(h, d_ptr, m_ptr, gm_ptr, gd_ptr, gl_ptr, C.byref(opts), C.byref(info),
                                      C.c_void_p(_stream_ptr(stream)))
    check(st, "madmap_solve_backward", allow_warn=True)
    return info


def madmap_noise_filter_vjp(n_lags, fs, sigma, fknee, alpha, grad_lags):
    g = np.ascontiguousarray(grad_lags, dtype=np.float64)
    out = np.zeros(3)
    check(load().madmap_noise_filter_vjp(int(n_lags), fs, sigma, fknee, alpha, g.ctypes.data, out.ctypes.data),
          "madmap_noise_filter_vjp")
    return out


def madmap_noise_filter(n_lags, fs, sigma, fknee, alpha, with_grad=False):
    lags = np.zeros(n_lags)
    dl = np.zeros((3, n_lags)) if with_grad else None
    check(load().madmap_noise_filter(n_lags, fs, sigma, fknee, alpha, lags.ctypes.data,
                                     dl.ctypes.data if with_grad else None), "madmap_noise_filter")
    return (lags, dl) if with_grad else lags


def madmap_paper_fft_length(n_lags, longest) -> int:
    return int(load().madmap_paper_fft_length(int(n_lags), int(longest)))


def madmap_apply_ninv_noalloc(precision, n_samples, interval_offsets, interval_filter, filter_lags, y_ptr, w_ptr,
                              stream=None):
    """w = N^-1 y without a plan and without any device allocation (fixed scratch)."""
    off = np.ascontiguousarray(interval_offsets, dtype=np.int64)
    filt = np.ascontiguousarray(interval_filter, dtype=np.int32)
    lags = np.ascontiguousarray(np.atleast_2d(filter_lags), dtype=np.float64)
    check(load().madmap_apply_ninv_noalloc(_PREC[precision], int(n_samples), int(filt.shape[0]), off.ctypes.data,
                                           filt.ctypes.data if filt.size else None, int(lags.shape[0]),
                                           int(lags.shape[1]), lags.ctypes.data, y_ptr, w_ptr,
                                           C.c_void_p(_stream_ptr(stream))), "madmap_apply_ninv_noalloc")


def madmap_kernel_launch_count() -> int:
    return int(load().madmap_kernel_launch_count())


def madmap_polarisation_weights(psi, precision="fp32", stream=None):
    """(cos 2psi, sin 2psi) of a float32 CUDA tensor of angles, formed as the
    operator kernels of `precision` ("fp32" or "fp64") form them."""
    torch = _torch()
    ptr = _dev_ptr(psi, torch.float32, "psi")
    dt = torch.float32 if _PREC[precision] == MADMAP_FP32 else torch.float64
    c = torch.empty(psi.shape, dtype=dt, device=psi.device)
    s = torch.empty_like(c)
    check(load().madmap_polarisation_weights(_PREC[precision], int(psi.numel()), ptr, c.data_ptr(), s.data_ptr(),
                                             C.c_void_p(_stream_ptr(stream))), "madmap_polarisation_weights")
    return c, s


def madmap_time_operator(h, precision, reps, stream=None):
    """(ms[4], launches[3]): mean ms per launch of k_f1, k_f2, k_f3 (chunks in sequence) and, in
    ms[3], mean ms of one application as solves launch it (chunks overlapped)."""
    ms = np.zeros(4)
    n = np.zeros(3, dtype=np.int32)
    check(load().madmap_time_operator(h, precision, int(reps), ms.ctypes.data, n.ctypes.data,
                                      C.c_void_p(_stream_ptr(stream))), "madmap_time_operator")
    return ms, n


def madmap_last_error() -> str:
    return load().madmap_last_error().decode(errors="replace")


noise_filter = madmap_noise_filter
paper_fft_length = madmap_paper_fft_length


# ----------------------------------------------------------------- convenience wrapper
class Plan:
    """A libmadmap plan over device-resident pointing.

    pix: int32 CUDA tensor [n_t] (global pixel, -1 flagged); psi: float32 CUDA
    tensor [n_t] or None (temperature); interval_offsets [n_ivl+1],
    interval_filter [n_ivl] and filter_lags [n_filters, n_lags] are host arrays.
    pix_pol (int32 CUDA tensor [n_t], with n_pix_pol) puts Q and U on a second
    pixelisation (multi-resolution maps, IQU only): maps are then [n_obs, 3]
    slots, I of observed I pixel k and Q, U of observed Q/U pixel k in row k.
    extra_index (int32 CUDA tensor [n_t], -1 = none, with n_extra) adds one
    unit-weight extra column per sample (destriping offsets, binned templates):
    maps then have n_obs = sky rows + n_extra rows, the extra amplitudes in
    column 0 of the last n_extra rows.
    hwp = (angle, tau, interval_group, n_groups) adds the 32-parameter half-wave-plate
    model per group of intervals (angle, tau: float32 CUDA tensors [n_t]; interval_group:
    host int32 [n_ivl], -1 = none): 32 * n_groups more rows after the extra rows.
    allreduce = fn(ptr, count, dtype, stream_ptr) makes a sharded plan over this
    rank's share of the intervals (shard_range); fn sums a device buffer across
    the ranks, e.g. torch_allreduce().  Every rank must make the same calls.
    deterministic = True sums every map in a fixed order (bit-reproducible maps).
    autotune = True times candidate FFT lengths and launch chunk sizes, then the
    other split of the length into column and row transforms and the scatter with
    and without run sums, and keeps the fastest (stats["tuned"] lists
    (fft_len, tiles_per_chunk, ms, runs, n2) per candidate).
    scatter_runs = 1 / -1 forces the scatter's run sums on / off (0: the plan's rule).
    fft_split = 1 makes the FFT's column transforms half the default length.
    """

    def __init__(self, pix, psi, n_pix, interval_offsets, interval_filter, filter_lags, rcond_excise=0.0,
                 rcond_fp64=0.0, fft_len=0, tiles_per_chunk=0, stream=None, pix_pol=None, n_pix_pol=0,
                 extra_index=None, n_extra=0, hwp=None, allreduce=None, deterministic=False, autotune=False,
                 scatter_runs=0, fft_split=0):
        torch = _torch()
        self._h = None
        self._reduce = None
        off = np.ascontiguousarray(interval_offsets, dtype=np.int64)
        filt = np.ascontiguousarray(interval_filter, dtype=np.int32)
        lags = np.ascontiguousarray(np.atleast_2d(filter_lags), dtype=np.float64)
        n_t = int(pix.numel())
        d = _lib.madmap_plan_desc()
        d.n_stokes = 1 if psi is None else 3
        d.n_samples = n_t
        d.n_pix = int(n_pix)
        d.pix = _dev_ptr(pix, torch.int32, "pix") if n_t else None
        d.psi = _dev_ptr(psi, torch.float32, "psi") if (psi is not None and n_t) else None
        d.n_intervals = int(filt.shape[0])
        d.interval_offsets = off.ctypes.data
        d.interval_filter = filt.ctypes.data if filt.size else None
        d.n_filters, d.n_lags = int(lags.shape[0]), int(lags.shape[1])
        d.filter_lags = lags.ctypes.data
        d.rcond_excise, d.rcond_fp64 = float(rcond_excise), float(rcond_fp64)
        d.fft_len, d.tiles_per_chunk = int(fft_len), int(tiles_per_chunk)
        if pix_pol is not None:
            if int(pix_pol.numel()) != n_t:
                raise ValueError("pix_pol must have one entry per sample")
            d.pix_pol = _dev_ptr(pix_pol, torch.int32, "pix_pol") if n_t else None
            d.n_pix_pol = int(n_pix_pol)
            if not n_t:  # the library reads no sample, but needs a non-NULL pointer to know the layout
                pix_pol = torch.zeros(1, dtype=torch.int32, device="cuda")
                d.pix_pol = _dev_ptr(pix_pol, torch.int32, "pix_pol")
        if extra_index is not None:
            if int(extra_index.numel()) != n_t:
                raise ValueError("extra_index must have one entry per sample")
            keep_extra = extra_index if n_t else torch.full((1,), -1, dtype=torch.int32, device="cuda")
            d.extra_index = _dev_ptr(keep_extra, torch.int32, "extra_index")
            d.n_extra = int(n_extra)
        keep_hwp = None
        if hwp is not None:
            ang, tau, grp, n_groups = hwp
            grp = np.ascontiguousarray(grp, dtype=np.int32)
            if int(ang.numel()) != n_t or int(tau.numel()) != n_t or grp.shape[0] != filt.shape[0]:
                raise ValueError("hwp angle and tau need one entry per sample, interval_group one per interval")
            if n_t:
                d.hwp_angle = _dev_ptr(ang, torch.float32, "hwp angle")
                d.hwp_tau = _dev_ptr(tau, torch.float32, "hwp tau")
            else:
                keep_hwp = torch.zeros(1, dtype=torch.float32, device="cuda")
                d.hwp_angle = d.hwp_tau = _dev_ptr(keep_hwp, torch.float32, "hwp")
            d.interval_hwp_group = grp.ctypes.data if grp.size else np.zeros(1, np.int32).ctypes.data
            d.n_hwp_groups = int(n_groups)
            keep_hwp = (keep_hwp, grp)
        if allreduce is not None:
            self._reduce = _reduce_callback(allreduce)
            d.allreduce = self._reduce[0]
        d.deterministic = 1 if deterministic else 0
        d.autotune = 1 if autotune else 0
        d.scatter_runs = int(scatter_runs)
        d.fft_split = int(fft_split)
        self._keep = (off, filt, lags, keep_hwp)
        self.multires = pix_pol is not None
        self._create(d, n_t, stream)

    def _create(self, d, n_t, stream):
        self._h = madmap_plan_create(d, stream)
        self.n_stokes = d.n_stokes
        self.n_samples = n_t
        self.stats = madmap_plan_get_stats(self._h)
        self.n_obs = self.stats["n_obs"]
        self.n_extra = self.stats["n_extra"]

    @classmethod
    def from_boresight(cls, boresight, bore_step, det_pointing, samples_per_det, width, height, polarised,
                       interval_offsets, interval_filter, filter_lags, rcond_excise=0.0, rcond_fp64=0.0, fft_len=0,
                       tiles_per_chunk=0, stream=None):
        """A plan whose pointing is expanded on the fly from compressed boresight pointing
        (no per-sample pointing is stored).  boresight: float32 CUDA tensor [n_bore, 4]
        (x, y, cos, sin per node, one node every bore_step detector samples);
        det_pointing: host [n_det, 4] (dx, dy, cos, sin); the grid is width x height pixels."""
        torch = _torch()
        self = cls.__new__(cls)
        self._h = None
        off = np.ascontiguousarray(interval_offsets, dtype=np.int64)
        filt = np.ascontiguousarray(interval_filter, dtype=np.int32)
        lags = np.ascontiguousarray(np.atleast_2d(filter_lags), dtype=np.float64)
        det = np.ascontiguousarray(det_pointing, dtype=np.float32).reshape(-1, 4)
        if boresight.dim() != 2 or boresight.shape[1] != 4:
            raise ValueError("boresight must be [n_bore, 4]")
        n_t = int(det.shape[0]) * int(samples_per_det)
        d = _lib.madmap_plan_desc()
        d.n_stokes = 3 if polarised else 1
        d.n_samples = n_t
        d.n_pix = int(width) * int(height)
        d.n_intervals = int(filt.shape[0])
        d.interval_offsets = off.ctypes.data
        d.interval_filter = filt.ctypes.data if filt.size else None
        d.n_filters, d.n_lags = int(lags.shape[0]), int(lags.shape[1])
        d.filter_lags = lags.ctypes.data
        d.rcond_excise, d.rcond_fp64 = float(rcond_excise), float(rcond_fp64)
        d.fft_len, d.tiles_per_chunk = int(fft_len), int(tiles_per_chunk)
        bore = boresight if boresight.numel() else torch.zeros((1, 4), dtype=torch.float32, device="cuda")
        d.boresight = _dev_ptr(bore, torch.float32, "boresight")
        d.n_bore = int(boresight.shape[0])
        d.bore_step = int(bore_step)
        d.det_pointing = det.ctypes.data
        d.n_det = int(det.shape[0])
        d.grid_width, d.grid_height = int(width), int(height)
        self._keep = (off, filt, lags, det)
        self.multires = False
        self._create(d, n_t, stream)
        return self

    def close(self):
        if self._h is not None:
            madmap_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def observed(self, stream=None):
        """(obs2glob int32, excised uint8) CUDA tensors over the observed (I) pixels."""
        torch = _torch()
        n = madmap_plan_observed(self._h)
        o = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        e = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
        madmap_plan_observed(self._h, o.data_ptr(), e.data_ptr(), stream)
        return o[:n], e[:n]

    def expand_pointing(self, stream=None):
        """(pix int32, cos2psi float32 or None, sin2psi float32 or None) CUDA tensors [n_samples]: the
        pointing a plan over compressed pointing computes for every sample."""
        torch = _torch()
        n = max(self.n_samples, 1)
        pix = torch.empty(n, dtype=torch.int32, device="cuda")
        c2 = torch.empty(n, dtype=torch.float32, device="cuda") if self.n_stokes == 3 else None
        s2 = torch.empty(n, dtype=torch.float32, device="cuda") if self.n_stokes == 3 else None
        madmap_plan_expand_pointing(self._h, pix.data_ptr(), c2.data_ptr() if c2 is not None else None,
                                    s2.data_ptr() if s2 is not None else None, stream)
        k = self.n_samples
        return pix[:k], (c2[:k] if c2 is not None else None), (s2[:k] if s2 is not None else None)

    def observed_pol(self, stream=None):
        """(obs2glob_pol int32, excised_pol uint8) CUDA tensors over the observed Q/U
        pixels of a multi-resolution plan (empty otherwise)."""
        torch = _torch()
        n = madmap_plan_observed_pol(self._h)
        o = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        e = torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")
        madmap_plan_observed_pol(self._h, o.data_ptr(), e.data_ptr(), stream)
        return o[:n], e[:n]

    def time_operator(self, precision="fp32", reps=10, stream=None):
        """Mean duration (ms) of one launch of each of the three operator kernels, and
        the launches of each per operator application."""
        return madmap_time_operator(self._h, _PREC[precision], reps, stream)

    def set_filters(self, filter_lags, stream=None):
        madmap_plan_set_filters(self._h, np.atleast_2d(filter_lags), stream)

    def _map_shape(self, n_rhs):
        return (n_rhs, self.n_obs, self.n_stokes)

    def apply_ATNA(self, x, precision="fp64", stream=None):
        torch = _torch()
        prec = _PREC[precision]
        dt = torch.float32 if prec == MADMAP_FP32 else torch.float64
        x = x.reshape(-1, self.n_obs, self.n_stokes)
        y = torch.empty_like(x)
        madmap_apply_ATNA(self._h, prec, x.shape[0], _dev_ptr(x, dt, "x"), y.data_ptr(), stream)
        return y

    def rhs(self, d, precision="fp64", stream=None):
        torch = _torch()
        prec = _PREC[precision]
        d = d.reshape(-1, self.n_samples)
        b = torch.empty(self._map_shape(d.shape[0]), dtype=torch.float32 if prec == MADMAP_FP32 else torch.float64,
                        device=d.device)
        madmap_rhs(self._h, prec, d.shape[0], _dev_ptr(d, torch.float32, "d"), b.data_ptr(), stream)
        return b

    def apply_ninv(self, y, precision="fp64", stream=None):
        torch = _torch()
        prec = _PREC[precision]
        dt = torch.float64 if prec == MADMAP_FP64 else torch.float32
        y = y.reshape(-1, self.n_samples)
        w = torch.empty_like(y)
        madmap_apply_ninv(self._h, prec, y.shape[0], _dev_ptr(y, dt, "y"), w.data_ptr(), stream)
        return w

    @staticmethod
    def _opts(precision, max_iter, rel_tol, max_outer, inner_rel_tol, use_graph, iters_per_sync, refine="df64",
              inner_restart=False, final_residual=False):
        o = _lib.madmap_solve_opts()
        o.max_iter, o.rel_tol, o.precision = int(max_iter), float(rel_tol), _PREC[precision]
        o.max_outer, o.inner_rel_tol = int(max_outer), float(inner_rel_tol)
        o.use_graph, o.iters_per_sync = (2 if use_graph is True else int(use_graph)), int(iters_per_sync)
        o.refine_precision = _PREC[refine]
        o.inner_restart = 1 if inner_restart else 0
        o.final_residual = 1 if final_residual else 0
        return o

    @staticmethod
    def _history(o, n_rhs, max_iter, want):
        """Host buffer for the residual history (max_iter + 1 entries per right-hand side)."""
        if not want:
            return None
        cap = min(int(max_iter), 4095) + 1
        h = np.zeros((n_rhs, cap))
        o.residual_history = h.ctypes.data
        o.history_capacity = cap
        return h

    @staticmethod
    def _info(i, hist=None, k=0):
        out = {f: getattr(i, f) for f, _ in i._fields_ if f != "pad_"}
        if hist is not None:
            out["history"] = hist[k, :i.history_len].copy()
        return out

    def solve_batched(self, d, precision="fp64", max_iter=50, rel_tol=1e-6, max_outer=10, inner_rel_tol=1e-4,
                      use_graph=True, iters_per_sync=8, out=None, stream=None, refine="df64", history=False,
                      inner_restart=False, final_residual=False):
        """Maps [n_rhs, n_obs, n_stokes] (float64) for d [n_rhs, n_samples], and per-rhs info dicts.
        refine ("df64" or "fp64"): arithmetic of the mixed solve's right-hand side and residuals.
        inner_restart: mixed refinement steps restart the float32 PCG instead of continuing it.
        final_residual: confirm every mixed stop with a full-precision residual (default: a continued
        PCG may stop on its recursive residual once a full-precision residual has replaced it).
        history: add each right-hand side's residual history (numpy) as info["history"]."""
        torch = _torch()
        d = d.reshape(-1, self.n_samples)
        n_rhs = d.shape[0]
        o = self._opts(precision, max_iter, rel_tol, max_outer, inner_rel_tol, use_graph, iters_per_sync, refine,
                       inner_restart, final_residual)
        hist = self._history(o, n_rhs, max_iter, history)
        m = out if out is not None else torch.empty((n_rhs, self.n_obs, self.n_stokes), dtype=torch.float64,
                                                    device="cuda")
        infos = madmap_solve_batched(self._h, n_rhs, _dev_ptr(d, torch.float32, "d") if d.numel() else None,
                                     _dev_ptr(m, torch.float64, "m") if m.numel() else None, o, stream)
        return m, [self._info(i, hist, k) for k, i in enumerate(infos)]

    def solve_backward(self, d, m, grad_m, want_d=True, want_lags=True, precision="mixed", max_iter=500,
                       rel_tol=1e-10, max_outer=20, inner_rel_tol=1e-4, use_graph=True, iters_per_sync=8,
                       stream=None, refine="df64"):
        """(dL/dd float32 [n_samples] or None, dL/dlags float64 [n_filters, n_lags] or None, info) for the
        map m of data d and grad_m = dL/dm, by one adjoint solve."""
        torch = _torch()
        o = self._opts(precision, max_iter, rel_tol, max_outer, inner_rel_tol, use_graph, iters_per_sync, refine)
        gd = torch.empty(self.n_samples, dtype=torch.float32, device="cuda") if want_d else None
        gl = (torch.empty((self.stats["n_filters"], self.stats["n_lags"]), dtype=torch.float64, device="cuda")
              if want_lags else None)
        info = madmap_solve_backward(self._h, _dev_ptr(d.reshape(-1), torch.float32, "d"),
                                     _dev_ptr(m, torch.float64, "m"), _dev_ptr(grad_m, torch.float64, "grad_m"),
                                     gd.data_ptr() if gd is not None else None,
                                     gl.data_ptr() if gl is not None else None, o, stream)
        return gd, gl, {k: getattr(info, k) for k, _ in info._fields_}

    def _checkpoints(self, o, checkpoint_every, on_checkpoint):
        if not checkpoint_every:
            return None
        cb = _CheckpointBuffers(self.n_obs, self.n_stokes, on_checkpoint)
        o.checkpoint_every = int(checkpoint_every)
        o.checkpoint = C.pointer(cb.c)
        o.on_checkpoint = cb.fn
        return cb

    def solve(self, d, precision="fp64", max_iter=50, rel_tol=1e-6, max_outer=10, inner_rel_tol=1e-4,
              use_graph=True, iters_per_sync=8, out=None, stream=None, refine="df64", checkpoint_every=0,
              on_checkpoint=None, history=False, inner_restart=False, final_residual=False):
        """Maximum-likelihood map [n_obs, n_stokes] (float64) and the solve info dict.
        refine ("df64" or "fp64"): arithmetic of the mixed solve's right-hand side and residuals.
        checkpoint_every > 0 (float64 solves): every that many iterations the solver state is
        passed to on_checkpoint(state dict); a true return stops the solve (status STOPPED).
        history: add the residual history after every iteration (numpy) as info["history"].
        inner_restart: mixed refinement steps restart the float32 PCG instead of continuing it.
        final_residual: confirm every mixed stop with a full-precision residual (default: a continued
        PCG may stop on its recursive residual once a full-precision residual has replaced it)."""
        torch = _torch()
        o = self._opts(precision, max_iter, rel_tol, max_outer, inner_rel_tol, use_graph, iters_per_sync, refine,
                       inner_restart, final_residual)
        hist = self._history(o, 1, max_iter, history)
        cb = self._checkpoints(o, checkpoint_every, on_checkpoint)
        m = out if out is not None else torch.empty((self.n_obs, self.n_stokes), dtype=torch.float64,
                                                    device="cuda")
        info = madmap_solve(self._h, _dev_ptr(d.reshape(-1), torch.float32, "d"), _dev_ptr(m, torch.float64, "m"),
                            o, stream)
        if cb is not None and cb.error is not None:
            raise cb.error
        return m, self._info(info, hist)

    def solve_resume(self, state, max_iter=50, rel_tol=1e-6, use_graph=True, iters_per_sync=8, out=None,
                     stream=None, checkpoint_every=0, on_checkpoint=None, history=False):
        """Continue a float64 solve from a checkpoint dict (as passed to on_checkpoint or read by
        load_checkpoint); returns the best map and the info dict of the whole solve."""
        torch = _torch()
        o = self._opts("fp64", max_iter, rel_tol, 1, 1e-4, use_graph, iters_per_sync, "fp64")
        hist = self._history(o, 1, max_iter, history)
        cb = self._checkpoints(o, checkpoint_every, on_checkpoint)
        c = _lib.madmap_checkpoint()
        keep = {}
        for k in _CKPT_MAPS:
            keep[k] = np.ascontiguousarray(state[k], dtype=np.float64).reshape(-1, self.n_stokes)
            setattr(c, k, keep[k].ctypes.data)
        for k in _CKPT_SCALARS:
            setattr(c, k, state[k])
        m = out if out is not None else torch.empty((self.n_obs, self.n_stokes), dtype=torch.float64,
                                                    device="cuda")
        info = madmap_solve_resume(self._h, c, _dev_ptr(m, torch.float64, "m"), o, stream)
        if cb is not None and cb.error is not None:
            raise cb.error
        return m, self._info(info, hist)


# ----------------------------------------------------------------- differentiable solve
def _per_filter(fn, n):
    """[fn(0), ..., fn(n-1)] on host threads (the library calls release the interpreter lock)."""
    if n < 2:
        return [fn(k) for k in range(n)]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=min(n, os.cpu_count() or 1)) as ex:
        return list(ex.map(fn, range(n)))


def _autograd_function():
    torch = _torch()

    class MadmapSolve(torch.autograd.Function):
        """m = MadmapSolve.apply(d, params, plan, fs, solve_kwargs)

        d: float32 CUDA tensor [n_samples]; params: float64 tensor [n_filters, 3]
        of (sigma, f_knee, alpha) per filter; plan: a Plan whose filters are
        rebuilt from params (madmap_noise_filter) before the solve.  The
        backward pass runs madmap_solve_backward (one adjoint solve) and the
        chain rule madmap_noise_filter_vjp; it returns gradients for d and params.
        """

        @staticmethod
        def forward(ctx, d, params, plan, fs, solve_kwargs):
            prm = params.detach().cpu().numpy().astype(np.float64)
            n_lags = plan.stats["n_lags"]
            lags = np.stack(_per_filter(lambda k: madmap_noise_filter(n_lags, fs, *prm[k]), prm.shape[0]))
            plan.set_filters(lags)
            kw = dict(solve_kwargs or {})
            m, info = plan.solve(d.detach().contiguous(), **kw)
            ctx.save_for_backward(d, m, params)
            ctx.plan, ctx.fs, ctx.kw = plan, fs, kw
            ctx.info = info
            return m

        @staticmethod
        def backward(ctx, grad_m):
            d, m, params = ctx.saved_tensors
            plan = ctx.plan
            bkw = {k: v for k, v in ctx.kw.items() if k in ("precision", "max_iter", "rel_tol", "max_outer",
                                                            "inner_rel_tol", "use_graph", "iters_per_sync")}
            gd, gl, _ = plan.solve_backward(d.detach().contiguous(), m.detach().contiguous(),
                                            grad_m.detach().contiguous().to(torch.float64),
                                            want_d=ctx.needs_input_grad[0], want_lags=ctx.needs_input_grad[1],
                                            **bkw)
            gp = None
            if ctx.needs_input_grad[1]:
                prm = params.detach().cpu().numpy().astype(np.float64)
                glh = gl.cpu().numpy()
                n_lags = plan.stats["n_lags"]
                out = np.stack(_per_filter(lambda k: madmap_noise_filter_vjp(n_lags, ctx.fs, *prm[k], glh[k]),
                                           prm.shape[0]))
                gp = torch.from_numpy(out).to(dtype=params.dtype, device=params.device)
            return (gd.view_as(d) if gd is not None else None), gp, None, None, None

    return MadmapSolve


def __getattr__(name):
    if name == "MadmapSolve":
        fn = _autograd_function()
        globals()["MadmapSolve"] = fn
        return fn
    raise AttributeError(name)
