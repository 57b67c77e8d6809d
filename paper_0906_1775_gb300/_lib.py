"""ctypes declarations of the libmadmap C ABI (include/madmap.h).

Argument marshalling only: every computation happens inside libmadmap.so.
Loading fails loudly when the library has not been built; there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes as C
import os

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmadmap.so")

MADMAP_OK = 0
MADMAP_WARN_MAXITER = 1
MADMAP_STOPPED = 2
MADMAP_ERR_INVALID_ARG = -1
MADMAP_ERR_CUDA = -2
MADMAP_ERR_OOM = -3
MADMAP_ERR_NOT_PD = -4
MADMAP_ERR_TIMEOUT = -5
MADMAP_ERR_INTERNAL = -6

MADMAP_FP64 = 0
MADMAP_MIXED = 1
MADMAP_FP32 = 2
MADMAP_DF64 = 3

STATUS_NAMES = {0: "OK", 1: "WARN_MAXITER", 2: "STOPPED", -1: "ERR_INVALID_ARG", -2: "ERR_CUDA", -3: "ERR_OOM",
                -4: "ERR_NOT_PD", -5: "ERR_TIMEOUT", -6: "ERR_INTERNAL"}


# madmap_reduce_fn: (buf, count, dtype, stream, user) -> 0 on success
REDUCE_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p)
MADMAP_REDUCE_F64, MADMAP_REDUCE_F32, MADMAP_REDUCE_I32 = 0, 1, 2
MADMAP_MAX_TUNED = 12


class madmap_plan_desc(C.Structure):
    _fields_ = [("n_stokes", C.c_int32), ("n_samples", C.c_int64), ("n_pix", C.c_int32),
                ("pix", C.c_void_p), ("psi", C.c_void_p), ("n_intervals", C.c_int32),
                ("interval_offsets", C.c_void_p), ("interval_filter", C.c_void_p),
                ("n_filters", C.c_int32), ("n_lags", C.c_int32), ("filter_lags", C.c_void_p),
                ("rcond_excise", C.c_double), ("rcond_fp64", C.c_double), ("fft_len", C.c_int32),
                ("tiles_per_chunk", C.c_int32), ("pix_pol", C.c_void_p), ("n_pix_pol", C.c_int32),
                ("boresight", C.c_void_p), ("n_bore", C.c_int32), ("bore_step", C.c_int32),
                ("det_pointing", C.c_void_p), ("n_det", C.c_int32), ("grid_width", C.c_int32),
                ("grid_height", C.c_int32), ("extra_index", C.c_void_p), ("n_extra", C.c_int32),
                ("hwp_angle", C.c_void_p), ("hwp_tau", C.c_void_p), ("interval_hwp_group", C.c_void_p),
                ("n_hwp_groups", C.c_int32), ("allreduce", REDUCE_FN), ("allreduce_user", C.c_void_p),
                ("deterministic", C.c_int32), ("autotune", C.c_int32), ("scatter_runs", C.c_int32),
                ("fft_split", C.c_int32)]


class madmap_plan_stats(C.Structure):
    _fields_ = [(n, C.c_int32) for n in ("n_obs", "n_excised", "n_fp64_pixels", "n_stokes", "fft_len", "n1",
                                         "n2", "n_segments", "n_tiles", "tiles_per_chunk", "n_lags",
                                         "n_filters")] + [("n_samples", C.c_int64), ("device_bytes", C.c_int64),
                                                          ("n_obs_pol", C.c_int32), ("n_excised_pol", C.c_int32),
                                                          ("n_extra", C.c_int32), ("n_excised_extra", C.c_int32),
                                                          ("n_hwp_params", C.c_int32), ("n_excised_hwp", C.c_int32),
                                                          ("n_map_replicas", C.c_int32),
                                                          ("deterministic", C.c_int32), ("sharded", C.c_int32),
                                                          ("n_tuned", C.c_int32), ("tuned_fft_len", C.c_int32 * MADMAP_MAX_TUNED),
                                                          ("tuned_tiles_per_chunk", C.c_int32 * MADMAP_MAX_TUNED),
                                                          ("tuned_ms", C.c_float * MADMAP_MAX_TUNED),
                                                          ("tuned_runs", C.c_int32 * MADMAP_MAX_TUNED),
                                                          ("tuned_n2", C.c_int32 * MADMAP_MAX_TUNED),
                                                          ("scatter_runs", C.c_int32),
                                                          ("repeat_frac", C.c_double)]


class madmap_checkpoint(C.Structure):
    _fields_ = [("n_obs", C.c_int32), ("n_stokes", C.c_int32), ("iters", C.c_int32), ("best_iter", C.c_int32),
                ("rz", C.c_double), ("bnorm", C.c_double), ("rel_res", C.c_double), ("best_rel_res", C.c_double),
                ("x", C.c_void_p), ("r", C.c_void_p), ("z", C.c_void_p), ("p", C.c_void_p), ("x_best", C.c_void_p)]


CHECKPOINT_FN = C.CFUNCTYPE(C.c_int32, C.POINTER(madmap_checkpoint), C.c_void_p)


class madmap_solve_opts(C.Structure):
    _fields_ = [("max_iter", C.c_int32), ("rel_tol", C.c_double), ("precision", C.c_int32),
                ("max_outer", C.c_int32), ("inner_rel_tol", C.c_double), ("use_graph", C.c_int32),
                ("iters_per_sync", C.c_int32),
                ("refine_precision", C.c_int32),
                ("checkpoint_every", C.c_int32), ("checkpoint", C.POINTER(madmap_checkpoint)),
                ("on_checkpoint", CHECKPOINT_FN), ("checkpoint_user", C.c_void_p),
                ("residual_history", C.c_void_p), ("history_capacity", C.c_int32),
                ("inner_restart", C.c_int32), ("final_residual", C.c_int32)]


class madmap_solve_info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("outer_iters", C.c_int32),
                ("best_iter", C.c_int32), ("fp64_applies", C.c_int32), ("fp32_applies", C.c_int32),
                ("final_rel_res", C.c_double), ("best_rel_res", C.c_double), ("t_rhs_ms", C.c_double),
                ("t_solve_ms", C.c_double), ("history_len", C.c_int32), ("pad_", C.c_int32),
                ("t_pcg_ms", C.c_double), ("t_refine_ms", C.c_double)]


# (name, restype, argtypes) of every entry point declared in include/madmap.h
PROTOTYPES = [
    ("madmap_plan_create", C.c_int, [C.POINTER(madmap_plan_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("madmap_plan_destroy", C.c_int, [C.c_void_p]),
    ("madmap_partition_intervals", C.c_int, [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]),
    ("madmap_plan_get_stats", C.c_int, [C.c_void_p, C.POINTER(madmap_plan_stats)]),
    ("madmap_plan_observed", C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_void_p, C.c_void_p, C.c_void_p]),
    ("madmap_plan_observed_pol", C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.c_void_p, C.c_void_p, C.c_void_p]),
    ("madmap_plan_set_filters", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("madmap_plan_expand_pointing", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("madmap_apply_ATNA", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("madmap_rhs", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("madmap_apply_ninv", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("madmap_solve_opts_default", None, [C.POINTER(madmap_solve_opts)]),
    ("madmap_solve", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(madmap_solve_opts),
                               C.POINTER(madmap_solve_info), C.c_void_p]),
    ("madmap_solve_resume", C.c_int, [C.c_void_p, C.POINTER(madmap_checkpoint), C.c_void_p,
                                      C.POINTER(madmap_solve_opts), C.POINTER(madmap_solve_info), C.c_void_p]),
    ("madmap_solve_batched", C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.POINTER(madmap_solve_opts),
                                       C.c_void_p, C.c_void_p]),
    ("madmap_solve_backward", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.POINTER(madmap_solve_opts), C.POINTER(madmap_solve_info), C.c_void_p]),
    ("madmap_noise_filter_vjp", C.c_int, [C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                          C.c_void_p]),
    ("madmap_noise_filter", C.c_int, [C.c_int32, C.c_double, C.c_double, C.c_double, C.c_double, C.c_void_p,
                                      C.c_void_p]),
    ("madmap_paper_fft_length", C.c_int64, [C.c_int64, C.c_int64]),
    ("madmap_apply_ninv_noalloc", C.c_int, [C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                            C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("madmap_kernel_launch_count", C.c_int64, []),
    ("madmap_polarisation_weights", C.c_int, [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                              C.c_void_p]),
    ("madmap_time_operator", C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("madmap_last_error", C.c_char_p, []),
    ("madmap_version", C.c_char_p, []),
]

_lib = None


def load() -> C.CDLL:
    """Load libmadmap.so (built in-tree by paper_0906_1775_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmadmap.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
    lib = C.CDLL(LIB_PATH)
    for name, res, args in PROTOTYPES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MadmapError(RuntimeError):
    def __init__(self, status: int, where: str, message: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {message}")


def check(status: int, where: str, allow_warn: bool = False) -> int:
    if status == MADMAP_OK or (allow_warn and status in (MADMAP_WARN_MAXITER, MADMAP_STOPPED)):
        return status
    msg = load().madmap_last_error().decode(errors="replace")
    raise MadmapError(status, where, msg)
