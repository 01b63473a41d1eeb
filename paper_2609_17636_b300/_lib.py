"""ctypes binding of libivis.so (the C ABI declared in include/ivis.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. There is no fallback: if the library is missing or cannot be loaded, import
fails with an error that says so.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libivis.so")

IVIS_FP64 = 0
IVIS_FP32 = 1
IVIS_PROJ = {"SIN": 0, "TAN": 1, "ARC": 2}

STATUS = {0: "IVIS_OK", 1: "IVIS_ERR_ARG", 2: "IVIS_ERR_STATE", 3: "IVIS_ERR_OOM",
          4: "IVIS_ERR_CUDA", 5: "IVIS_ERR_TIMEOUT", 6: "IVIS_ERR_NONFINITE",
          7: "IVIS_ERR_LINESEARCH"}

# Every entry point include/ivis.h declares.
EXPORTS = ["ivis_plan", "ivis_set_pointing", "ivis_set_pointing_grid", "ivis_set_vis", "ivis_set_sd", "ivis_prepare",
           "ivis_cost_grad", "ivis_cost_grad_async", "ivis_get_stream", "ivis_cost_grad_host", "ivis_predict", "ivis_sd_predict",
           "ivis_solve", "ivis_get_nufft_params", "ivis_profile", "ivis_stage_times",
           "ivis_launches_per_eval", "ivis_sd_predict_noalloc", "ivis_destroy", "ivis_last_error",
           "ivis_dirty_image", "ivis_solve_target", "ivis_tuning", "ivis_unet_create", "ivis_unet_num_params", "ivis_unet_set_params",
           "ivis_unet_get_params", "ivis_unet_forward", "ivis_unet_backward", "ivis_unet_get_grads",
           "ivis_unet_adam_step", "ivis_unet_use_tcgen05", "ivis_unet_destroy",
           "ivis_unet_last_error", "ivis_feather", "ivis_rayleigh_jeans", "ivis_unet_warm_start",
           "ivis_unet_planes", "ivis_reproject_grid"]


class IvisError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("nchan", ctypes.c_int), ("npoint", ctypes.c_int),
                ("nb", ctypes.c_int), ("cell_rad", ctypes.c_double), ("precision", ctypes.c_int),
                ("nufft_tol", ctypes.c_double), ("kernel_width", ctypes.c_int),
                ("lambda_r", ctypes.c_double), ("lambda_s", ctypes.c_double),
                ("positivity", ctypes.c_int), ("serial_pairs", ctypes.c_int),
                ("autotune", ctypes.c_int), ("toeplitz", ctypes.c_int), ("wterm", ctypes.c_int),
                ("grid_tile", ctypes.c_int),
                ("grid_kernel", ctypes.c_int)]


class SolveReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("evaluations", ctypes.c_int),
                ("f", ctypes.c_double), ("pg_inf", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int)]


_LIB = None


def load(path: str = LIB_PATH):
    """Load libivis.so; raise if it is absent (no CPU fallback exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise ImportError(f"libivis.so not found at {path}: build it with "
                          "`python -m paper_2609_17636_b300.build` (nvcc, sm_103a)")
    L = ctypes.CDLL(path)
    vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    dp = ctypes.POINTER(ctypes.c_double)
    L.ivis_plan.argtypes = [ctypes.POINTER(Config), vp, ctypes.POINTER(vp)]
    L.ivis_set_pointing.argtypes = [vp, i, i, i, vp]
    L.ivis_set_vis.argtypes = [vp, i, i, i64, vp, vp, vp]
    L.ivis_set_pointing_grid.argtypes = [vp, i, vp]
    L.ivis_set_sd.argtypes = [vp, i, vp, d, d]
    L.ivis_prepare.argtypes = [vp]
    L.ivis_cost_grad.argtypes = [vp, vp, dp, vp, dp]
    L.ivis_cost_grad_host.argtypes = [vp, vp, dp, vp, dp]
    L.ivis_cost_grad_async.argtypes = [vp, vp, vp, vp]
    L.ivis_get_stream.argtypes = [vp, ctypes.POINTER(vp)]
    L.ivis_predict.argtypes = [vp, vp, i, i, vp]
    L.ivis_sd_predict.argtypes = [vp, vp, vp]
    L.ivis_solve.argtypes = [vp, vp, i, i, d, d, ctypes.POINTER(SolveReport)]
    L.ivis_get_nufft_params.argtypes = [vp, ctypes.POINTER(i), dp, ctypes.POINTER(i)]
    L.ivis_profile.argtypes = [vp, i]
    L.ivis_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_char_p), dp, i, ctypes.POINTER(i)]
    L.ivis_launches_per_eval.argtypes = [vp, ctypes.POINTER(i)]
    L.ivis_sd_predict_noalloc.argtypes = [vp, i, i, d, vp, vp]
    L.ivis_destroy.argtypes = [vp]
    L.ivis_last_error.argtypes = [vp]
    L.ivis_last_error.restype = ctypes.c_char_p
    L.ivis_dirty_image.argtypes = [vp, vp, vp]
    L.ivis_tuning.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(ctypes.c_char_p)]
    L.ivis_solve_target.argtypes = [vp, vp, i, i, d, d, d, ctypes.POINTER(SolveReport)]
    L.ivis_unet_create.argtypes = [i, i, i, vp, ctypes.POINTER(vp)]
    L.ivis_unet_num_params.argtypes = [vp, ctypes.POINTER(i64)]
    L.ivis_unet_set_params.argtypes = [vp, vp]
    L.ivis_unet_get_params.argtypes = [vp, vp]
    L.ivis_unet_forward.argtypes = [vp, vp, vp, i, i, i]
    L.ivis_unet_warm_start.argtypes = [vp, vp, vp, i, i, i, d, d, d, vp]
    L.ivis_unet_planes.argtypes = [vp, vp, i, i64, d, d, vp, vp]
    L.ivis_unet_backward.argtypes = [vp, vp, vp, i, i, i, dp]
    L.ivis_unet_get_grads.argtypes = [vp, vp]
    L.ivis_unet_adam_step.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    L.ivis_unet_use_tcgen05.argtypes = [vp, i]
    L.ivis_unet_destroy.argtypes = [vp]
    L.ivis_unet_last_error.argtypes = [vp]
    L.ivis_unet_last_error.restype = ctypes.c_char_p
    L.ivis_feather.argtypes = [vp, vp, vp, d, d, vp]
    L.ivis_rayleigh_jeans.argtypes = [d]
    L.ivis_reproject_grid.argtypes = [i, d, d, d, d, d, d, d, i, vp]
    L.ivis_rayleigh_jeans.restype = d
    for name in EXPORTS:
        if name not in ("ivis_last_error", "ivis_unet_last_error", "ivis_rayleigh_jeans"):
            getattr(L, name).restype = ctypes.c_int
    _LIB = L
    return L
