"""ctypes binding of ``include/s3cmtf.h`` (argument marshalling only).

Every name here is the C-ABI name.  The library is the in-tree ``_build/libs3cmtf.so``;
loading fails loudly when it is missing or cannot be loaded -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

S3_OK, S3_ERR_ARG, S3_ERR_INDEX, S3_ERR_OOM, S3_ERR_CUDA, S3_ERR_DIVERGED, S3_ERR_STATE = (
    0, -1, -2, -3, -4, -5, -6)
S3_MINIBATCH, S3_HOGWILD = 0, 1
S3_FP32, S3_BF16 = 0, 1
S3_ROW_SUM, S3_ROW_MEAN = 0, 1

STATUS_NAMES = {0: "S3_OK", -1: "S3_ERR_ARG", -2: "S3_ERR_INDEX", -3: "S3_ERR_OOM",
                -4: "S3_ERR_CUDA", -5: "S3_ERR_DIVERGED", -6: "S3_ERR_STATE"}

# every function declared in include/s3cmtf.h
EXPORTS = ("s3_init", "s3_epoch", "s3_loss", "s3_rmse", "s3_set_test", "s3_predict",
           "s3_gradient", "s3_get_params", "s3_set_params", "s3_get_epoch", "s3_set_epoch",
           "s3_update_values", "s3_info", "s3_hog_config", "s3_profile", "s3_profile_read",
           "s3_rmse_noalloc", "s3_finalize_qr", "s3_measure_fp32_peak", "s3_set_counts",
           "s3_apply_gradient",
           "s3_last_error", "s3_destroy")
S3_K_ALL, S3_K_TENSOR_HOG, S3_K_TENSOR_MB, S3_K_TENSOR_GRAD, S3_K_TENSOR_FWD = -1, 0, 1, 2, 3


class s3_coo_tensor(C.Structure):
    _fields_ = [("n_modes", C.c_int), ("dims", C.POINTER(C.c_int64)), ("nnz", C.c_int64),
                ("idx", C.POINTER(C.c_void_p)), ("val", C.c_void_p)]


class s3_coo_matrix(C.Structure):
    _fields_ = [("coupled_mode", C.c_int), ("rows", C.c_int64), ("cols", C.c_int64),
                ("nnz", C.c_int64), ("r", C.c_void_p), ("c", C.c_void_p), ("val", C.c_void_p)]


class s3_hparams(C.Structure):
    _fields_ = [("lr0", C.c_float), ("mu", C.c_float), ("lambda_reg", C.c_float),
                ("lambda_m", C.c_float), ("batch", C.c_int), ("core_scale", C.c_float),
                ("row_rule", C.c_int), ("hog_tile", C.c_int), ("hog_staleness", C.c_float),
                ("hog_ctas", C.c_int), ("mb_ctas", C.c_int), ("cp", C.c_int), ("nonneg", C.c_int),
                ("grad_chunk", C.c_int), ("hog_core_sync", C.c_int), ("wait_limit_us", C.c_int),
                ("device_bytes_cap", C.c_int64)]


class S3Error(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libs3cmtf.so (building it with nvcc first if it is absent or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and not _build.up_to_date():
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing; run "
                               "paper_1708_08640_gb300.build.build() (needs nvcc)")
        lib = C.CDLL(path)
        vp, pp = C.c_void_p, C.POINTER(C.c_void_p)
        lib.s3_init.argtypes = [C.POINTER(vp), C.POINTER(s3_coo_tensor), C.POINTER(s3_coo_matrix),
                                C.c_int, C.POINTER(C.c_int), C.POINTER(s3_hparams), C.c_uint64,
                                vp, C.c_int, vp]
        lib.s3_epoch.argtypes = [vp, C.c_int, C.c_int]
        lib.s3_loss.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.s3_rmse.argtypes = [vp, C.POINTER(s3_coo_tensor), C.c_int, C.POINTER(C.c_double)]
        lib.s3_set_test.argtypes = [vp, C.POINTER(s3_coo_tensor), C.c_int]
        lib.s3_predict.argtypes = [vp, pp, C.c_int64, vp]
        lib.s3_gradient.argtypes = [vp, vp, vp, pp, pp]
        lib.s3_get_params.argtypes = [vp, vp, pp, pp]
        lib.s3_set_params.argtypes = [vp, vp, pp, pp]
        lib.s3_get_epoch.argtypes = [vp, C.POINTER(C.c_int64)]
        lib.s3_set_epoch.argtypes = [vp, C.c_int64]
        lib.s3_update_values.argtypes = [vp, vp, pp]
        lib.s3_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.s3_finalize_qr.argtypes = [vp]
        lib.s3_hog_config.argtypes = [vp, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.s3_profile.argtypes = [vp, C.c_int]
        lib.s3_profile_read.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int64),
                                        C.POINTER(C.c_int64)]
        lib.s3_rmse_noalloc.argtypes = [vp, pp, vp, C.c_int64, C.POINTER(C.c_double)]
        lib.s3_measure_fp32_peak.argtypes = [C.POINTER(C.c_double)] * 3
        lib.s3_set_counts.argtypes = [vp, pp, C.c_int64]
        lib.s3_apply_gradient.argtypes = [vp, vp, pp, pp]
        lib.s3_last_error.argtypes = [vp]
        lib.s3_last_error.restype = C.c_char_p
        lib.s3_destroy.argtypes = [vp]
        lib.s3_destroy.restype = None
        for name in EXPORTS:
            if name not in ("s3_last_error", "s3_destroy"):
                getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


def check(lib, ctx, status):
    if status != S3_OK:
        msg = lib.s3_last_error(ctx) if ctx else b""
        raise S3Error(status, (msg or b"").decode(errors="replace"))
    return status


def ptr_array(ptrs):
    arr = (C.c_void_p * max(1, len(ptrs)))()
    for k, p in enumerate(ptrs):
        arr[k] = p
    return arr
