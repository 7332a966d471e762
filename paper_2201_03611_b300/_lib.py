"""ctypes binding of libshine.so: the C ABI of include/shine.h, with the same names.

Marshalling only: every step of the pipeline runs in the library's CUDA kernels. If the
library is missing this module raises ImportError; there is no fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# SHINE_LIBRARY selects another build of the library (the index-checking libshine_debug.so).
LIB_PATH = os.environ.get("SHINE_LIBRARY") or os.path.join(_HERE, "libshine.so")
DEBUG_LIB_PATH = os.path.join(_HERE, "libshine_debug.so")

SHINE_OK, SHINE_ERR_INVALID_ARG, SHINE_ERR_ALIGNMENT, SHINE_ERR_WORKSPACE, SHINE_ERR_UNSUPPORTED, \
    SHINE_ERR_CUDA = range(6)
SHINE_F32, SHINE_BF16, SHINE_F16 = 0, 1, 2
SHINE_VALID, SHINE_CLAMP = 0, 1
SHINE_MODE_FWD, SHINE_MODE_FWD_BWD = 1, 3
SHINE_ORDER_LONGEST_FIRST, SHINE_ORDER_IMAGE, SHINE_ORDER_LARGEST_IMAGE_FIRST = 0, 1, 2


class ShineError(RuntimeError):
    def __init__(self, status: int, what: str, cuda_error: int = 0):
        msg = f"{what}: {status_string(status)} (status {status})"
        if status == SHINE_ERR_CUDA:
            msg += f", cudaError {cuda_error}"
        super().__init__(msg)
        self.status = status


class ImageDesc(ctypes.Structure):
    """shine_image_desc."""
    _fields_ = [("img", ctypes.c_void_p), ("out", ctypes.c_void_p), ("grad_out", ctypes.c_void_p),
                ("grad_img", ctypes.c_void_p), ("H", ctypes.c_int64), ("W", ctypes.c_int64),
                ("img_pitch", ctypes.c_int64), ("out_pitch", ctypes.c_int64),
                ("gout_pitch", ctypes.c_int64), ("gimg_pitch", ctypes.c_int64)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_2201_03611_b300.build` "
                          f"(nvcc for sm_103a). The pipeline has no CPU or library fallback.")
    L = ctypes.CDLL(LIB_PATH)
    p, i64, i32, f, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_size_t
    st = ctypes.c_int
    sigs = {
        "shine_output_shape": (st, [i64, i64, f, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "shine_pipeline_fwd": (st, [p, i64, i64, i64, f, f, p, p, p, p, i64, f, p]),
        "shine_pipeline_fwd_bwd": (st, [p, i64, i64, i64, f, f, p, p, p, p, i64, p, i64, p, i64, p, p, p, p,
                                        sz, p]),
        "shine_pipeline_bwd_workspace": (st, [i64, i64, f, ctypes.POINTER(sz)]),
        "shine_pipeline_bwd": (st, [p, i64, i64, i64, f, f, p, p, p, p, i64, f, p, i64, p, p, p, p, sz, p]),
        "shine_pipeline_bwd_noalloc": (st, [p, i64, i64, i64, f, f, p, p, p, p, i64, f, p, i64, p, p, p, p]),
        "shine_pipeline_host_workspace": (st, [i64, i64, f, i32, ctypes.POINTER(sz)]),
        "shine_pipeline_host": (st, [p, p, p, p, i64, i64, f, f, p, p, p, p, p, p, p, p, p, sz, i32, p]),
        "shine_mv": (st, [p, i64, i64, i64, f, p, p, p]),
        "shine_wait_status": (st, [ctypes.POINTER(f), f]),
        "shine_debug_bounds_status": (st, [ctypes.POINTER(f), ctypes.POINTER(ctypes.c_uint), f]),
        "shine_partition": (st, [i64, i64, i64, i64, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "shine_selftest_bounded_wait": (st, [i32, p, p]),
        "shine_iterate_sum": (st, [p, i64, i32, i32, p, p]),
        "shine_iterate_reduce": (st, [p, i64, i32, i32, f, p, p]),
        "shine_iterate_stencil": (st, [p, i64, i64, i64, p, i32, p, i64, p]),
        "shine_stencil2d": (st, [p, i64, i64, i64, f, f, i32, p, p, p, p, i64, f, p]),
        "shine_harris_window": (st, [p, i64, i64, i64, f, p, p, p, i32, p, p, p, i64, f, p]),
        "shine_corners": (st, [p, i64, i64, i64, f, f, p, p, p, ctypes.c_float, p, i64, p, i64, f, p]),
        "shine_plan_create": (st, [ctypes.POINTER(i64), i32, f, f, i32, ctypes.c_char_p, ctypes.POINTER(p)]),
        "shine_plan_workspace": (st, [p, ctypes.POINTER(sz)]),
        "shine_plan_tile_rows": (st, [p, i32, ctypes.POINTER(i32)]),
        "shine_plan_schedule": (st, [p, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                     ctypes.POINTER(i32)]),
        "shine_pipeline_batched": (st, [p, p, p, p, p, p, p, p, p, sz, p]),
        "shine_plan_destroy": (None, [p]),
        "shine_status_string": (ctypes.c_char_p, [f]),
        "shine_tune_key": (ctypes.c_int, [ctypes.c_char_p, sz]),
        "shine_last_cuda_error": (ctypes.c_int, []),
        "shine_workspace_status": (st, [p, ctypes.POINTER(ctypes.c_int)]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def status_string(status: int) -> str:
    return lib().shine_status_string(status).decode()


def check(status: int, what: str) -> None:
    if status != SHINE_OK:
        raise ShineError(status, what, lib().shine_last_cuda_error() if status == SHINE_ERR_CUDA else 0)
