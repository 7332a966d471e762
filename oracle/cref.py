"""Loader and NumPy-facing wrappers of the FP64 C reference ``harris_ref.c``.

ORACLE -- test infrastructure only (see ``oracle/__init__.py``). The library is compiled here
with gcc (``-O2 -fopenmp -ffp-contract=off``: no fused multiply-adds, so each FP64 operation
rounds once, as written) into ``oracle/_build/``. It never touches a GPU.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "harris_ref.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libharris_ref.so")
_lib = None

VALID, CLAMP = 0, 1
_BORDERS = {"valid": VALID, "clamp": CLAMP, VALID: VALID, CLAMP: CLAMP}


def build(force: bool = False) -> str:
    """Compile the reference library if it is missing or older than its source."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared",
                        "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        p, i64, d, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.oracle_harris_forward.argtypes = [p, i64, i64, i, d, p, p, p, i]
        L.oracle_harris_backward.argtypes = [p, p, i64, i64, i, d, p, p, p, p, p, p, p, i]
        L.oracle_harris_forward_points.argtypes = [p, i64, i64, i, d, p, p, p, i64, p, i]
        L.oracle_harris_backward_points.argtypes = [p, p, i64, i64, i, d, p, p, p, i64, p, i]
        L.oracle_harris_param_grads.argtypes = [p, p, i64, i64, i, d, p, p, p, p, p, i]
        for f in (L.oracle_harris_forward, L.oracle_harris_backward, L.oracle_harris_forward_points,
                  L.oracle_harris_backward_points, L.oracle_harris_param_grads):
            f.restype = ctypes.c_int
        L.oracle_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    """Exact FP64 image of the stored values (bf16, fp16 and f32 all embed exactly)."""
    if hasattr(a, "detach"):
        a = a.detach().cpu().double().numpy()
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def out_shape(h: int, w: int, border) -> tuple[int, int]:
    return (h, w) if _BORDERS[border] == CLAMP else (h - 4, w - 4)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"{what}: oracle returned {rc}")


def forward(img, kappa, wx, wy, border, nthreads: int = 0) -> np.ndarray:
    """R (FP64) of an H x W x 3 image."""
    x = _f64(img)
    h, w = x.shape[0], x.shape[1]
    b = _BORDERS[border]
    ho, wo = out_shape(h, w, b)
    out = np.empty((max(ho, 0), max(wo, 0)), np.float64)
    wxd, wyd = _f64(wx).reshape(9), _f64(wy).reshape(9)
    _check(lib().oracle_harris_forward(_ptr(x), h, w, b, float(kappa), _ptr(wxd), _ptr(wyd),
                                       _ptr(out), nthreads), "forward")
    return out


def backward(img, g, kappa, wx, wy, border, nthreads: int = 0, with_abs: bool = False):
    """(d img [H,W,3], d kappa, d Wx [3,3], d Wy [3,3]) in FP64 for L = sum(g * R).

    with_abs: also return the sum of |term| of each parameter cotangent's sum, as
    (abs kappa, abs Wx [3,3], abs Wy [3,3])."""
    x, gg = _f64(img), _f64(g)
    h, w = x.shape[0], x.shape[1]
    b = _BORDERS[border]
    if gg.shape != out_shape(h, w, b):
        raise ValueError(f"cotangent shape {gg.shape} != output shape {out_shape(h, w, b)}")
    gimg = np.empty((h, w, 3), np.float64)
    gk = np.zeros(1, np.float64)
    gwx, gwy = np.zeros(9, np.float64), np.zeros(9, np.float64)
    wxd, wyd = _f64(wx).reshape(9), _f64(wy).reshape(9)
    absp = np.zeros(19, np.float64)
    _check(lib().oracle_harris_backward(_ptr(x), _ptr(gg), h, w, b, float(kappa), _ptr(wxd),
                                        _ptr(wyd), _ptr(gimg), _ptr(gk), _ptr(gwx), _ptr(gwy),
                                        _ptr(absp), nthreads), "backward")
    out = (gimg, float(gk[0]), gwx.reshape(3, 3), gwy.reshape(3, 3))
    if with_abs:
        return out + ((float(absp[0]), absp[1:10].reshape(3, 3), absp[10:19].reshape(3, 3)),)
    return out


def forward_points(img, kappa, wx, wy, border, pts, nthreads: int = 0) -> np.ndarray:
    """R at output positions pts (n x 2 int64: row, column)."""
    x = _f64(img)
    h, w = x.shape[0], x.shape[1]
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.int64).reshape(-1, 2))
    out = np.empty(p.shape[0], np.float64)
    wxd, wyd = _f64(wx).reshape(9), _f64(wy).reshape(9)
    _check(lib().oracle_harris_forward_points(_ptr(x), h, w, _BORDERS[border], float(kappa),
                                              _ptr(wxd), _ptr(wyd), _ptr(p), p.shape[0],
                                              _ptr(out), nthreads), "forward_points")
    return out


def backward_points(img, g, kappa, wx, wy, border, pts, nthreads: int = 0) -> np.ndarray:
    """d img (n x 3) at image positions pts (n x 2 int64: row, column)."""
    x, gg = _f64(img), _f64(g)
    h, w = x.shape[0], x.shape[1]
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.int64).reshape(-1, 2))
    out = np.empty((p.shape[0], 3), np.float64)
    wxd, wyd = _f64(wx).reshape(9), _f64(wy).reshape(9)
    _check(lib().oracle_harris_backward_points(_ptr(x), _ptr(gg), h, w, _BORDERS[border],
                                               float(kappa), _ptr(wxd), _ptr(wyd), _ptr(p),
                                               p.shape[0], _ptr(out), nthreads), "backward_points")
    return out


def param_grads(img, g, kappa, wx, wy, border, nthreads: int = 0):
    """(d kappa, d Wx, d Wy) as a sum of per-output chain-rule contributions (any image size)."""
    x, gg = _f64(img), _f64(g)
    h, w = x.shape[0], x.shape[1]
    gk = np.zeros(1, np.float64)
    gwx, gwy = np.zeros(9, np.float64), np.zeros(9, np.float64)
    wxd, wyd = _f64(wx).reshape(9), _f64(wy).reshape(9)
    _check(lib().oracle_harris_param_grads(_ptr(x), _ptr(gg), h, w, _BORDERS[border], float(kappa),
                                           _ptr(wxd), _ptr(wyd), _ptr(gk), _ptr(gwx), _ptr(gwy),
                                           nthreads), "param_grads")
    return float(gk[0]), gwx.reshape(3, 3), gwy.reshape(3, 3)


def num_threads() -> int:
    return int(lib().oracle_num_threads())
