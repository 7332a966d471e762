"""Torch-facing calls of the fused Harris pipeline (device memory and streams from torch;
every computation in libshine's CUDA kernels).

Images are (H, W, 3) CUDA tensors with channel stride 1 and pixel stride 3 (any row stride
>= 3W); response maps and cotangents are (H_out, W_out) with column stride 1. kappa is a
CUDA float32 tensor with one element; wx, wy are (3, 3) CUDA float32 tensors.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L

_DT = {torch.float32: L.SHINE_F32, torch.bfloat16: L.SHINE_BF16, torch.float16: L.SHINE_F16}
_BORDER = {"valid": L.SHINE_VALID, "clamp": L.SHINE_CLAMP}


def dtype_code(dt: torch.dtype) -> int:
    if dt not in _DT:
        raise TypeError(f"unsupported storage dtype {dt}; use float32, bfloat16 or float16")
    return _DT[dt]


def border_code(border: str) -> int:
    if border not in _BORDER:
        raise ValueError(f"border must be 'valid' or 'clamp', not {border!r}")
    return _BORDER[border]


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(dev: torch.device) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def _check_img(img: torch.Tensor) -> None:
    if not img.is_cuda or img.dim() != 3 or img.shape[2] != 3:
        raise ValueError("img must be a CUDA tensor of shape (H, W, 3)")
    if img.stride(2) != 1 or img.stride(1) != 3:
        raise ValueError("img must have channel stride 1 and pixel stride 3 (rows may be padded)")


def _check_map(t: torch.Tensor, shape, name: str) -> None:
    if not t.is_cuda or tuple(t.shape) != tuple(shape) or (t.shape[1] > 1 and t.stride(1) != 1):
        raise ValueError(f"{name} must be a CUDA tensor of shape {tuple(shape)} with column stride 1")


def _param(t, name: str, numel: int) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous() \
            or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor with {numel} elements")
    return t


def output_shape(h: int, w: int, border: str) -> tuple[int, int]:
    ho, wo = ctypes.c_int64(), ctypes.c_int64()
    L.check(L.lib().shine_output_shape(h, w, border_code(border), ctypes.byref(ho), ctypes.byref(wo)),
            "shine_output_shape")
    return ho.value, wo.value


def bwd_workspace_bytes(h: int, w: int, border: str) -> int:
    n = ctypes.c_size_t()
    L.check(L.lib().shine_pipeline_bwd_workspace(h, w, border_code(border), ctypes.byref(n)),
            "shine_pipeline_bwd_workspace")
    return n.value


def workspace_failed(workspace: torch.Tensor) -> bool:
    """True when the last backward pass on this workspace gave up a bounded wait (results
    invalid). Synchronises with the device."""
    f = ctypes.c_int()
    L.check(L.lib().shine_workspace_status(_ptr(workspace), ctypes.byref(f)), "shine_workspace_status")
    return bool(f.value)


def wait_failed(clear: bool = True) -> bool:
    """True when a bounded wait of a forward, corner or window call on the current GPU gave up
    since the last clear (those results are invalid). Synchronises with the device."""
    f = ctypes.c_int()
    L.check(L.lib().shine_wait_status(ctypes.byref(f), 1 if clear else 0), "shine_wait_status")
    return bool(f.value)


def _row_pitch(t: torch.Tensor) -> int:
    return t.stride(0)


def pipeline_fwd(img, kappa, wx, wy, border: str = "clamp", out_dtype=None, out=None) -> torch.Tensor:
    """R = fused Harris response (shine_pipeline_fwd)."""
    _check_img(img)
    _param(kappa, "kappa", 1); _param(wx, "wx", 9); _param(wy, "wy", 9)
    h, w = img.shape[0], img.shape[1]
    ho, wo = output_shape(h, w, border)
    odt = img.dtype if out_dtype is None else out_dtype
    if out is None:
        out = torch.empty(ho, wo, device=img.device, dtype=odt)
    _check_map(out, (ho, wo), "out")
    L.check(L.lib().shine_pipeline_fwd(_ptr(img), h, w, _row_pitch(img), dtype_code(img.dtype), border_code(border),
                                       _ptr(kappa), _ptr(wx), _ptr(wy), _ptr(out), _row_pitch(out),
                                       dtype_code(out.dtype), _stream(img.device)), "shine_pipeline_fwd")
    return out


def corners(img, kappa, wx, wy, threshold: float, border: str = "clamp", mask=None, out=None, out_dtype=None):
    """Corner mask (uint8, 1 where R > threshold and R >= its 8 neighbours inside the output) of
    the fused forward + non-maximum suppression kernel (shine_corners). With out (or out_dtype)
    the kernel also writes R; returns (mask, R or None)."""
    _check_img(img)
    _param(kappa, "kappa", 1); _param(wx, "wx", 9); _param(wy, "wy", 9)
    h, w = img.shape[0], img.shape[1]
    ho, wo = output_shape(h, w, border)
    if mask is None:
        mask = torch.empty(ho, wo, device=img.device, dtype=torch.uint8)
    if mask.dtype != torch.uint8:
        raise TypeError("mask must be uint8")
    _check_map(mask, (ho, wo), "mask")
    if out is None and out_dtype is not None:
        out = torch.empty(ho, wo, device=img.device, dtype=out_dtype)
    if out is not None:
        _check_map(out, (ho, wo), "out")
    L.check(L.lib().shine_corners(_ptr(img), h, w, _row_pitch(img), dtype_code(img.dtype), border_code(border),
                                  _ptr(kappa), _ptr(wx), _ptr(wy), float(threshold), _ptr(mask), _row_pitch(mask),
                                  _ptr(out), _row_pitch(out) if out is not None else 0,
                                  dtype_code(out.dtype) if out is not None else dtype_code(img.dtype),
                                  _stream(img.device)), "shine_corners")
    return mask, out


def _grads_out(img, need_img, need_params, grad_img=None):
    dev = img.device
    gimg = grad_img if grad_img is not None else (torch.empty_like(img) if need_img else None)
    gk = torch.empty(1, device=dev, dtype=torch.float32) if need_params else None
    gwx = torch.empty(3, 3, device=dev, dtype=torch.float32) if need_params else None
    gwy = torch.empty(3, 3, device=dev, dtype=torch.float32) if need_params else None
    return gimg, gk, gwx, gwy


def pipeline_bwd(img, grad_out, kappa, wx, wy, border: str = "clamp", need_img: bool = True,
                 need_params: bool = True, workspace=None, grad_img=None):
    """(d img, d kappa, d wx, d wy) of L = sum(grad_out * R) (shine_pipeline_bwd)."""
    _check_img(img)
    _param(kappa, "kappa", 1); _param(wx, "wx", 9); _param(wy, "wy", 9)
    h, w = img.shape[0], img.shape[1]
    ho, wo = output_shape(h, w, border)
    _check_map(grad_out, (ho, wo), "grad_out")
    gimg, gk, gwx, gwy = _grads_out(img, need_img, need_params, grad_img)
    if gimg is not None:
        _check_img(gimg)
    nbytes = bwd_workspace_bytes(h, w, border)
    if workspace is None:
        workspace = torch.empty(max(nbytes, 16), device=img.device, dtype=torch.uint8)
    L.check(L.lib().shine_pipeline_bwd(_ptr(img), h, w, _row_pitch(img), dtype_code(img.dtype), border_code(border),
                                       _ptr(kappa), _ptr(wx), _ptr(wy), _ptr(grad_out), _row_pitch(grad_out),
                                       dtype_code(grad_out.dtype), _ptr(gimg),
                                       _row_pitch(gimg) if gimg is not None else 0, _ptr(gk), _ptr(gwx), _ptr(gwy),
                                       _ptr(workspace), workspace.numel(), _stream(img.device)),
            "shine_pipeline_bwd")
    return gimg, gk, gwx, gwy


def pipeline_fwd_bwd(img, grad_out, kappa, wx, wy, border: str = "clamp", need_img: bool = True,
                     need_params: bool = True, workspace=None, out=None, grad_img=None):
    """(R, d img, d kappa, d wx, d wy) in one pass (shine_pipeline_fwd_bwd)."""
    _check_img(img)
    _param(kappa, "kappa", 1); _param(wx, "wx", 9); _param(wy, "wy", 9)
    h, w = img.shape[0], img.shape[1]
    ho, wo = output_shape(h, w, border)
    _check_map(grad_out, (ho, wo), "grad_out")
    if grad_out.dtype != img.dtype:
        raise TypeError("shine_pipeline_fwd_bwd takes grad_out in the image's storage dtype")
    if out is None:
        out = torch.empty(ho, wo, device=img.device, dtype=img.dtype)
    _check_map(out, (ho, wo), "out")
    gimg, gk, gwx, gwy = _grads_out(img, need_img, need_params, grad_img)
    nbytes = bwd_workspace_bytes(h, w, border)
    if workspace is None:
        workspace = torch.empty(max(nbytes, 16), device=img.device, dtype=torch.uint8)
    L.check(L.lib().shine_pipeline_fwd_bwd(_ptr(img), h, w, _row_pitch(img), dtype_code(img.dtype),
                                           border_code(border), _ptr(kappa), _ptr(wx), _ptr(wy), _ptr(grad_out),
                                           _row_pitch(grad_out), _ptr(out), _row_pitch(out), _ptr(gimg),
                                           _row_pitch(gimg) if gimg is not None else 0, _ptr(gk), _ptr(gwx),
                                           _ptr(gwy), _ptr(workspace), workspace.numel(), _stream(img.device)),
            "shine_pipeline_fwd_bwd")
    return out, gimg, gk, gwx, gwy


def host_workspace_bytes(h: int, w: int, border: str, nbands: int) -> int:
    n = ctypes.c_size_t()
    L.check(L.lib().shine_pipeline_host_workspace(h, w, border_code(border), nbands, ctypes.byref(n)),
            "shine_pipeline_host_workspace")
    return n.value


def pipeline_host(img_h, g_h, kappa, wx, wy, dev_img, dev_g, dev_out, dev_gimg, workspace, out_h=None,
                  gimg_h=None, grad_params=None, border: str = "clamp", nbands: int = 16) -> None:
    """Forward + backward of a host (pinned) image with band-pipelined copies
    (shine_pipeline_host). Enqueues on the current stream; synchronise before reading the host
    outputs."""
    h, w = img_h.shape[0], img_h.shape[1]
    for t in (img_h, g_h, out_h, gimg_h):
        if t is not None and (t.is_cuda or not t.is_contiguous()):
            raise ValueError("host buffers must be contiguous CPU tensors (pinned for overlap)")
    L.check(L.lib().shine_pipeline_host(_ptr(img_h), _ptr(g_h), _ptr(out_h), _ptr(gimg_h), h, w,
                                        dtype_code(img_h.dtype), border_code(border), _ptr(kappa), _ptr(wx),
                                        _ptr(wy), _ptr(grad_params), _ptr(dev_img), _ptr(dev_g), _ptr(dev_out),
                                        _ptr(dev_gimg), _ptr(workspace), workspace.numel(), nbands,
                                        _stream(dev_img.device)), "shine_pipeline_host")


def mv(A: torch.Tensor, x: torch.Tensor, out=None) -> torch.Tensor:
    """y = A x (shine_mv): A is an (M, N) CUDA tensor (float32, bfloat16 or float16) with column
    stride 1, x an (N,) float32 CUDA tensor; y is float32."""
    if not A.is_cuda or A.dim() != 2 or (A.shape[1] > 1 and A.stride(1) != 1):
        raise ValueError("A must be a 2-D CUDA tensor with column stride 1")
    m, n = A.shape
    if not x.is_cuda or x.dtype != torch.float32 or x.shape != (n,) or (n > 1 and x.stride(0) != 1):
        raise ValueError(f"x must be a contiguous float32 CUDA tensor of shape ({n},)")
    if out is None:
        out = torch.empty(m, device=A.device, dtype=torch.float32)
    if out.shape != (m,) or out.dtype != torch.float32 or (m > 1 and out.stride(0) != 1):
        raise ValueError(f"out must be a contiguous float32 tensor of shape ({m},)")
    lda = A.stride(0) if m > 1 else max(n, 1)
    L.check(L.lib().shine_mv(_ptr(A), m, n, lda, dtype_code(A.dtype), _ptr(x), _ptr(out), _stream(A.device)),
            "shine_mv")
    return out


_REDUCE = {"sum": 0, "max": 1, "min": 2}


def iterate_sum(x: torch.Tensor, n: int, k: int, out=None, op: str = "sum") -> torch.Tensor:
    """iterate(k, split(n) >> map(reduce(op, identity))) of a contiguous float32 CUDA vector of
    length (n^k) m (shine_iterate_reduce; op "sum", "max" or "min"); returns the m tree
    reductions."""
    if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 1 or not x.is_contiguous():
        raise ValueError("x must be a contiguous 1-D float32 CUDA tensor")
    span = n ** k
    if n < 1 or k < 0 or x.numel() % span:
        raise ValueError(f"length {x.numel()} is not a multiple of n^k = {span}")
    m = x.numel() // span
    if out is None:
        out = torch.empty(m, device=x.device, dtype=torch.float32)
    if out.shape != (m,) or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous float32 tensor of shape ({m},)")
    if op not in _REDUCE:
        raise ValueError(f"op must be one of {sorted(_REDUCE)}")
    L.check(L.lib().shine_iterate_reduce(_ptr(x), m, n, k, _REDUCE[op], _ptr(out), _stream(x.device)),
            "shine_iterate_reduce")
    return out


def iterate_stencil(x: torch.Tensor, weights, k: int, out=None) -> torch.Tensor:
    """k rounds of the clamp-padded 3x3 stencil (iterate with a size-preserving body,
    shine_iterate_stencil) of an (H, W) float32 CUDA array with column stride 1; weights: 3 x 3
    host values (CPU tensor or nested sequence), applied as a correlation."""
    if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 2 or (x.shape[1] > 1 and x.stride(1) != 1):
        raise ValueError("x must be a 2-D float32 CUDA tensor with column stride 1")
    wt = torch.as_tensor(weights, dtype=torch.float32).cpu().contiguous()
    if wt.shape != (3, 3):
        raise ValueError("weights must be 3 x 3")
    h, w = x.shape
    if out is None:
        out = torch.empty(h, w, device=x.device, dtype=torch.float32)
    _check_map(out, (h, w), "out")
    if out.dtype != torch.float32:
        raise ValueError("out must be float32")
    L.check(L.lib().shine_iterate_stencil(_ptr(x), h, w, _row_pitch(x) if h > 1 else max(w, 1),
                                          ctypes.c_void_p(wt.data_ptr()), k, _ptr(out),
                                          _row_pitch(out) if h > 1 else max(w, 1), _stream(x.device)),
            "shine_iterate_stencil")
    return out


def stencil2d(x: torch.Tensor, weights=None, wv=None, wh=None, border: str = "clamp", out=None,
              out_dtype=None) -> torch.Tensor:
    """One slide2D(K, 1) + reduce stage (shine_stencil2d) of an (H, W) CUDA array (float32 or
    bfloat16, column stride 1). weights: (K, K) host weights, or wv and wh (K each) for the
    separable form. Weights are host values (CPU tensors or sequences)."""
    if not x.is_cuda or x.dim() != 2 or (x.shape[1] > 1 and x.stride(1) != 1):
        raise ValueError("x must be a 2-D CUDA tensor with column stride 1")
    h, w = x.shape
    if weights is not None:
        wt = torch.as_tensor(weights, dtype=torch.float32).cpu().contiguous()
        if wt.dim() != 2 or wt.shape[0] != wt.shape[1]:
            raise ValueError("weights must be K x K")
        K = wt.shape[0]
        wp, vp, hp = ctypes.cast(wt.data_ptr(), ctypes.c_void_p), None, None
        keep = (wt,)
    else:
        v = torch.as_tensor(wv, dtype=torch.float32).cpu().contiguous()
        hh = torch.as_tensor(wh, dtype=torch.float32).cpu().contiguous()
        if v.dim() != 1 or v.shape != hh.shape:
            raise ValueError("wv and wh must be 1-D of the same length K")
        K = v.shape[0]
        wp, vp, hp = None, ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(hh.data_ptr())
        keep = (v, hh)
    r = (K - 1) // 2
    ho, wo = (h, w) if border == "clamp" else (h - 2 * r, w - 2 * r)
    odt = x.dtype if out_dtype is None else out_dtype
    if out is None:
        out = torch.empty(max(ho, 0), max(wo, 0), device=x.device, dtype=odt)
    _check_map(out, (ho, wo), "out")
    L.check(L.lib().shine_stencil2d(_ptr(x), h, w, _row_pitch(x) if h > 1 else max(w, 1), dtype_code(x.dtype),
                                    border_code(border), K, wp, vp, hp, _ptr(out),
                                    _row_pitch(out) if out.shape[0] > 1 else max(wo, 1), dtype_code(out.dtype),
                                    _stream(x.device)), "shine_stencil2d")
    del keep
    return out


def harris_window(img, kappa, wx, wy, gv, gh, out=None, out_dtype=None) -> torch.Tensor:
    """R of the Harris pipeline with a separable K-tap window (gv down the columns, gh along the
    rows; host values) at A4, CLAMP borders (shine_harris_window)."""
    _check_img(img)
    _param(kappa, "kappa", 1); _param(wx, "wx", 9); _param(wy, "wy", 9)
    v = torch.as_tensor(gv, dtype=torch.float32).cpu().contiguous()
    hh = torch.as_tensor(gh, dtype=torch.float32).cpu().contiguous()
    if v.dim() != 1 or v.shape != hh.shape:
        raise ValueError("gv and gh must be 1-D of the same length K")
    h, w = img.shape[0], img.shape[1]
    if out is None:
        out = torch.empty(h, w, device=img.device, dtype=img.dtype if out_dtype is None else out_dtype)
    _check_map(out, (h, w), "out")
    L.check(L.lib().shine_harris_window(_ptr(img), h, w, _row_pitch(img), dtype_code(img.dtype), _ptr(kappa),
                                        _ptr(wx), _ptr(wy), v.shape[0], ctypes.c_void_p(v.data_ptr()),
                                        ctypes.c_void_p(hh.data_ptr()), _ptr(out), _row_pitch(out),
                                        dtype_code(out.dtype), _stream(img.device)), "shine_harris_window")
    return out


def _as_param(v, like: torch.Tensor, shape) -> torch.Tensor:
    if isinstance(v, torch.Tensor):
        return v
    return torch.full(shape, float(v), device=like.device, dtype=torch.float32)


class HarrisFn(torch.autograd.Function):
    """R = harris(img, kappa, wx, wy) with the hand-written adjoint kernel as its backward.

    Gradients are returned for img (storage dtype), kappa, wx and wy (float32). The Sobel
    stage is recomputed in the backward kernel; only the inputs are saved."""

    @staticmethod
    def forward(ctx, img, kappa, wx, wy, border="clamp", out_dtype=None):
        kappa_c = kappa.reshape(1).contiguous()
        out = pipeline_fwd(img, kappa_c, wx.contiguous(), wy.contiguous(), border, out_dtype)
        ctx.save_for_backward(img, kappa_c, wx, wy)
        ctx.border = border
        ctx.kappa_shape = kappa.shape
        return out

    @staticmethod
    def backward(ctx, grad_out):
        img, kappa, wx, wy = ctx.saved_tensors
        need_img = ctx.needs_input_grad[0]
        need_params = any(ctx.needs_input_grad[1:4])
        if not (need_img or need_params):
            return None, None, None, None, None, None
        if grad_out.dtype not in (img.dtype, torch.float32):
            grad_out = grad_out.float()
        grad_out = grad_out.contiguous()  # autograd may hand over an expanded (stride 0) tensor
        gimg, gk, gwx, gwy = pipeline_bwd(img, grad_out, kappa, wx.contiguous(), wy.contiguous(), ctx.border,
                                          need_img=need_img, need_params=need_params)
        return (gimg if need_img else None,
                gk.reshape(ctx.kappa_shape) if ctx.needs_input_grad[1] else None,
                gwx if ctx.needs_input_grad[2] else None,
                gwy if ctx.needs_input_grad[3] else None, None, None)


def harris(img, kappa=0.04, wx=None, wy=None, border: str = "clamp", out_dtype=None) -> torch.Tensor:
    """Differentiable Harris response of an (H, W, 3) CUDA image (default Sobel weights)."""
    if wx is None or wy is None:
        sx = torch.tensor([[-1.0, 0.0, 1.0], [-2.0, 0.0, 2.0], [-1.0, 0.0, 1.0]], device=img.device)
        wx = sx if wx is None else wx
        wy = sx.t().contiguous() if wy is None else wy
    kappa = _as_param(kappa, img, (1,))
    return HarrisFn.apply(img, kappa, wx, wy, border, out_dtype)
