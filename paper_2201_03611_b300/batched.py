"""Many images of uneven sizes in one persistent launch (shine_plan_* / shine_pipeline_batched).

    plan = BatchedPlan([(H, W), ...], torch.bfloat16, "clamp", fwd_bwd=True)
    batch = plan.bind(imgs, outs, grad_outs, grad_imgs)     # device descriptor array
    plan.run(batch, kappa, wx, wy, grad_kappa, grad_wx, grad_wy)   # no alloc, no sync

``run`` only enqueues work on the current stream, so it can be captured in a CUDA graph.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .ops import _ptr, _stream, border_code, dtype_code


class BatchedPlan:
    def __init__(self, shapes, dtype: torch.dtype, border: str = "clamp", fwd_bwd: bool = True,
                 tune_cache: str | None = None):
        self.shapes = [(int(h), int(w)) for h, w in shapes]
        self.n = len(self.shapes)
        self.dtype = dtype
        self.border = border
        self.mode = L.SHINE_MODE_FWD_BWD if fwd_bwd else L.SHINE_MODE_FWD
        hw = (ctypes.c_int64 * (2 * self.n))(*[v for s in self.shapes for v in s])
        handle = ctypes.c_void_p()
        L.check(L.lib().shine_plan_create(hw, self.n, dtype_code(dtype), border_code(border), self.mode,
                                          tune_cache.encode() if tune_cache else None, ctypes.byref(handle)),
                "shine_plan_create")
        self._h = handle
        n = ctypes.c_size_t()
        L.check(L.lib().shine_plan_workspace(self._h, ctypes.byref(n)), "shine_plan_workspace")
        self.workspace_bytes = n.value

    def tile_rows(self, i: int) -> int:
        r = ctypes.c_int32()
        L.check(L.lib().shine_plan_tile_rows(self._h, i, ctypes.byref(r)), "shine_plan_tile_rows")
        return r.value

    def schedule(self) -> dict:
        """The schedule the plan chose (claim order, staging, edge weight x 4, segment origin)."""
        v = [ctypes.c_int32() for _ in range(4)]
        L.check(L.lib().shine_plan_schedule(self._h, *[ctypes.byref(x) for x in v]), "shine_plan_schedule")
        return dict(zip(("order", "staging", "edge_w4", "origin"), (x.value for x in v)))

    def bind(self, imgs, outs=None, grad_outs=None, grad_imgs=None) -> torch.Tensor:
        """Device array of shine_image_desc for these tensors (kept alive by the caller)."""
        if len(imgs) != self.n:
            raise ValueError("one image per planned shape")
        descs = (L.ImageDesc * self.n)()
        for i, img in enumerate(imgs):
            h, w = self.shapes[i]
            if tuple(img.shape) != (h, w, 3) or img.dtype != self.dtype or img.stride(2) != 1 or img.stride(1) != 3:
                raise ValueError(f"image {i}: expected ({h}, {w}, 3) {self.dtype} with pixel stride 3")
            d = descs[i]
            d.img = img.data_ptr()
            d.H, d.W, d.img_pitch = h, w, img.stride(0)
            for name, lst in (("out", outs), ("grad_out", grad_outs), ("grad_img", grad_imgs)):
                t = None if lst is None else lst[i]
                if t is not None:
                    if t.dtype != self.dtype:
                        raise ValueError(f"{name}[{i}] must have the plan dtype")
                    setattr(d, name, t.data_ptr())
                    setattr(d, {"out": "out_pitch", "grad_out": "gout_pitch", "grad_img": "gimg_pitch"}[name],
                            t.stride(0))
        host = torch.frombuffer(bytearray(bytes(descs)), dtype=torch.uint8)
        return host.to(imgs[0].device)

    def new_workspace(self, device) -> torch.Tensor:
        return torch.empty(max(self.workspace_bytes, 256), device=device, dtype=torch.uint8)

    def run(self, descs: torch.Tensor, kappa, wx, wy, grad_kappa=None, grad_wx=None, grad_wy=None,
            workspace: torch.Tensor | None = None) -> None:
        if workspace is None:
            workspace = self.new_workspace(descs.device)
        L.check(L.lib().shine_pipeline_batched(self._h, _ptr(descs), _ptr(kappa), _ptr(wx), _ptr(wy),
                                               _ptr(grad_kappa), _ptr(grad_wx), _ptr(grad_wy), _ptr(workspace),
                                               workspace.numel(), _stream(descs.device)),
                "shine_pipeline_batched")

    def close(self) -> None:
        if getattr(self, "_h", None):
            L.lib().shine_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
