"""Helpers for the GPU parity tests: metrics and device copies of the seeded inputs."""
import numpy as np
import torch

# Tolerances (normwise: max |x - ref| / max |ref| per output tensor; pointwise relative error is
# ill-posed where R cancels to ~0):
#   float32 storage, against the FP64 oracle ............................ 1e-5
#   bf16 / fp16 storage, against the oracle run on the quantised input .. 2e-2
#   float32 gradients against the oracle's FP64 reverse-mode gradient ... 1e-5 for d img,
#                                         1e-4 for the summed parameter cotangents
#   float32 gradients against FP64 finite differences on a 32x32 crop ... 1e-4
TOL_F32 = 1e-5
TOL_16 = 2e-2
TOL_GIMG = 1e-5
TOL_PARAM = 1e-4
TOL_FD = 1e-4


def rel(got, ref) -> float:
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.abs(got - ref).max(initial=0.0) / max(np.abs(ref).max(initial=0.0), 1e-300))


def host(t: torch.Tensor) -> np.ndarray:
    return t.detach().float().cpu().double().numpy()


def dev_params(kappa, wx, wy):
    k = torch.tensor([float(kappa)], dtype=torch.float32, device="cuda")
    return k, wx.float().contiguous().cuda(), wy.float().contiguous().cuda()


def padded_image(img: torch.Tensor, extra: int) -> torch.Tensor:
    """Same pixels, with rows padded by `extra` elements (row pitch 3W + extra)."""
    h, w, _ = img.shape
    store = torch.zeros(h, 3 * w + extra, dtype=img.dtype, device=img.device)
    store[:, :3 * w] = img.reshape(h, 3 * w)
    return store.as_strided((h, w, 3), (3 * w + extra, 3, 1))
