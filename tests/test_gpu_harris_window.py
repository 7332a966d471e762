"""Parity of the Gaussian-window Harris kernel (shine_harris_window) with the FP64 oracle.

R cancels (det - kappa trace^2), so as for the forward pass the gate is normwise:
max|R - R_ref| / max|R_ref| <= 1e-5 for float32 storage and 2e-2 for bf16 storage (the oracle
runs on the bf16-quantised image).
"""
import numpy as np
import pytest
import torch

import gpu_util as U
import workloads as wl
from oracle import harris_window as HW

pytestmark = pytest.mark.gpu

SHAPES = [(37, 250), (130, 300), (3, 517), (1, 1), (2, 5), (64, 129)]


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


def _params(seed):
    wx, wy = wl.random_weights(seed)
    return torch.tensor([0.04], device="cuda"), wx.cuda(), wy.cuda(), wx.double().numpy(), wy.double().numpy()


@pytest.mark.parametrize("K", [3, 5, 7])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_matches_oracle(shine, K, shape, dtype):
    h, w = shape
    img = wl.random_image(h, w, seed=h * 3 + w + K).to(dtype)
    k, wx, wy, wxn, wyn = _params(K + h)
    gv, gh = wl.gaussian_window(K)
    r = shine.harris_window(img.cuda(), k, wx, wy, gv, gh, out_dtype=torch.float32).cpu().numpy()
    ref = HW.harris_window_np(img.double().numpy(), 0.04, wxn, wyn, gv.double().numpy(), gh.double().numpy())
    assert U.rel(r, ref) <= (U.TOL_F32 if dtype == torch.float32 else U.TOL_16)


def test_unit_box_window_is_close_to_the_forward(shine):
    """With gv = gh = (1, 1, 1) the window is the forward's 3x3 box (same value up to rounding)."""
    img = wl.random_image(90, 270, seed=4).cuda()
    k, wx, wy, _, _ = _params(4)
    r_win = shine.harris_window(img, k, wx, wy, [1.0] * 3, [1.0] * 3)
    r_fwd = shine.pipeline_fwd(img, k, wx, wy, "clamp")
    assert U.rel(r_win.cpu().numpy(), r_fwd.double().cpu().numpy()) <= 1e-6


def test_unaligned_rows(shine):
    h, w = 40, 301
    base = wl.random_image(h, w + 1, seed=6).cuda()
    img = base[:, :w]
    k, wx, wy, wxn, wyn = _params(6)
    gv, gh = wl.gaussian_window(5)
    r = shine.harris_window(img, k, wx, wy, gv, gh).cpu().numpy()
    ref = HW.harris_window_np(img.double().cpu().numpy(), 0.04, wxn, wyn, gv.double().numpy(), gh.double().numpy())
    assert U.rel(r, ref) <= U.TOL_F32


def test_full_size_sampled(shine):
    """The 8192 x 8192 salt workload with a 5-tap Gaussian window, sampled outputs."""
    img = wl.salt_8192()["img"]
    k = torch.tensor([wl.KAPPA], device="cuda")
    wx, wy = wl.sobel_weights()
    gv, gh = wl.gaussian_window(5)
    r = shine.harris_window(img.cuda(), k, wx.cuda(), wy.cuda(), gv, gh)
    pts = wl.sample_points(8192, 8192, 600, seed=13)
    got = r[pts[:, 0].cuda(), pts[:, 1].cuda()].cpu().numpy()
    ref = HW.harris_window_points(img.numpy(), wl.KAPPA, wx.double().numpy(), wy.double().numpy(),
                                  gv.double().numpy(), gh.double().numpy(), pts.numpy())
    assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= U.TOL_F32
