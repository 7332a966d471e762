"""Parity of the fused corner kernel (shine_corners: forward + threshold + 3x3 non-maximum
suppression) with the oracle's definition applied to the same R.

The mask is integer output decided by floating point: the test takes the decision in the
kernel's precision, on the kernel's own float32 R (shine_pipeline_fwd with a float32 output,
bit-identical to the R the corner kernel computes), and requires the masks to be equal bit
for bit. R itself is checked against the FP64 oracle by the forward tests.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import corners as C

pytestmark = pytest.mark.gpu

SHAPES = [((37, 250), "clamp"), ((70, 245), "valid"), ((203, 517), "clamp"), ((130, 256), "clamp"),
          ((1, 1), "clamp"), ((3, 3), "clamp"), ((9, 9), "valid"), ((64, 1000), "valid")]


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


def _params(seed):
    wx, wy = wl.random_weights(seed)
    return (torch.tensor([0.04], device="cuda"), wx.cuda(), wy.cuda())


@pytest.mark.parametrize("shape,border", SHAPES)
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("q", [0.0, 0.5, 0.9])
def test_mask_matches_definition_on_kernel_R(shine, shape, border, dtype, q):
    h, w = shape
    img = wl.random_image(h, w, seed=h + 3 * w).to(dtype).cuda()
    k, wx, wy = _params(h)
    r32 = shine.pipeline_fwd(img, k, wx, wy, border, out_dtype=torch.float32).cpu().numpy()
    thr = float(np.quantile(r32, q)) if r32.size > 1 else float(r32.min()) - 1.0
    mask, r = shine.corners(img, k, wx, wy, thr, border, out_dtype=torch.float32)
    torch.cuda.synchronize()
    assert np.array_equal(r.cpu().numpy(), r32)          # the kernel's R is the forward's R
    assert np.array_equal(mask.cpu().numpy(), C.nms(r32, thr))


def test_mask_without_R_and_with_storage_R(shine):
    img = wl.random_image(150, 300, seed=3).to(torch.bfloat16).cuda()
    k, wx, wy = _params(3)
    r32 = shine.pipeline_fwd(img, k, wx, wy, "clamp", out_dtype=torch.float32).cpu().numpy()
    thr = float(np.quantile(r32, 0.7))
    m0, none = shine.corners(img, k, wx, wy, thr, "clamp")
    m1, r16 = shine.corners(img, k, wx, wy, thr, "clamp", out_dtype=torch.bfloat16)
    assert none is None
    assert torch.equal(m0, m1)
    assert np.array_equal(m0.cpu().numpy(), C.nms(r32, thr))
    assert torch.equal(r16, shine.pipeline_fwd(img, k, wx, wy, "clamp"))


def test_unaligned_pitches(shine):
    """Image and mask rows that allow no vector access (odd pitches): the element paths."""
    h, w = 61, 301
    base = wl.random_image(h, w + 1, seed=5).cuda()
    img = base[:, :w]                                   # pitch 3 (w + 1) elements
    mbase = torch.zeros(h, w + 3, dtype=torch.uint8, device="cuda")
    mask = mbase[:, 1:w + 1]                             # odd offset and pitch
    k, wx, wy = _params(5)
    r32 = shine.pipeline_fwd(img, k, wx, wy, "clamp").cpu().numpy()
    thr = float(np.quantile(r32, 0.8))
    shine.corners(img, k, wx, wy, thr, "clamp", mask=mask)
    torch.cuda.synchronize()
    assert np.array_equal(mask.cpu().numpy(), C.nms(r32, thr))
    assert (mbase[:, 0] == 0).all() and (mbase[:, w + 1:] == 0).all()   # nothing outside


def test_constant_image_ties(shine):
    """With the Sobel weights (rows summing to zero) a constant image has R == 0 exactly: every
    pixel ties with its neighbours, so every pixel is a corner for a negative threshold and
    none for threshold 0."""
    img = torch.full((40, 300, 3), 0.25, device="cuda")
    k = torch.tensor([0.04], device="cuda")
    wx, wy = [t.cuda() for t in wl.sobel_weights()]
    assert int((shine.pipeline_fwd(img, k, wx, wy, "clamp") != 0).sum()) == 0
    m, _ = shine.corners(img, k, wx, wy, -1.0, "clamp")
    assert bool((m == 1).all())
    m, _ = shine.corners(img, k, wx, wy, 0.0, "clamp")
    assert int(m.sum()) == 0


def test_full_size_salt_8192(shine):
    """The 8192 x 8192 salt workload in the benchmark's configuration: every mask byte."""
    img = wl.salt_8192()["img"].cuda()
    k = torch.tensor([wl.KAPPA], device="cuda")
    wx, wy = [t.cuda() for t in wl.sobel_weights()]
    r32 = shine.pipeline_fwd(img, k, wx, wy, "clamp").cpu().numpy()
    thr = wl.CORNER_THRESHOLD
    mask, _ = shine.corners(img, k, wx, wy, thr, "clamp")
    got = mask.cpu().numpy()
    assert np.array_equal(got, C.nms(r32, thr))
    assert 0 < got.sum() < got.size // 10


def test_nan_in_R(shine):
    """NaN pixels make NaN patches in R: a NaN is never a corner and, since no value is >= NaN,
    neither is a pixel with a NaN neighbour (the definition, applied to the kernel's own R)."""
    img = wl.random_image(90, 300, seed=9).cuda()
    for y, x, ch in ((40, 100, 0), (10, 250, 2), (89, 0, 1), (0, 299, 0)):
        img[y, x, ch] = float("nan")
    k, wx, wy = _params(9)
    r32 = shine.pipeline_fwd(img, k, wx, wy, "clamp").cpu().numpy()
    assert np.isnan(r32).any() and np.isfinite(r32).any()
    thr = float(np.quantile(r32[np.isfinite(r32)], 0.6))
    mask, _ = shine.corners(img, k, wx, wy, thr, "clamp")
    assert np.array_equal(mask.cpu().numpy(), C.nms(r32, thr))
