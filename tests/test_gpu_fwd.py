"""Forward kernel parity against the FP64 oracle, element by element (small images spanning
several warp segments and row bands with ragged tails) and on sampled outputs at full size."""
import numpy as np
import pytest
import torch

import gpu_util as U
import workloads as wl
from oracle import cref

pytestmark = pytest.mark.gpu

SHAPES = [((1, 1), "clamp"), ((1, 7), "clamp"), ((2, 3), "clamp"), ((3, 5), "clamp"), ((7, 129), "clamp"),
          ((37, 250), "clamp"), ((130, 367), "clamp"), ((300, 5), "clamp"), ((5, 300), "clamp"),
          ((64, 121), "clamp"), ((64, 124), "clamp"), ((5, 5), "valid"), ((9, 133), "valid"),
          ((70, 245), "valid"), ((256, 256), "valid")]


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


@pytest.mark.parametrize("shape,border", SHAPES)
@pytest.mark.parametrize("weights", ["sobel", "random"])
def test_fwd_f32_matches_oracle(shine, shape, border, weights):
    h, w = shape
    img = wl.random_image(h, w, seed=h * 1000 + w)
    wx, wy = wl.sobel_weights() if weights == "sobel" else wl.random_weights(h + w)
    ref = cref.forward(img, 0.04, wx, wy, border)
    k, dwx, dwy = U.dev_params(0.04, wx, wy)
    out = shine.pipeline_fwd(img.cuda(), k, dwx, dwy, border)
    torch.cuda.synchronize()
    assert out.shape == ref.shape
    assert U.rel(U.host(out), ref) <= U.TOL_F32


def test_plain_256_valid(shine):
    cfg = wl.plain_256()
    wx, wy = wl.sobel_weights()
    ref = cref.forward(cfg["img"], cfg["kappa"], wx, wy, cfg["border"])
    k, dwx, dwy = U.dev_params(cfg["kappa"], wx, wy)
    out = shine.pipeline_fwd(cfg["img"].cuda(), k, dwx, dwy, cfg["border"])
    assert out.shape == (252, 252)
    assert U.rel(U.host(out), ref) <= U.TOL_F32


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
@pytest.mark.parametrize("shape,border", [((37, 250), "clamp"), ((130, 367), "clamp"), ((70, 245), "valid"),
                                          ((3, 5), "clamp")])
def test_fwd_16bit_storage(shine, dtype, shape, border):
    h, w = shape
    img = wl.random_image(h, w, seed=5, dtype=dtype)          # already RN-quantised
    wx, wy = wl.sobel_weights()
    ref_q = cref.forward(img, 0.04, wx, wy, border)          # oracle on the quantised input
    k, dwx, dwy = U.dev_params(0.04, wx, wy)
    out16 = shine.pipeline_fwd(img.cuda(), k, dwx, dwy, border)
    out32 = shine.pipeline_fwd(img.cuda(), k, dwx, dwy, border, out_dtype=torch.float32)
    assert out16.dtype == img.dtype
    assert U.rel(U.host(out16), ref_q) <= U.TOL_16
    assert U.rel(U.host(out32), ref_q) <= U.TOL_F32          # float32 arithmetic, float32 output


@pytest.mark.parametrize("shape,border", [((37, 250), "clamp"), ((70, 245), "valid"), ((9, 7), "clamp")])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_unaligned_pitch_path_is_bit_identical(shine, shape, border, dtype):
    h, w = shape
    img = wl.random_image(h, w, seed=2).to(dtype).cuda()
    k, dwx, dwy = U.dev_params(0.05, *wl.random_weights(3))
    a = shine.pipeline_fwd(img, k, dwx, dwy, border)
    b = shine.pipeline_fwd(U.padded_image(img, 1), k, dwx, dwy, border)   # element-wise staging
    ho, wo = a.shape
    store = torch.zeros(ho, wo + 1, dtype=dtype, device="cuda")
    c = shine.pipeline_fwd(img, k, dwx, dwy, border, out=store[:, 1:])   # element-wise stores
    assert torch.equal(a, b) and torch.equal(a, c)


def test_homogeneity_bit_exact(shine):
    """R(2 img) = 16 R(img) exactly: every step scales by a power of two."""
    img = wl.random_image(97, 301, seed=9).cuda()
    k, dwx, dwy = U.dev_params(0.04, *wl.random_weights(9))
    for border in ("clamp", "valid"):
        r1 = shine.pipeline_fwd(img, k, dwx, dwy, border)
        r2 = shine.pipeline_fwd(img * 2, k, dwx, dwy, border)
        assert torch.equal(r2, r1 * 16)


def test_constant_image_gives_zero(shine):
    img = torch.full((33, 250, 3), 0.375, device="cuda")
    k, dwx, dwy = U.dev_params(0.04, *wl.sobel_weights())
    for border in ("clamp", "valid"):
        assert torch.count_nonzero(shine.pipeline_fwd(img, k, dwx, dwy, border)) == 0


def test_guard_band_untouched(shine):
    """Writes stay inside the output rows: a sentinel-filled pitch gap is left intact."""
    img = wl.random_image(41, 131, seed=4).cuda()
    k, dwx, dwy = U.dev_params(0.04, *wl.sobel_weights())
    for border in ("clamp", "valid"):
        ho, wo = shine.output_shape(41, 131, border)
        store = torch.full((ho, wo + 9), 7.0, device="cuda")
        shine.pipeline_fwd(img, k, dwx, dwy, border, out=store[:, :wo])
        assert torch.all(store[:, wo:] == 7.0)


def test_salt_8192_sampled(shine):
    """The 8192 x 8192 salt-noise workload: sampled outputs (interior, corners and border bands)
    against the oracle's point form, plus exact homogeneity over the whole map."""
    cfg = wl.salt_8192()
    img = cfg["img"]
    wx, wy = wl.sobel_weights()
    k, dwx, dwy = U.dev_params(cfg["kappa"], wx, wy)
    dimg = img.cuda()
    out = shine.pipeline_fwd(dimg, k, dwx, dwy, "clamp")
    pts = wl.sample_points(8192, 8192, 4000, seed=21)
    ref = cref.forward_points(img, cfg["kappa"], wx, wy, "clamp", pts)
    got = U.host(out[pts[:, 0].cuda(), pts[:, 1].cuda()])
    assert U.rel(got, ref) <= U.TOL_F32
    out2 = shine.pipeline_fwd(dimg * 2, k, dwx, dwy, "clamp")
    assert torch.equal(out2, out * 16)


def test_diff_2048_full_map(shine):
    """The 2048 x 2048 differentiation image, CLAMP, float32: the whole response map against the
    oracle element by element (16-byte aligned rows: bulk-staged interior segments, register-staged
    edge segments), with the default and with random non-symmetric weights."""
    cfg = wl.diff_2048()
    for ww in (wl.sobel_weights(), wl.random_weights(31)):
        ref = cref.forward(cfg["img"], wl.KAPPA, *ww, "clamp")
        k, dwx, dwy = U.dev_params(wl.KAPPA, *ww)
        out = shine.pipeline_fwd(cfg["img"].cuda(), k, dwx, dwy, "clamp")
        torch.cuda.synchronize()
        assert U.rel(U.host(out), ref) <= U.TOL_F32


def test_salt_8192_full_rows(shine):
    """The 8192 x 8192 salt workload in the benchmark's launch configuration, compared element by
    element over three bands of 600 whole rows (the top, the middle and the bottom of the image).
    At this size each warp streams a strip of about 250 rows, so the staging ring's slots and
    phases wrap many times within a strip, and strips end and start inside every band. The oracle
    runs on each band as an image of its own; R of a band's image equals R of the full image
    except within 2 rows of a cut (the clamp), so those rows are left out."""
    cfg = wl.salt_8192()
    img = cfg["img"]
    wx, wy = wl.sobel_weights()
    k, dwx, dwy = U.dev_params(cfg["kappa"], wx, wy)
    out = U.host(shine.pipeline_fwd(img.cuda(), k, dwx, dwy, "clamp"))
    n = 600
    for a in (0, 4096 - n // 2, 8192 - n):
        ref = cref.forward(img[a:a + n].contiguous(), cfg["kappa"], wx, wy, "clamp")
        lo = 0 if a == 0 else 2
        hi = n if a + n == 8192 else n - 2
        assert U.rel(out[a + lo:a + hi], ref[lo:hi]) <= U.TOL_F32, a
