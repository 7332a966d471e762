"""Adjoint kernel parity: against the oracle's FP64 reverse-mode gradient element by element,
against FP64 finite differences on a 32x32 crop, determinism, the fused forward+backward
entry, and the torch.autograd.Function."""
import numpy as np
import pytest
import torch

import gpu_util as U
import workloads as wl
from oracle import cref

pytestmark = pytest.mark.gpu

SHAPES = [((1, 1), "clamp"), ((1, 6), "clamp"), ((2, 2), "clamp"), ((4, 3), "clamp"), ((7, 129), "clamp"),
          ((37, 250), "clamp"), ((130, 367), "clamp"), ((301, 9), "clamp"), ((64, 124), "clamp"),
          ((5, 5), "valid"), ((9, 133), "valid"), ((70, 245), "valid")]


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


@pytest.fixture
def wide_adjoint(monkeypatch):
    """16-bit CLAMP images with 16-byte aligned rows take the eight-column adjoint at any size
    (by default only from 2^25 pixels on, where it is the faster one)."""
    monkeypatch.setenv("SHINE_WIDE_BWD_MIN_PIXELS", "0")


def _run_bwd(shine, img, g, kappa, wx, wy, border, **kw):
    k, dwx, dwy = U.dev_params(kappa, wx, wy)
    return shine.pipeline_bwd(img.cuda(), g.cuda(), k, dwx, dwy, border, **kw)


@pytest.mark.parametrize("shape,border", SHAPES)
def test_bwd_f32_matches_oracle(shine, shape, border):
    h, w = shape
    img = wl.random_image(h, w, seed=h * 7 + w)
    wx, wy = wl.random_weights(h)
    ho, wo = shine.output_shape(h, w, border)
    g = wl.random_cotangent(ho, wo, seed=w)
    ref = cref.backward(img, g, 0.05, wx, wy, border, with_abs=True)
    dgi, dgk, dgwx, dgwy = _run_bwd(shine, img, g, 0.05, wx, wy, border)
    torch.cuda.synchronize()
    assert U.rel(U.host(dgi), ref[0]) <= U.TOL_GIMG
    U.assert_params((dgk, dgwx, dgwy), ref[1:])


def test_fd_on_32x32_crop(shine):
    """The differentiation workload's check: FP64 central differences of the oracle on the
    top-left 32x32 crop (as a CLAMP image of its own) for all 3072 + 1 + 18 parameters."""
    cfg = wl.diff_2048()
    img = cfg["img"][:32, :32].contiguous()
    g = cfg["w"][:32, :32].contiguous()
    wx, wy = wl.sobel_weights()
    kappa = cfg["kappa"]
    img64, g64 = img.double(), g.double().numpy()

    def L(im=img64, k=kappa, a=wx.double(), b=wy.double()):
        return float(np.sum(g64 * cref.forward(im, k, a, b, "clamp")))
    fd_img = np.zeros((32, 32, 3))
    for i in range(32):
        for j in range(32):
            for c in range(3):
                hh = 1e-6 * max(1.0, abs(float(img64[i, j, c])))
                p, m = img64.clone(), img64.clone()
                p[i, j, c] += hh
                m[i, j, c] -= hh
                fd_img[i, j, c] = (L(im=p) - L(im=m)) / (2 * hh)
    hk = 1e-6 * max(1.0, kappa)
    fd_k = (L(k=kappa + hk) - L(k=kappa - hk)) / (2 * hk)
    fd_w = []
    for which in (0, 1):
        out = np.zeros((3, 3))
        base = (wx if which == 0 else wy).double()
        for a in range(3):
            for b in range(3):
                hh = 1e-6 * max(1.0, abs(float(base[a, b])))
                p, m = base.clone(), base.clone()
                p[a, b] += hh
                m[a, b] -= hh
                out[a, b] = ((L(a=p) - L(a=m)) if which == 0 else (L(b=p) - L(b=m))) / (2 * hh)
        fd_w.append(out)
    dgi, dgk, dgwx, dgwy = _run_bwd(shine, img, g, kappa, wx, wy, "clamp")
    assert U.rel(U.host(dgi), fd_img) <= U.TOL_FD
    assert U.rel(U.host(dgk), [fd_k]) <= U.TOL_FD
    assert U.rel(U.host(dgwx), fd_w[0]) <= U.TOL_FD
    assert U.rel(U.host(dgwy), fd_w[1]) <= U.TOL_FD


def test_diff_2048_full(shine):
    """The 2048 x 2048 differentiation workload against the oracle's full FP64 gradient."""
    cfg = wl.diff_2048()
    wx, wy = wl.sobel_weights()
    ref = cref.backward(cfg["img"], cfg["w"], cfg["kappa"], wx, wy, "clamp", with_abs=True)
    dgi, dgk, dgwx, dgwy = _run_bwd(shine, cfg["img"], cfg["w"], cfg["kappa"], wx, wy, "clamp")
    assert U.rel(U.host(dgi), ref[0]) <= U.TOL_GIMG
    U.assert_params((dgk, dgwx, dgwy), ref[1:])


def test_salt_8192_full(shine):
    """The benchmark's adjoint workload (8192 x 8192 salt image, N(0,1) cotangent from seed 1, in
    the launch configuration the benchmark times) against the oracle's full FP64 gradient."""
    img = wl.salt_8192()["img"]
    g = wl.random_cotangent(8192, 8192, seed=1)
    wx, wy = wl.sobel_weights()
    dgi, dgk, dgwx, dgwy = _run_bwd(shine, img, g, wl.KAPPA, wx, wy, "clamp")
    torch.cuda.synchronize()
    dgi = U.host(dgi)
    ref = cref.backward(img, g, wl.KAPPA, wx, wy, "clamp", with_abs=True)
    assert U.rel(dgi, ref[0]) <= U.TOL_GIMG
    U.assert_params((dgk, dgwx, dgwy), ref[1:])


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_bwd_16bit_storage(shine, dtype):
    img = wl.random_image(130, 367, seed=3, dtype=dtype)
    g = wl.random_cotangent(130, 367, seed=4, dtype=dtype)
    wx, wy = wl.sobel_weights()
    ref = cref.backward(img, g, 0.04, wx, wy, "clamp", with_abs=True)  # oracle on quantised inputs
    dgi, dgk, dgwx, dgwy = _run_bwd(shine, img, g, 0.04, wx, wy, "clamp")
    assert dgi.dtype == img.dtype
    assert U.rel(U.host(dgi), ref[0]) <= U.TOL_16
    U.assert_params((dgk, dgwx, dgwy), ref[1:])                          # float32 arithmetic
    # float32 cotangent with a 16-bit image
    dgi32 = _run_bwd(shine, img, g.float(), 0.04, wx, wy, "clamp")[0]
    assert U.rel(U.host(dgi32), ref[0]) <= U.TOL_16


def test_bwd_deterministic(shine):
    img = wl.random_image(300, 500, seed=5)
    g = wl.random_cotangent(300, 500, seed=6)
    wx, wy = wl.random_weights(5)
    a = _run_bwd(shine, img, g, 0.04, wx, wy, "clamp")
    b = _run_bwd(shine, img, g, 0.04, wx, wy, "clamp")
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("shape,border", [((37, 250), "clamp"), ((70, 245), "valid"), ((3, 3), "clamp"),
                                          ((67, 256), "clamp"), ((130, 1000), "clamp")])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("wide", [False, True])
def test_fused_equals_separate(shine, shape, border, dtype, wide, monkeypatch):
    """The fused pass gives the forward's R and the adjoint's cotangents bit for bit (with the
    eight-column kernel allowed at any size, 16-byte aligned 16-bit rows -- 256 and 1000 columns --
    take it for both)."""
    if wide:
        monkeypatch.setenv("SHINE_WIDE_BWD_MIN_PIXELS", "0")
    h, w = shape
    img = wl.random_image(h, w, seed=8).to(dtype).cuda()
    ho, wo = shine.output_shape(h, w, border)
    g = wl.random_cotangent(ho, wo, seed=9).to(dtype).cuda()
    k, dwx, dwy = U.dev_params(0.04, *wl.random_weights(8))
    r = shine.pipeline_fwd(img, k, dwx, dwy, border)
    sep = shine.pipeline_bwd(img, g, k, dwx, dwy, border)
    fused = shine.pipeline_fwd_bwd(img, g, k, dwx, dwy, border)
    assert torch.equal(fused[0], r)
    for x, y in zip(fused[1:], sep):
        assert torch.equal(x, y)


def test_bwd_unaligned_paths_bit_identical(shine):
    img = wl.random_image(41, 250, seed=10).cuda()
    g = wl.random_cotangent(41, 250, seed=11).cuda()
    k, dwx, dwy = U.dev_params(0.04, *wl.random_weights(10))
    a = shine.pipeline_bwd(img, g, k, dwx, dwy, "clamp")
    gstore = torch.zeros(41, 251, device="cuda")
    gstore[:, 1:] = g
    b = shine.pipeline_bwd(U.padded_image(img, 1), gstore[:, 1:], k, dwx, dwy, "clamp")
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_autograd_function(shine):
    img = wl.random_image(45, 140, seed=12).cuda().requires_grad_(True)
    wx, wy = wl.random_weights(12)
    k = torch.tensor([0.05], device="cuda", requires_grad=True)
    wxd = wx.cuda().requires_grad_(True)
    wyd = wy.cuda().requires_grad_(True)
    g = wl.random_cotangent(45, 140, seed=13).cuda()
    r = shine.harris(img, k, wxd, wyd, "clamp")
    (r * g).sum().backward()
    ref = cref.backward(img.detach().cpu(), g.cpu(), 0.05, wx, wy, "clamp", with_abs=True)
    assert U.rel(U.host(img.grad), ref[0]) <= U.TOL_GIMG
    U.assert_params((k.grad, wxd.grad, wyd.grad), ref[1:])
    # sum() hands an expanded cotangent to backward
    img2 = img.detach().clone().requires_grad_(True)
    shine.harris(img2, 0.05, wxd.detach(), wyd.detach(), "valid").sum().backward()
    gi2 = cref.backward(img.detach().cpu(), torch.ones(41, 136), 0.05, wx, wy, "valid")[0]
    assert U.rel(U.host(img2.grad), gi2) <= U.TOL_GIMG


def test_bounded_waits_report_no_failure(shine):
    """Every wait of the staging pipeline is bounded; a normal run must report none gave up."""
    from paper_2201_03611_b300.ops import bwd_workspace_bytes, workspace_failed
    for (h, w) in ((517, 1030), (64, 124), (3, 5)):
        img = wl.random_image(h, w, seed=1).cuda()
        g = wl.random_cotangent(h, w, seed=2).cuda()
        k, wx, wy = U.dev_params(0.04, *wl.random_weights(1))
        ws = torch.empty(bwd_workspace_bytes(h, w, "clamp"), dtype=torch.uint8, device="cuda")
        shine.pipeline_bwd(img, g, k, wx, wy, "clamp", workspace=ws)
        assert not workspace_failed(ws)


@pytest.mark.parametrize("shape,border,dtype,nbands", [((203, 517), "clamp", torch.float32, 16),
                                                       ((203, 517), "valid", torch.float32, 3),
                                                       ((96, 250), "clamp", torch.bfloat16, 5),
                                                       ((64, 130), "clamp", torch.float32, 1),
                                                       ((1030, 700), "clamp", torch.float32, 48)])
def test_host_pipeline_matches_device_calls(shine, shape, border, dtype, nbands):
    """shine_pipeline_host (host buffers, band-pipelined copies) gives the device calls' R and
    d img bit for bit, and the same parameter cotangents within the summation bound."""
    from paper_2201_03611_b300 import ops
    h, w = shape
    ho, wo = shine.output_shape(h, w, border)
    img_h = wl.random_image(h, w, seed=31).to(dtype).pin_memory()
    g_h = wl.random_cotangent(ho, wo, seed=32).to(dtype).pin_memory()
    k, wx, wy = U.dev_params(0.05, *wl.random_weights(31))
    dev_img = torch.empty(h, w, 3, dtype=dtype, device="cuda")
    dev_g = torch.empty(ho, wo, dtype=dtype, device="cuda")
    dev_out = torch.empty(ho, wo, dtype=dtype, device="cuda")
    dev_gimg = torch.empty(h, w, 3, dtype=dtype, device="cuda")
    out_h = torch.empty(ho, wo, dtype=dtype).pin_memory()
    gimg_h = torch.empty(h, w, 3, dtype=dtype).pin_memory()
    par = torch.empty(19, device="cuda")
    ws = torch.empty(ops.host_workspace_bytes(h, w, border, nbands), dtype=torch.uint8, device="cuda")
    ops.pipeline_host(img_h, g_h, k, wx, wy, dev_img, dev_g, dev_out, dev_gimg, ws, out_h=out_h, gimg_h=gimg_h,
                      grad_params=par, border=border, nbands=nbands)
    torch.cuda.synchronize()
    img, g = img_h.cuda(), g_h.cuda()
    r = shine.pipeline_fwd(img, k, wx, wy, border)
    gi, gk, gwx, gwy = shine.pipeline_bwd(img, g, k, wx, wy, border)
    assert torch.equal(out_h, r.cpu())
    assert torch.equal(gimg_h, gi.cpu())
    ref = cref.backward(img_h, g_h, 0.05, wx.cpu(), wy.cpu(), border, with_abs=True)
    U.assert_params((par[0:1], par[1:10].reshape(3, 3), par[10:19].reshape(3, 3)), ref[1:])


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("shape", [(1, 8), (3, 16), (9, 248), (37, 256), (64, 496), (130, 512), (300, 264),
                                   (5, 1024), (257, 744)])
def test_bwd_16bit_wide_path(shine, dtype, shape, wide_adjoint):
    """16-bit CLAMP images whose rows are 16-byte aligned (W a multiple of 8) take the eight-
    columns-per-lane adjoint: interior segments bulk-staged, edge segments staged per lane, ragged
    column and row tails. d img must equal, bit for bit, the four-column adjoint's (reached through
    an unaligned row pitch, same arithmetic per pixel), and everything must match the oracle on the
    quantised input."""
    h, w = shape
    img = wl.random_image(h, w, seed=h + w).to(dtype).cuda()
    g = wl.random_cotangent(h, w, seed=h * w).to(dtype).cuda()
    wx, wy = wl.random_weights(h)
    k, dwx, dwy = U.dev_params(0.05, wx, wy)
    wide = shine.pipeline_bwd(img, g, k, dwx, dwy, "clamp")
    narrow = shine.pipeline_bwd(U.padded_image(img, 1), g, k, dwx, dwy, "clamp")
    torch.cuda.synchronize()
    assert torch.equal(wide[0], narrow[0])
    ref = cref.backward(img.cpu(), g.cpu(), 0.05, wx, wy, "clamp", with_abs=True)
    assert U.rel(U.host(wide[0]), ref[0]) <= U.TOL_16
    U.assert_params(wide[1:], ref[1:])


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
@pytest.mark.parametrize("shape", [(3, 70000), (70001, 8), (2, 65536), (5, 1), (1, 131072)])
def test_extreme_aspect_ratios(shine, dtype, shape, wide_adjoint):
    """Very wide and very tall images (hundreds of column segments of a few rows each, or one
    segment of tens of thousands of rows): forward and adjoint against the oracle."""
    h, w = shape
    img = wl.random_image(h, w, seed=h + 7 * w).to(dtype)
    g = wl.random_cotangent(h, w, seed=h + 3 * w).to(dtype)
    wx, wy = wl.random_weights(w % 97)
    k, dwx, dwy = U.dev_params(0.04, wx, wy)
    tol = U.TOL_F32 if dtype == torch.float32 else U.TOL_16
    r = shine.pipeline_fwd(img.cuda(), k, dwx, dwy, "clamp")
    gi, gk, gwx, gwy = shine.pipeline_bwd(img.cuda(), g.cuda(), k, dwx, dwy, "clamp")
    torch.cuda.synchronize()
    assert U.rel(U.host(r), cref.forward(img, 0.04, wx, wy, "clamp")) <= tol
    ref = cref.backward(img, g, 0.04, wx, wy, "clamp", with_abs=True)
    assert U.rel(U.host(gi), ref[0]) <= (U.TOL_GIMG if dtype == torch.float32 else U.TOL_16)
    U.assert_params((gk, gwx, gwy), ref[1:])


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_zero_cotangent_gives_exact_zeros(shine, dtype, wide_adjoint):
    """A zero cotangent: every cotangent output is exactly zero (both adjoint kernels)."""
    for w in (256, 250):  # aligned 16-bit rows (eight-column kernel) and not
        img = wl.random_image(97, w, seed=w).to(dtype).cuda()
        g = torch.zeros(97, w, dtype=dtype, device="cuda")
        k, dwx, dwy = U.dev_params(0.04, *wl.random_weights(3))
        for t in shine.pipeline_bwd(img, g, k, dwx, dwy, "clamp"):
            assert torch.count_nonzero(t) == 0


@pytest.mark.parametrize("dtype", [torch.bfloat16, torch.float16])
def test_wide_path_with_8_byte_aligned_outputs(shine, dtype, wide_adjoint):
    """16-byte aligned image and cotangent rows take the eight-column kernel; d img (and R) rows
    that are only 8-byte aligned (260 columns: 1560-byte rows) are then written element by
    element. Same bits as the four-column kernel on an unpadded image."""
    h, w = 70, 260
    img = wl.random_image(h, w, seed=41).to(dtype)
    g = wl.random_cotangent(h, w, seed=42).to(dtype)
    k, dwx, dwy = U.dev_params(0.05, *wl.random_weights(41))
    img_a, g_a = wl.to_device(wl.padded(img), "cuda"), wl.to_device(wl.padded(g), "cuda")
    assert img_a.stride(0) * 2 % 16 == 0 and g_a.stride(0) * 2 % 16 == 0
    gi8 = torch.empty(h, w, 3, dtype=dtype, device="cuda")      # 1560-byte rows
    r8 = torch.empty(h, w, dtype=dtype, device="cuda")          # 520-byte rows
    gi_ref, *p_ref = shine.pipeline_bwd(U.padded_image(img.cuda(), 1), g.cuda(), k, dwx, dwy, "clamp")
    gi_w = shine.pipeline_bwd(img_a, g_a, k, dwx, dwy, "clamp", grad_img=gi8)[0]
    assert torch.equal(gi_w, gi_ref)
    fused = shine.pipeline_fwd_bwd(img_a, g_a, k, dwx, dwy, "clamp", out=r8, grad_img=torch.empty_like(gi8))
    assert torch.equal(fused[0], shine.pipeline_fwd(img.cuda(), k, dwx, dwy, "clamp"))
    assert torch.equal(fused[1], gi_ref)
