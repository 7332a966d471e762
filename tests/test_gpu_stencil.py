"""Parity of the generalised stencil kernel (shine_stencil2d: slide2D(K, 1) + reduce, K odd) with
the FP64 oracle.

Tolerance (derived from the arithmetic): an output is a float32 chain of K*K fused multiply-adds
(separable: K down the columns, then K along the row), so |got - exact| <= n u S with u = 2^-24,
n the chain length (K*K; separable 2K) and S = sum over taps of |W x| (separable: the taps of
the outer product); a bf16 output adds its own rounding, 2^-8 |exact|.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import stencil as ST

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


def _check(got, ref, scale, n, bf16_out=False):
    tol = n * 2.0 ** -24 * scale + (2.0 ** -8 * np.abs(ref) if bf16_out else 0.0) + 1e-30
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= tol), float((err / tol).max())


SHAPES = [((37, 250), "clamp"), ((130, 300), "clamp"), ((61, 245), "valid"), ((9, 9), "valid"),
          ((1, 1), "clamp"), ((3, 517), "clamp")]


@pytest.mark.parametrize("K", [1, 3, 5, 7, 9])
@pytest.mark.parametrize("shape,border", SHAPES)
def test_stencil_matches_oracle(shine, K, shape, border):
    h, w = shape
    if border == "valid" and (h < K or w < K):
        pytest.skip("VALID needs H, W >= K")
    x, W = wl.stencil_inputs(h, w, K, seed=K * 100 + h)
    got = shine.stencil2d(x.cuda(), W, border=border).cpu().numpy()
    xd = x.double().numpy()
    _check(got, ST.stencil2d_np(xd, W.double().numpy(), border), ST.stencil_abs_np(xd, W.double().numpy(), border),
           K * K)


@pytest.mark.parametrize("K", [1, 3, 5, 9])
@pytest.mark.parametrize("shape,border", SHAPES[:3])
def test_separable_stencil_matches_oracle(shine, K, shape, border):
    h, w = shape
    x, _ = wl.stencil_inputs(h, w, K, seed=K + h)
    wv, wh = wl.separable_weights(K, seed=K)
    got = shine.stencil2d(x.cuda(), wv=wv, wh=wh, border=border).cpu().numpy()
    xd = x.double().numpy()
    ref = ST.stencil2d_sep_np(xd, wv.double().numpy(), wh.double().numpy(), border)
    scale = ST.stencil_abs_np(xd, np.outer(np.abs(wv.double().numpy()), np.abs(wh.double().numpy())), border)
    _check(got, ref, scale, 2 * K)


@pytest.mark.parametrize("out_dtype", [torch.bfloat16, torch.float32])
def test_bf16_input(shine, out_dtype):
    h, w, K = 70, 333, 5
    x, W = wl.stencil_inputs(h, w, K, seed=3)
    xq = x.to(torch.bfloat16)
    got = shine.stencil2d(xq.cuda(), W, border="clamp", out_dtype=out_dtype).float().cpu().numpy()
    xd = xq.double().numpy()
    _check(got, ST.stencil2d_np(xd, W.double().numpy(), "clamp"), ST.stencil_abs_np(xd, W.double().numpy(), "clamp"),
           K * K, bf16_out=out_dtype == torch.bfloat16)


def test_unaligned_pitches(shine):
    h, w, K = 50, 301, 7
    x, W = wl.stencil_inputs(h, w + 1, K, seed=8)
    xv = x.cuda()[:, 1:]                        # odd offset and pitch
    obase = torch.zeros(h, w + 2, device="cuda")
    out = obase[:, 1:w + 1]
    shine.stencil2d(xv, W, border="clamp", out=out)
    xd = x[:, 1:].double().numpy()
    _check(out.cpu().numpy(), ST.stencil2d_np(xd, W.double().numpy(), "clamp"),
           ST.stencil_abs_np(xd, W.double().numpy(), "clamp"), K * K)
    assert (obase[:, 0] == 0).all() and (obase[:, w + 1] == 0).all()


def test_stencil_rejects_bad_arguments(shine):
    from paper_2201_03611_b300 import _lib as L
    x = torch.empty(16, 16, device="cuda")
    o = torch.empty(16, 16, device="cuda")
    Wt = torch.ones(4, 4)
    for K in (0, 2, 11):
        assert L.lib().shine_stencil2d(x.data_ptr(), 16, 16, 16, 0, 1, K, Wt.data_ptr(), None, None, o.data_ptr(),
                                       16, 0, None) == L.SHINE_ERR_INVALID_ARG
    assert L.lib().shine_stencil2d(x.data_ptr(), 4, 16, 16, 0, 0, 5, Wt.data_ptr(), None, None, o.data_ptr(),
                                   16, 0, None) == L.SHINE_ERR_INVALID_ARG   # VALID needs H >= K
    assert L.lib().shine_stencil2d(x.data_ptr(), 16, 16, 16, 0, 1, 3, None, None, None, o.data_ptr(),
                                   16, 0, None) == L.SHINE_ERR_INVALID_ARG   # no weights at all


@pytest.mark.parametrize("K,sep", [(9, False), (9, True), (5, False)])
def test_full_size_sampled(shine, K, sep):
    """The 8192 x 8192 float32 workload of the benchmark on sampled outputs (corners, borders,
    random points)."""
    n = 8192
    x, W = wl.stencil_inputs(n, n, K, seed=0)
    pts = wl.sample_points(n, n, 1500, seed=11)
    if sep:
        wv, wh = wl.separable_weights(K, seed=0)
        got = shine.stencil2d(x.cuda(), wv=wv, wh=wh)
        Wd = np.outer(wv.double().numpy(), wh.double().numpy())
        nchain = 2 * K
    else:
        got = shine.stencil2d(x.cuda(), W)
        Wd = W.double().numpy()
        nchain = K * K
    g = got[pts[:, 0].cuda(), pts[:, 1].cuda()].cpu().numpy()
    vals, scales = ST.stencil2d_points(x.numpy(), Wd, "clamp", pts.numpy())
    _check(g, vals, scales, nchain)
