"""Pins of the generalised stencil oracle (slide2D(K) + reduce, K odd) against facts that do not
come from the oracle itself: scipy's correlate with nearest-edge padding (a library special
case of the clamp-padded correlation), closed forms, and the Harris oracle's 3x3 stages."""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import stencil as S


def _rand(seed, *shape):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("K", [1, 3, 5, 7, 9])
@pytest.mark.parametrize("border", ["clamp", "valid"])
def test_list_form_numpy_form_and_scipy_agree(K, border):
    h, w = 11, 14
    x = _rand(K, h, w)
    W = _rand(K + 100, K, K)
    a = np.array(S.stencil2d(x.tolist(), W.tolist(), border))
    b = S.stencil2d_np(x, W, border)
    assert a.shape == b.shape == ((h, w) if border == "clamp" else (h - K + 1, w - K + 1))
    assert np.allclose(a, b, rtol=0, atol=1e-12)
    lib = ndi.correlate(x, W, mode="nearest")        # centre tap aligned with the output pixel
    r = (K - 1) // 2
    ref = lib if border == "clamp" else lib[r:h - r, r:w - r]
    assert np.allclose(b, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("K", [3, 5, 9])
@pytest.mark.parametrize("border", ["clamp", "valid"])
def test_separable_form_equals_the_outer_product_weights(K, border):
    x = _rand(7, 13, 10)
    wv, wh = _rand(8, K), _rand(9, K)
    a = np.array(S.stencil2d_sep(x.tolist(), wv.tolist(), wh.tolist(), border))
    b = S.stencil2d_sep_np(x, wv, wh, border)
    c = S.stencil2d_np(x, np.outer(wv, wh), border)
    assert np.allclose(a, b, rtol=0, atol=1e-12) and np.allclose(b, c, rtol=0, atol=1e-12)


def test_closed_forms():
    # a constant image under clamp padding gives sum(W) * c everywhere
    W = _rand(3, 5, 5)
    out = S.stencil2d_np(np.full((6, 9), 2.5), W, "clamp")
    assert np.allclose(out, 2.5 * W.sum(), rtol=0, atol=1e-12)
    # an impulse far from the border reproduces the weights (correlation: flipped footprint)
    x = np.zeros((15, 15)); x[7, 7] = 1.0
    out = S.stencil2d_np(x, W, "valid")     # output (i, j) is centred at input (i+2, j+2)
    assert np.allclose(out[3:8, 3:8], W[::-1, ::-1], rtol=0, atol=0)
    # a linear ramp under a zero-sum antisymmetric weight gives a constant slope inside
    ramp = np.tile(np.arange(12, dtype=float), (8, 1))
    Wd = np.zeros((3, 3)); Wd[1, 0], Wd[1, 2] = -1.0, 1.0
    assert np.allclose(S.stencil2d_np(ramp, Wd, "valid"), 2.0)


def test_three_tap_case_is_the_harris_sobel_stage():
    from oracle import harris as H
    x = _rand(5, 9, 12)
    W = _rand(6, 3, 3)
    ref = np.array(H.stencil3(x.tolist(), W.tolist(), "clamp"))
    assert np.allclose(S.stencil2d_np(x, W, "clamp"), ref, rtol=0, atol=1e-12)


def test_abs_scale_bounds_the_value():
    x, W = _rand(1, 10, 10), _rand(2, 7, 7)
    assert np.all(np.abs(S.stencil2d_np(x, W, "clamp")) <= S.stencil_abs_np(x, W, "clamp") + 1e-12)


@pytest.mark.parametrize("border", ["clamp", "valid"])
def test_point_form_equals_the_full_form(border):
    x, W = _rand(3, 12, 15), _rand(4, 5, 5)
    full = S.stencil2d_np(x, W, border)
    h, w = full.shape
    pts = np.array([(i, j) for i in range(h) for j in range(w)])
    vals, scales = S.stencil2d_points(x, W, border, pts)
    assert np.allclose(vals, full.reshape(-1), rtol=0, atol=1e-12)
    assert np.allclose(scales, S.stencil_abs_np(x, W, border).reshape(-1), rtol=0, atol=1e-12)
