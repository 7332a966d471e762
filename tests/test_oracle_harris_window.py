"""Pins of the Gaussian-window Harris oracle: it reduces to the pinned box-window Harris oracle,
to a closed form without a window, and its window stage matches scipy's correlate1d."""
import numpy as np
import pytest
import scipy.ndimage as ndi

import workloads as wl
from oracle import harris as H
from oracle import harris_window as HW
from oracle import stencil as ST


def _img(seed, h, w):
    return wl.random_image(h, w, seed=seed).double().numpy()


def test_ones_window_of_three_is_the_box_harris():
    img = _img(1, 9, 11)
    wx, wy = [t.double().numpy() for t in wl.random_weights(1)]
    ref = np.array(H.harris(img.tolist(), 0.05, wx.tolist(), wy.tolist(), "clamp"))
    a = np.array(HW.harris_window(img.tolist(), 0.05, wx.tolist(), wy.tolist(), [1.0] * 3, [1.0] * 3))
    b = HW.harris_window_np(img, 0.05, wx, wy, np.ones(3), np.ones(3))
    assert np.allclose(a, ref, rtol=1e-12, atol=1e-9) and np.allclose(b, ref, rtol=1e-12, atol=1e-9)


def test_no_window_gives_the_rank_one_closed_form():
    img = _img(2, 7, 8)
    wx, wy = [t.double().numpy() for t in wl.sobel_weights()]
    r = HW.harris_window_np(img, 0.04, wx, wy, np.ones(1), np.ones(1))
    g = HW._gray_np(img)
    ix, iy = ST.stencil2d_np(g, wx, "clamp"), ST.stencil2d_np(g, wy, "clamp")
    assert np.allclose(r, -0.04 * (ix * ix + iy * iy) ** 2, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("K", [3, 5, 7])
def test_list_form_numpy_form_and_scipy_window_agree(K):
    img = _img(K, 10, 13)
    wx, wy = [t.double().numpy() for t in wl.random_weights(K)]
    gv, gh = [t.double().numpy() for t in wl.gaussian_window(K)]
    a = np.array(HW.harris_window(img.tolist(), 0.04, wx.tolist(), wy.tolist(), gv.tolist(), gh.tolist()))
    b = HW.harris_window_np(img, 0.04, wx, wy, gv, gh)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-9)
    g = HW._gray_np(img)
    ix, iy = ST.stencil2d_np(g, wx, "clamp"), ST.stencil2d_np(g, wy, "clamp")
    win = lambda p: ndi.correlate1d(ndi.correlate1d(p, gv, axis=0, mode="nearest"), gh, axis=1, mode="nearest")
    sxx, sxy, syy = win(ix * ix), win(ix * iy), win(iy * iy)
    assert np.allclose(b, sxx * syy - sxy * sxy - 0.04 * (sxx + syy) ** 2, rtol=1e-12, atol=1e-9)


def test_point_form_equals_the_full_form():
    img = _img(9, 20, 23)
    wx, wy = [t.double().numpy() for t in wl.random_weights(9)]
    gv, gh = [t.double().numpy() for t in wl.gaussian_window(7)]
    full = HW.harris_window_np(img, 0.04, wx, wy, gv, gh)
    pts = np.array([(i, j) for i in range(20) for j in range(23)])
    pt = HW.harris_window_points(img, 0.04, wx, wy, gv, gh, pts)
    assert np.allclose(pt, full.reshape(-1), rtol=1e-13, atol=1e-12)
