"""Pins of the iterated-stencil oracle (iterate with a size-preserving body: k rounds of the
clamp-padded 3x3 stencil, Sec. 6 with n = 1) against facts that do not come from the oracle:
scipy's correlate with nearest-edge padding applied round by round, closed forms (the trinomial
spread of an iterated box blur, an iterated shift, a constant image), and the transpose
symmetry."""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import iterate_stencil as IS


def _rand(seed, *shape):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_list_form_numpy_form_and_scipy_rounds_agree(k):
    x = _rand(k, 9, 13)
    W = _rand(k + 50, 3, 3)
    a = np.array(IS.iterate_stencil(x.tolist(), W.tolist(), k))
    b = IS.iterate_stencil_np(x, W, k)
    ref = x.copy()
    for _ in range(k):
        ref = ndi.correlate(ref, W, mode="nearest")  # clamp padding before every round
    assert a.shape == b.shape == x.shape
    assert np.allclose(a, b, rtol=0, atol=1e-12)
    assert np.allclose(b, ref, rtol=0, atol=1e-11)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_iterated_box_blur_spreads_an_impulse_as_trinomial_coefficients(k):
    # ((1 + z + z^2) / 3)^k in each direction, far from the border
    t = np.array([1.0])
    for _ in range(k):
        t = np.convolve(t, np.ones(3) / 3.0)
    n = 2 * k + 7
    x = np.zeros((n, n)); x[n // 2, n // 2] = 1.0
    out = IS.iterate_stencil_np(x, np.full((3, 3), 1.0 / 9.0), k)
    c = n // 2
    assert np.allclose(out[c - k:c + k + 1, c - k:c + k + 1], np.outer(t, t), rtol=0, atol=1e-15)
    out[c - k:c + k + 1, c - k:c + k + 1] = 0.0
    assert np.all(out == 0.0)


@pytest.mark.parametrize("k", [1, 3, 5])
def test_iterated_shift_clamps_at_every_round(k):
    # W picks the left neighbour: each round moves the row right by one, repeating column 0
    x = _rand(3, 4, 9)
    W = np.zeros((3, 3)); W[1, 0] = 1.0
    out = IS.iterate_stencil_np(x, W, k)
    cols = np.maximum(np.arange(9) - k, 0)
    assert np.array_equal(out, x[:, cols])


def test_constant_image_scales_by_the_weight_sum_per_round():
    W = _rand(4, 3, 3)
    out = IS.iterate_stencil_np(np.full((7, 10), 1.5), W, 4)
    assert np.allclose(out, 1.5 * W.sum() ** 4, rtol=1e-12, atol=0)


def test_per_round_clamp_differs_from_one_wide_pad_only_near_the_border():
    # the plausible mistake: pad once by k and run k unpadded rounds
    k = 3
    x = _rand(8, 16, 16)
    W = _rand(9, 3, 3)
    good = IS.iterate_stencil_np(x, W, k)
    wrong = np.pad(x, k, mode="edge")
    for _ in range(k):
        p = wrong
        wrong = sum(W[a, b] * p[a:a + p.shape[0] - 2, b:b + p.shape[1] - 2] for a in range(3) for b in range(3))
    assert np.allclose(good[k:-k, k:-k], wrong[k:-k, k:-k], rtol=0, atol=1e-11)
    assert not np.allclose(good, wrong, rtol=0, atol=1e-6)


def test_transpose_symmetry():
    x = _rand(10, 8, 11)
    W = _rand(11, 3, 3)
    assert np.allclose(IS.iterate_stencil_np(x.T, W.T, 3), IS.iterate_stencil_np(x, W, 3).T, rtol=0, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_point_form_matches_the_full_form_everywhere_it_is_sampled(k):
    x = _rand(12 + k, 13, 17)
    W = _rand(13 + k, 3, 3)
    full = IS.iterate_stencil_np(x, W, k)
    scale = IS.iterate_stencil_abs_np(x, W, k)
    pts = np.array([(y, c) for y in range(13) for c in range(17)])
    v, s = IS.iterate_stencil_points(x, W, k, pts)
    assert np.allclose(v, full[pts[:, 0], pts[:, 1]], rtol=0, atol=1e-12)
    assert np.allclose(s, scale[pts[:, 0], pts[:, 1]], rtol=0, atol=1e-12)
