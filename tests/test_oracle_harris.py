"""The Harris oracle (CPU only): both oracles against the pins, against each other, and the
point-sampled forms against the full-array forms."""
import numpy as np
import pytest
import torch

import oracle_pins as PINS
import workloads as wl
from oracle import cref
from oracle import harris as H


@pytest.mark.parametrize("which", ["pattern", "c"])
@pytest.mark.parametrize("pin", sorted(PINS.ALL_PINS))
def test_pin(which, pin):
    fwd, vjp = PINS.pattern_oracle() if which == "pattern" else PINS.c_oracle()
    fails = PINS.ALL_PINS[pin](fwd, vjp)
    assert not fails, fails


SHAPES = [((1, 1), "clamp"), ((1, 7), "clamp"), ((2, 2), "clamp"), ((3, 5), "clamp"),
          ((9, 4), "clamp"), ((5, 5), "valid"), ((5, 9), "valid"), ((11, 6), "valid"),
          ((13, 17), "clamp"), ((13, 17), "valid")]


@pytest.mark.parametrize("shape,border", SHAPES)
def test_c_reference_equals_pattern_oracle(shape, border):
    h, w = shape
    img = wl.random_image(h, w, seed=h * 100 + w)
    wx, wy = wl.random_weights(h + w)
    kappa = 0.037
    r_pat = np.array(H.harris(H.to_nested(img), kappa, H.to_nested(wx), H.to_nested(wy), border))
    r_c = cref.forward(img, kappa, wx, wy, border)
    assert r_c.shape == cref.out_shape(h, w, border)
    assert PINS.rel(r_c, r_pat.reshape(r_c.shape)) <= 1e-13
    g = wl.random_cotangent(*r_c.shape, seed=7)
    gi_p, gk_p, gwx_p, gwy_p = H.harris_vjp(H.to_nested(img), kappa, H.to_nested(wx),
                                            H.to_nested(wy), border, H.to_nested(g))
    gi_c, gk_c, gwx_c, gwy_c = cref.backward(img, g, kappa, wx, wy, border)
    assert PINS.rel(gi_c, np.array(gi_p)) <= 1e-13
    assert PINS.rel([gk_c], [gk_p]) <= 1e-13
    assert PINS.rel(gwx_c, np.array(gwx_p)) <= 1e-13
    assert PINS.rel(gwy_c, np.array(gwy_p)) <= 1e-13


def test_valid_shapes_rejected():
    img = wl.random_image(4, 9, 0)
    wx, wy = wl.sobel_weights()
    with pytest.raises(ValueError):
        cref.forward(img, 0.04, wx, wy, "valid")


def test_plain_256_output_shape():
    cfg = wl.plain_256()
    wx, wy = wl.sobel_weights()
    r = cref.forward(cfg["img"], cfg["kappa"], wx, wy, cfg["border"])
    assert r.shape == (252, 252)


def test_valid_equals_clamp_interior():
    """No clamp read happens at distance >= 2 from the border, so VALID is CLAMP cropped."""
    img = wl.random_image(14, 19, 3)
    wx, wy = wl.random_weights(3)
    rv = cref.forward(img, 0.04, wx, wy, "valid")
    rc = cref.forward(img, 0.04, wx, wy, "clamp")
    assert np.array_equal(rv, rc[2:-2, 2:-2])


def test_transpose_symmetry():
    """With Wy = Wx^T, transposing the image transposes R (R is symmetric in Ix <-> Iy)."""
    img = wl.random_image(9, 12, 5)
    wx, _ = wl.random_weights(5)
    wy = wx.t().contiguous()
    for border in ("clamp", "valid"):
        r = cref.forward(img, 0.04, wx, wy, border)
        rt = cref.forward(img.transpose(0, 1).contiguous(), 0.04, wx, wy, border)
        assert PINS.rel(rt, r.T) <= 1e-13


def test_translation_equivariance():
    img = wl.random_image(20, 20, 6)
    wx, wy = wl.random_weights(6)
    r = cref.forward(img, 0.04, wx, wy, "valid")
    r2 = cref.forward(img[3:, 2:].contiguous(), 0.04, wx, wy, "valid")
    assert np.array_equal(r2, r[3:, 2:])


@pytest.mark.parametrize("shape,border", [((23, 31), "clamp"), ((23, 31), "valid"), ((1, 5), "clamp"),
                                          ((2, 3), "clamp")])
def test_point_forms_equal_full_arrays(shape, border):
    h, w = shape
    img = wl.random_image(h, w, 11)
    wx, wy = wl.random_weights(11)
    r = cref.forward(img, 0.05, wx, wy, border)
    g = wl.random_cotangent(*r.shape, seed=12)
    gimg, gk, gwx, gwy = cref.backward(img, g, 0.05, wx, wy, border)
    opts = wl.sample_points(r.shape[0], r.shape[1], 40, seed=13)
    assert np.array_equal(cref.forward_points(img, 0.05, wx, wy, border, opts), r[opts[:, 0], opts[:, 1]])
    ipts = wl.sample_points(h, w, 40, seed=14)
    bp = cref.backward_points(img, g, 0.05, wx, wy, border, ipts)
    assert PINS.rel(bp, gimg[ipts[:, 0], ipts[:, 1]]) <= 1e-13
    pk, pwx, pwy = cref.param_grads(img, g, 0.05, wx, wy, border)
    assert PINS.rel([pk], [gk]) <= 1e-13
    assert PINS.rel(pwx, gwx) <= 1e-12 and PINS.rel(pwy, gwy) <= 1e-12


def test_dkappa_closed_form():
    """dL/dkappa = -sum g (Sxx + Syy)^2, with S from the library (conv2d) pipeline."""
    img = wl.random_image(10, 13, 15)
    wx, wy = wl.random_weights(15)
    g = wl.random_cotangent(10, 13, 16)
    _, gk, _, _ = cref.backward(img, g, 0.05, wx, wy, "clamp")
    # trace of S via the library pipeline: R(kappa=0) - R(kappa=1) = (Sxx+Syy)^2
    t2 = PINS.library_harris(img, 0.0, wx.double(), wy.double(), "clamp") - \
        PINS.library_harris(img, 1.0, wx.double(), wy.double(), "clamp")
    assert abs(gk - float(-(g.double().numpy() * t2).sum())) <= 1e-10 * abs(gk)


def _direct_harris(img, kappa, wx, wy, border):
    """R by direct nested loops over each output's 5 x 5 footprint, written from the stage
    definitions (gray, 3x3 correlation, products, 3x3 box, det - kappa trace^2) with the clamp
    of each stage applied to the index it reads -- no patterns, no intermediate arrays."""
    h, w = len(img), len(img[0])
    clamp = border == "clamp"
    cy = (lambda y: min(max(y, 0), h - 1)) if clamp else (lambda y: y)
    cx = (lambda x: min(max(x, 0), w - 1)) if clamp else (lambda x: x)

    def gray(y, x):
        p = img[y][x]
        return 0.299 * p[0] + 0.587 * p[1] + 0.114 * p[2]

    def grad(y, x):  # Sobel at (y, x); its 3x3 reads clamp at the gray stage
        ix = iy = 0.0
        for a in range(3):
            for b in range(3):
                g = gray(cy(y + a - 1), cx(x + b - 1))
                ix += wx[a][b] * g
                iy += wy[a][b] * g
        return ix, iy

    out = []
    ys = range(h) if clamp else range(2, h - 2)
    xs = range(w) if clamp else range(2, w - 2)
    for y in ys:
        row = []
        for x in xs:
            sxx = sxy = syy = 0.0
            for a in (-1, 0, 1):
                for b in (-1, 0, 1):
                    ix, iy = grad(cy(y + a), cx(x + b))   # the products clamp at their own stage
                    sxx += ix * ix
                    sxy += ix * iy
                    syy += iy * iy
            row.append(sxx * syy - sxy * sxy - kappa * (sxx + syy) ** 2)
        out.append(row)
    return out


@pytest.mark.parametrize("shape,border", [((1, 1), "clamp"), ((3, 4), "clamp"), ((7, 9), "clamp"),
                                          ((16, 16), "clamp"), ((12, 5), "clamp"), ((5, 5), "valid"),
                                          ((16, 13), "valid")])
def test_brute_force_direct_formula(shape, border):
    """The pattern oracle equals a direct 5x5-footprint nested-loop formula (no patterns)."""
    h, w = shape
    img = wl.random_image(h, w, seed=h * 31 + w).double().tolist()
    wx, wy = [t.double().tolist() for t in wl.random_weights(h + 2 * w)]
    a = np.array(H.harris(img, 0.06, wx, wy, border))
    b = np.array(_direct_harris(img, 0.06, wx, wy, border))
    assert a.shape == b.shape
    assert np.max(np.abs(a - b)) <= 1e-13 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("border", ["clamp", "valid"])
def test_adjoint_dot_product_with_a_forward_difference_jvp(border):
    """<J v, g> = <v, J^T g>: the reverse pass of the pattern oracle against a central-difference
    directional derivative of its forward pass, for a direction in the image and in every
    parameter at once."""
    h, w = 8, 9
    img = wl.random_image(h, w, seed=5).double().numpy()
    wx, wy = [t.double().numpy() for t in wl.random_weights(5)]
    kappa = 0.05
    rng = np.random.default_rng(6)
    v_img, v_k = rng.standard_normal(img.shape), rng.standard_normal()
    v_wx, v_wy = rng.standard_normal((3, 3)), rng.standard_normal((3, 3))
    ho, wo = (h, w) if border == "clamp" else (h - 4, w - 4)
    g = rng.standard_normal((ho, wo))

    def R(t):
        return np.array(H.harris((img + t * v_img).tolist(), kappa + t * v_k, (wx + t * v_wx).tolist(),
                                 (wy + t * v_wy).tolist(), border))
    eps = 1e-5
    jvp = (R(eps) - R(-eps)) / (2 * eps)
    lhs = float(np.sum(jvp * g))
    d_img, d_k, d_wx, d_wy = H.harris_vjp(img.tolist(), kappa, wx.tolist(), wy.tolist(), border, g.tolist())
    rhs = float(np.sum(np.array(d_img) * v_img) + d_k * v_k + np.sum(np.array(d_wx) * v_wx)
                + np.sum(np.array(d_wy) * v_wy))
    assert abs(lhs - rhs) <= 1e-6 * max(1.0, abs(rhs))
