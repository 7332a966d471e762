"""Parity of the iterated-stencil kernel (shine_iterate_stencil: k rounds of the clamp-padded 3x3
stencil, double-buffered in shared memory per tile) with the FP64 oracle.

Tolerance (derived from the arithmetic): each round's output is a float32 chain of 9 fused
multiply-adds, so its rounding error is at most 9 u (u = 2^-24) times the sum of |tap terms|,
and the error of the round's input propagates through the stencil at most scaled by |W|. After
k rounds |got - exact| <= 9 k u S_k, with S_k = k rounds of |W| applied to |x| (the oracle's
abs-scale); the test allows 10 k u S_k.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import iterate_stencil as IS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


def _check(got, ref, scale, k):
    tol = 10 * k * 2.0 ** -24 * scale + 1e-30
    err = np.abs(np.asarray(got, np.float64) - ref)
    assert np.all(err <= tol), float((err / tol).max())


# several tiles (64 x 112) with ragged edges, single rows and columns, tiles smaller than the halo
SHAPES = [(1, 1), (1, 300), (300, 1), (5, 7), (64, 112), (65, 113), (200, 333), (131, 515)]


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("shape", SHAPES)
def test_iterate_stencil_matches_oracle(shine, k, shape):
    h, w = shape
    x, W = wl.iterate_stencil_inputs(h, w, seed=h * 7 + w + k, blur=k % 2 == 1)
    got = shine.iterate_stencil(x.cuda(), W, k).cpu().numpy()
    xd, Wd = x.double().numpy(), W.double().numpy()
    _check(got, IS.iterate_stencil_np(xd, Wd, k), IS.iterate_stencil_abs_np(xd, Wd, k), k)


def test_unaligned_pitches_and_offsets(shine):
    h, w, k = 150, 301, 4
    x, W = wl.iterate_stencil_inputs(h, w + 3, seed=21)
    xv = x.cuda()[:, 1:w + 1]                   # odd offset, pitch w + 3
    obase = torch.zeros(h, w + 2, device="cuda")
    out = obase[:, 1:w + 1]
    shine.iterate_stencil(xv, W, k, out=out)
    xd, Wd = x[:, 1:w + 1].double().numpy(), W.double().numpy()
    _check(out.cpu().numpy(), IS.iterate_stencil_np(xd, Wd, k), IS.iterate_stencil_abs_np(xd, Wd, k), k)
    assert torch.all(obase[:, 0] == 0) and torch.all(obase[:, w + 1] == 0)   # nothing outside out


def test_full_size_sampled(shine):
    """8192^2, k = 4 (the measured configuration): sampled outputs at the corners, every border,
    tile seams and random interior points, against the oracle's crop form."""
    h = w = 8192
    k = 4
    x, W = wl.iterate_stencil_inputs(h, w, seed=4)
    got = shine.iterate_stencil(x.cuda(), W, k).cpu().numpy()
    rng = np.random.default_rng(0)
    pts = [(0, 0), (0, w - 1), (h - 1, 0), (h - 1, w - 1), (1, 2), (h - 2, w - 3), (63, 111), (64, 112),
           (65, 113), (127, 223), (128, 224), (8191, 8175), (8190, 8176)]
    pts += [(int(rng.integers(h)), c) for c in (0, 1, 3, 4, w - 5, w - 1) for _ in range(4)]
    pts += [(r, int(rng.integers(w))) for r in (0, 2, 3, 4, h - 5, h - 1) for _ in range(4)]
    pts += [tuple(int(v) for v in rng.integers(0, (h, w))) for _ in range(200)]
    pts = np.array(pts)
    xd = x.double().numpy()
    ref, scale = IS.iterate_stencil_points(xd, W.double().numpy(), k, pts)
    _check(got[pts[:, 0], pts[:, 1]], ref, scale, k)


def test_repeatable_and_k1_is_one_stencil(shine):
    h, w = 257, 1030
    x, W = wl.iterate_stencil_inputs(h, w, seed=5, blur=False)
    xc = x.cuda()
    a = shine.iterate_stencil(xc, W, 6)
    b = shine.iterate_stencil(xc, W, 6)
    assert torch.equal(a, b)
    one = shine.iterate_stencil(xc, W, 1)
    assert torch.equal(one, shine.stencil2d(xc, W, border="clamp"))   # same chain, same bits


def test_argument_errors(shine):
    from paper_2201_03611_b300 import _lib as L
    x = torch.rand(16, 16, device="cuda")
    W = torch.rand(3, 3)
    for bad_k in (0, 9):
        with pytest.raises(L.ShineError):
            shine.iterate_stencil(x, W, bad_k)
    with pytest.raises(L.ShineError):
        shine.iterate_stencil(x, W, 2, out=x)   # in and out overlap
