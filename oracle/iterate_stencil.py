"""iterate with a size-preserving stencil body (Sec. 6 with n = 1): k rounds of the clamp-padded
3x3 stencil, each round's output the next round's input.

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

The paper's iterate(n, m, k, body, arr) applies body k times; with n = 1 the body keeps the
length, and with body = slide2D(3, 1) after pad_clamp2D(1), then map(reduce(+, 0)) of the
window times W (a correlation), it is an iterated stencil (k blur steps for a smoothing W):

    x_0 = in,  x_{i+1} = stencil(x_i),  out = x_k

The clamp padding belongs to the body, so it is applied before every round (not once with a
k-wide pad: the two differ within k of the border).

* ``iterate_stencil``: ``patterns.iterate`` over the stencil oracle's pattern composition on
  nested lists (FP64), for small arrays.
* ``iterate_stencil_np``: the same rounds with the numpy form of the stencil oracle (any size).
* ``iterate_stencil_abs_np``: the same rounds with |W| on |in|, the scale to which k rounds of
  float32 fused multiply-add chains determine each output.
* ``iterate_stencil_points``: outputs at chosen points only, each from the crop of radius k
  around it (cut at the image border): an output depends on nothing farther than k rows or
  columns, and the positions the crop's cut edges spoil move one step inward per round, so
  after k rounds they have not reached the centre; where the crop edge is the image border the
  per-round clamp is the image's own.
"""
from __future__ import annotations

import numpy as np

from .patterns import iterate
from .stencil import stencil2d, stencil2d_np


def iterate_stencil(x, W, k: int) -> list:
    return iterate(k, lambda a: stencil2d(a, W, "clamp"), [list(map(float, row)) for row in x])


def iterate_stencil_np(x, W, k: int) -> np.ndarray:
    cur = np.asarray(x, dtype=np.float64)
    for _ in range(k):
        cur = stencil2d_np(cur, W, "clamp")
    return cur


def iterate_stencil_abs_np(x, W, k: int) -> np.ndarray:
    return iterate_stencil_np(np.abs(np.asarray(x, dtype=np.float64)), np.abs(np.asarray(W, dtype=np.float64)), k)


def iterate_stencil_points(x, W, k: int, pts):
    """(values, scales) at the points (rows of pts = (y, x)) of an (H, W) array."""
    x = np.asarray(x)
    h, w = x.shape
    vals, scales = [], []
    for y, c in np.asarray(pts):
        y0, y1 = max(0, y - k), min(h, y + k + 1)
        c0, c1 = max(0, c - k), min(w, c + k + 1)
        crop = x[y0:y1, c0:c1]
        vals.append(float(iterate_stencil_np(crop, W, k)[y - y0, c - c0]))
        scales.append(float(iterate_stencil_abs_np(crop, W, k)[y - y0, c - c0]))
    return np.array(vals), np.array(scales)
