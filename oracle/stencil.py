"""The generalised stencil: one slide2D(K, 1) + reduce stage with K x K weights, K odd.

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

    out = map(map(nbh => reduce(+, 0)(map(*)(zip(join nbh, join W)))))(slide2D(K, 1)(pad(x)))

with pad = pad_clamp2D(r) (r = (K-1)/2, output H x W) for CLAMP and no padding (output
(H-K+1) x (W-K+1)) for VALID; the weights act as a correlation, W[a][b] on window[a][b] =
x[i+a][j+b] of the padded array. The separable form is a different composition of the same
patterns: a K-tap stage down the columns with wv, then a K-tap stage along the rows with wh,
each over the clamp-padded array:

    V   = transpose(map(col => map(w => reduce(+,0)(map(*)(zip(w, wv))))(slide(K,1)(col)))(transpose(pad(x))))
    out = map(row => map(w => reduce(+,0)(map(*)(zip(w, wh))))(slide(K,1)(row)))(V)

* ``stencil2d`` / ``stencil2d_sep``: those compositions on nested lists (FP64), for small arrays.
* ``stencil2d_np`` / ``stencil2d_sep_np``: the same sums with numpy, one shifted view of the
  padded array per tap, taps in row-major order from zero (arrays of any size).
* ``stencil_abs_np``: sum over taps of |W[a][b] x| at each output, the scale to which a float32
  K x K sum is determined (the separable form: the product of the two 1-D scales).
* ``stencil2d_points``: the K x K form at chosen output points only, each as the dot product of
  its window of the padded array with the weights (for arrays too large for the full form).
"""
from __future__ import annotations

import numpy as np

from .patterns import join, map_, pad_clamp, pad_clamp2D, reduce_, slide, slide2D, transpose, zip_


def _pad(x, r: int, border: str):
    if border == "clamp":
        return pad_clamp2D(r, r, x)
    if border == "valid":
        return [list(row) for row in x]
    raise ValueError(border)


def stencil2d(x, W, border: str) -> list:
    K = len(W)
    r = (K - 1) // 2
    flatW = join(W)
    windows = slide2D(K, 1, _pad(x, r, border))
    return map_(lambda wrow: map_(lambda nbh: reduce_(lambda a, b: a + b, 0.0,
                                                      map_(lambda p: p[0] * p[1], zip_(join(nbh), flatW))), wrow),
                windows)


def stencil2d_sep(x, wv, wh, border: str) -> list:
    K = len(wv)
    r = (K - 1) // 2
    p = _pad(x, r, border)
    tap = lambda w: (lambda win: reduce_(lambda a, b: a + b, 0.0, map_(lambda q: q[0] * q[1], zip_(win, w))))
    cols = transpose(p)
    V = transpose(map_(lambda col: map_(tap(wv), slide(K, 1, col)), cols))
    return map_(lambda row: map_(tap(wh), slide(K, 1, row)), V)


def _pad_np(x, r: int, border: str):
    x = np.asarray(x, dtype=np.float64)
    if border == "clamp":
        return np.pad(x, r, mode="edge")
    if border == "valid":
        return x
    raise ValueError(border)


def stencil2d_np(x, W, border: str) -> np.ndarray:
    W = np.asarray(W, dtype=np.float64)
    K = W.shape[0]
    r = (K - 1) // 2
    p = _pad_np(x, r, border)
    ho, wo = p.shape[0] - K + 1, p.shape[1] - K + 1
    out = np.zeros((ho, wo))
    for a in range(K):
        for b in range(K):
            out = out + W[a, b] * p[a:a + ho, b:b + wo]
    return out


def stencil2d_sep_np(x, wv, wh, border: str) -> np.ndarray:
    wv = np.asarray(wv, dtype=np.float64)
    wh = np.asarray(wh, dtype=np.float64)
    K = wv.shape[0]
    r = (K - 1) // 2
    p = _pad_np(x, r, border)
    ho, wo = p.shape[0] - K + 1, p.shape[1] - K + 1
    V = np.zeros((ho, p.shape[1]))
    for a in range(K):
        V = V + wv[a] * p[a:a + ho, :]
    out = np.zeros((ho, wo))
    for b in range(K):
        out = out + wh[b] * V[:, b:b + wo]
    return out


def stencil_abs_np(x, W, border: str) -> np.ndarray:
    return stencil2d_np(np.abs(np.asarray(x, dtype=np.float64)), np.abs(np.asarray(W, dtype=np.float64)), border)


def stencil2d_points(x, W, border: str, pts) -> np.ndarray:
    """out[i][j] at the given output points (rows of pts = (i, j)); returns (value, scale)."""
    x = np.asarray(x)
    W = np.asarray(W, dtype=np.float64)
    K = W.shape[0]
    r = (K - 1) // 2
    h, w = x.shape
    vals, scales = [], []
    for i, j in np.asarray(pts):
        ci, cj = (i, j) if border == "clamp" else (i + r, j + r)   # centre in input coordinates
        rows = np.clip(np.arange(ci - r, ci + r + 1), 0, h - 1)
        cols = np.clip(np.arange(cj - r, cj + r + 1), 0, w - 1)
        win = x[np.ix_(rows, cols)].astype(np.float64)
        vals.append(float((W * win).sum()))
        scales.append(float((np.abs(W) * np.abs(win)).sum()))
    return np.array(vals), np.array(scales)
