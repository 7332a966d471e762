"""Harris with a weighted window at A4 (the generalised stencil stage in the pipeline), FP64.

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

The pipeline of ``harris.py`` with its A4 stage -- an unweighted 3x3 box -- replaced by a
separable K-tap window (K odd): the products P_c are clamp-padded by r = (K-1)/2 at their own
stage and summed with weights gv down the columns, then gh along the rows (for example a
Gaussian window, gv = gh = normalised Gaussian taps). A1-A3 and A5 are unchanged, and so is the
per-stage clamp of A2. CLAMP borders only (output H x W).

  A4' S_c = map(row => map(w => reduce(+,0)(map(*)(zip(w, gh))))(slide(K,1)(row)))
            (transpose(map(col => map(w => reduce(+,0)(map(*)(zip(w, gv))))(slide(K,1)(col)))
            (transpose(pad_clamp2D(r)(P_c)))))

* ``harris_window``: the pattern composition on nested lists (uses ``harris`` for A1-A3, A5 and
  ``stencil.stencil2d_sep`` for A4').
* ``harris_window_np``: the same stages with numpy (arrays of any size).
* ``harris_window_points``: R at chosen pixels only, each from ``harris_window_np`` on the
  crop of radius r + 2 around it (clipped to the image, so that image borders stay borders):
  a pixel depends on inputs within r + 1 of it, so no crop boundary inside the image reaches it.
"""
from __future__ import annotations

import numpy as np

from . import harris as H
from . import stencil as ST


def harris_window(img, kappa, wx, wy, gv, gh) -> list:
    g = H.gray(img)
    ix = H.stencil3(g, wx, H.CLAMP)
    iy = H.stencil3(g, wy, H.CLAMP)
    p = H.products(ix, iy)
    planes = [H.map2(lambda t, c=c: t[c], p) for c in range(3)]
    sxx, sxy, syy = (ST.stencil2d_sep(pc, gv, gh, "clamp") for pc in planes)
    return H.response(sxx, sxy, syy, kappa)


def _gray_np(img):
    img = np.asarray(img, dtype=np.float64)
    return img[..., 0] * H.GRAY_COEF[0] + img[..., 1] * H.GRAY_COEF[1] + img[..., 2] * H.GRAY_COEF[2]


def harris_window_np(img, kappa, wx, wy, gv, gh) -> np.ndarray:
    g = _gray_np(img)
    ix = ST.stencil2d_np(g, wx, "clamp")
    iy = ST.stencil2d_np(g, wy, "clamp")
    pxx, pxy, pyy = ix * ix, ix * iy, iy * iy
    sxx, sxy, syy = (ST.stencil2d_sep_np(pc, gv, gh, "clamp") for pc in (pxx, pxy, pyy))
    return sxx * syy - sxy * sxy - kappa * (sxx + syy) ** 2


def harris_window_points(img, kappa, wx, wy, gv, gh, pts) -> np.ndarray:
    img = np.asarray(img)
    h, w = img.shape[:2]
    m = (len(gv) - 1) // 2 + 2
    out = []
    for i, j in np.asarray(pts):
        i0, i1, j0, j1 = max(i - m, 0), min(i + m + 1, h), max(j - m, 0), min(j + m + 1, w)
        r = harris_window_np(img[i0:i1, j0:j1], kappa, wx, wy, gv, gh)
        out.append(r[i - i0, j - j0])
    return np.array(out)
