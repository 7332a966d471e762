"""Threshold + 3x3 non-maximum suppression of a Harris response (the corner step after A5).

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

The paper does not spell out this step (it cites the corner-detection image pipeline as the
domain that the slide2D patterns serve); the reading fixed here is the plain definition

    corner(y, x)  <=>  R[y][x] > threshold  and  R[y][x] >= R[q]
                       for every 8-neighbour q of (y, x) inside the array

(neighbours outside the array are ignored; equal maxima are all kept; a NaN is never a corner).

* ``nms_loop``: the definition as nested Python loops (small arrays).
* ``nms``: the same with numpy, comparing each pixel against its 8 shifted neighbours in a
  -inf padded copy (no reordering beyond the definition: max and >= are exact).

Both take R as given: the decision is made on the values of R that are passed in, in their
own precision (float32 R stays float32 here), so that a kernel's mask can be checked bit for
bit against the definition applied to the kernel's own R.
"""
from __future__ import annotations

import numpy as np


def nms_loop(R, threshold: float) -> np.ndarray:
    R = np.asarray(R)
    h, w = R.shape
    out = np.zeros((h, w), dtype=np.uint8)
    for y in range(h):
        for x in range(w):
            v = R[y, x]
            if not v > threshold:
                continue
            keep = True
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dy == 0 and dx == 0:
                        continue
                    yy, xx = y + dy, x + dx
                    if 0 <= yy < h and 0 <= xx < w and not v >= R[yy, xx]:
                        keep = False
            out[y, x] = 1 if keep else 0
    return out


def nms(R, threshold: float) -> np.ndarray:
    R = np.asarray(R)
    h, w = R.shape
    P = np.full((h + 2, w + 2), -np.inf, dtype=R.dtype)
    P[1:-1, 1:-1] = R
    keep = R > R.dtype.type(threshold)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            keep &= R >= P[1 + dy:1 + dy + h, 1 + dx:1 + dx + w]
    return keep.astype(np.uint8)
