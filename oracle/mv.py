"""The paper's running example, matrix-vector multiply, as pattern compositions (FP64).

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

* ``mv``: for each row of M, zip it with x, multiply the pairs, reduce with + from 0
  (Sec. 4, the high-level MV listing).
* ``mv_opt``: the optimised form after the strategy of Sec. 4.3: split the rows into groups of
  s, map over groups and over rows in a group, and fuse the multiply into a sequential
  reduction with a private accumulator (``fuseReduceMap``), then join the groups back.
* ``mv_rows``: ``mv`` restricted to chosen rows, with the row's reduce(+) of the zipped
  products done by numpy's float64 dot (a library primitive as one step), for matrices too
  large for the list form; ``mv_abs_rows`` gives sum_j |A[i][j] x[j]| of the same rows, the
  scale to which a floating-point dot product is determined.
"""
from __future__ import annotations

import numpy as np

from .patterns import fst, join, map_, reduce_, reduce_seq, snd, split, zip_


def mv(M, x):
    return map_(lambda row: reduce_(lambda a, b: a + b, 0.0,
                                    map_(lambda ax: fst(ax) * snd(ax), zip_(row, x))), M)


def mv_opt(M, x, s: int):
    def dot_seq(row):
        return reduce_seq(lambda acc, ax: acc + fst(ax) * snd(ax), 0.0, zip_(row, x))
    return join(map_(lambda rows: map_(dot_seq, rows), split(s, M)))


def mv_rows(A, x, rows=None):
    """y[i] = sum_j A[i][j] * x[j] in float64 for the given rows (all rows if None)."""
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    sel = A if rows is None else A[np.asarray(rows)]
    return np.array([np.dot(r, x) for r in sel], dtype=np.float64)


def mv_abs_rows(A, x, rows=None):
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    sel = A if rows is None else A[np.asarray(rows)]
    return np.array([np.dot(np.abs(r), np.abs(x)) for r in sel], dtype=np.float64)
