"""The paper's running example, matrix-vector multiply, as pattern compositions (FP64).

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

* ``mv``: for each row of M, zip it with x, multiply the pairs, reduce with + from 0
  (Sec. 4, the high-level MV listing).
* ``mv_opt``: the optimised form after the strategy of Sec. 4.3: split the rows into groups of
  s, map over groups and over rows in a group, and fuse the multiply into a sequential
  reduction with a private accumulator (``fuseReduceMap``), then join the groups back.
"""
from __future__ import annotations

from .patterns import fst, join, map_, reduce_, reduce_seq, snd, split, zip_


def mv(M, x):
    return map_(lambda row: reduce_(lambda a, b: a + b, 0.0,
                                    map_(lambda ax: fst(ax) * snd(ax), zip_(row, x))), M)


def mv_opt(M, x, s: int):
    def dot_seq(row):
        return reduce_seq(lambda acc, ax: acc + fst(ax) * snd(ax), 0.0, zip_(row, x))
    return join(map_(lambda rows: map_(dot_seq, rows), split(s, M)))
