"""iterate with a summing body (Sec. 6): k rounds of split(n) >> map(reduce(+, 0)).

ORACLE -- test infrastructure only (see ``oracle/__init__.py``).

The paper's iterate repeatedly applies a body that shrinks its input by a factor n, passing
each round's output to the next, over Array[(n^k) m] to Array[m]; with the body
split(n) >> map(reduce(+, 0)) every output is the level-by-level tree sum of n^k consecutive
inputs, each round a left fold from 0 of every n consecutive values.

* ``iterate_sum``: the pattern composition itself (``patterns.iterate``, ``split``, ``map_``,
  ``reduce_``) on lists, FP64 (or whatever number type the inputs carry).
* ``iterate_sum_np``: the same rounds on numpy arrays in a chosen dtype: each round views the
  values as rows of n and folds the columns left to right from 0. In float64 it is the
  reference; in float32 it fixes the float32 value of the definition (the order of every
  addition is the pattern's), against which a float32 kernel is checked bit for bit.
* ``tree_bound``: sum |x| * k (n-1) eps, the first-order error bound of such a tree sum.
* ``iterate_fold`` / ``iterate_fold_np``: the same iterate with the body
  split(n) >> map(reduce(op, identity)) for op max (from -inf) or min (from +inf), with the
  IEEE maxNum / minNum reading (a NaN operand is ignored unless both are NaN).
"""
from __future__ import annotations

import numpy as np

from .patterns import iterate, map_, reduce_, split


def iterate_sum(xs, n: int, k: int) -> list:
    body = lambda arr: map_(lambda chunk: reduce_(lambda a, b: a + b, 0.0, chunk), split(n, arr))
    return iterate(k, body, list(xs))


def iterate_sum_np(x, n: int, k: int, dtype=np.float64) -> np.ndarray:
    cur = np.asarray(x, dtype=dtype)
    for _ in range(k):
        rows = cur.reshape(-1, n)
        s = np.zeros(rows.shape[0], dtype=dtype)
        for e in range(n):
            s = s + rows[:, e]
        cur = s
    return cur


def tree_bound(x, n: int, k: int, eps: float) -> np.ndarray:
    """Per output: k (n - 1) eps * sum |x| over its n^k inputs."""
    a = np.abs(np.asarray(x, dtype=np.float64)).reshape(-1, n ** k).sum(axis=1)
    return k * max(n - 1, 0) * eps * a


_FOLD = {"max": (lambda a, b: b if a != a else (a if b != b else max(a, b)), float("-inf")),
         "min": (lambda a, b: b if a != a else (a if b != b else min(a, b)), float("inf"))}


def iterate_fold(xs, n: int, k: int, op: str) -> list:
    f, ident = _FOLD[op]
    body = lambda arr: map_(lambda chunk: reduce_(f, ident, chunk), split(n, arr))
    return iterate(k, body, list(xs))


def iterate_fold_np(x, n: int, k: int, op: str, dtype=np.float64) -> np.ndarray:
    g = np.fmax if op == "max" else np.fmin
    ident = -np.inf if op == "max" else np.inf
    cur = np.asarray(x, dtype=dtype)
    for _ in range(k):
        rows = cur.reshape(-1, n)
        s = np.full(rows.shape[0], ident, dtype=dtype)
        for e in range(n):
            s = g(s, rows[:, e])
        cur = s
    return cur
