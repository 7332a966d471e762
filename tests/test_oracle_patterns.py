"""Pattern semantics of the oracle (CPU only): shapes, definitions, rewrite rules, MV, iterate.

The pins here are facts the paper or plain mathematics fixes, not re-statements of the code:
primitive types (Sec. 4.1 and Sec. 5.1), the three algorithmic rewrite rules of Sec. 4.2 as
equalities, the MV example of Sec. 4 against a plain double loop and numpy, the iterate typing
of Sec. 6, and adjoint identities for the linear patterns.
"""
import math
import random

import numpy as np
import pytest

from oracle import patterns as P
from oracle import mv as MV


def test_map_keeps_length_and_order():
    xs = [3.0, 1.0, 2.0]
    assert P.map_(lambda v: v * 2, xs) == [6.0, 2.0, 4.0]
    assert P.map_(lambda v: v, []) == []


def test_zip_requires_equal_lengths():
    assert P.zip_([1, 2], [3, 4]) == [(1, 3), (2, 4)]
    with pytest.raises(ValueError):
        P.zip_([1, 2], [3])


def test_reduce_is_a_left_fold():
    # a non-commutative, non-associative operator exposes the fold order
    assert P.reduce_(lambda a, b: f"({a}{b})", "z", ["1", "2", "3"]) == "(((z1)2)3)"
    assert P.reduce_seq(lambda a, b: f"({a}{b})", "z", ["1", "2", "3"]) == "(((z1)2)3)"
    assert P.reduce_(lambda a, b: a + b, 0.0, []) == 0.0


def test_split_join_types():
    xs = list(range(12))
    s = P.split(4, xs)                       # Array[4*3] -> Array[3, Array[4]]
    assert len(s) == 3 and all(len(c) == 4 for c in s)
    assert s[1] == [4, 5, 6, 7]
    assert P.join(s) == xs                   # join . split = id
    assert P.split(4, P.join(s)) == s        # split . join = id
    with pytest.raises(ValueError):
        P.split(5, xs)


def test_slide_lengths_and_windows():
    xs = list(range(10))
    w = P.slide(3, 1, xs)
    assert len(w) == 10 - 3 + 1
    assert w[4] == [4, 5, 6]
    w2 = P.slide(3, 2, list(range(9)))      # s*n + k - s = 9 -> n = 4
    assert len(w2) == 4 and w2[3] == [6, 7, 8]
    # two valid 3x3 stages shrink 256 -> 254 -> 252 (the plain 256x256 workload)
    assert len(P.slide(3, 1, list(range(256)))) == 254
    assert len(P.slide(3, 1, list(range(254)))) == 252


def test_slide2D_window_contents():
    h, w = 5, 6
    x = [[10 * i + j for j in range(w)] for i in range(h)]
    win = P.slide2D(3, 1, x)
    assert len(win) == h - 2 and len(win[0]) == w - 2
    for i in range(h - 2):
        for j in range(w - 2):
            for a in range(3):
                for b in range(3):
                    assert win[i][j][a][b] == x[i + a][j + b]


def test_pad_clamp():
    xs = [5, 6, 7]
    assert P.pad_clamp(2, 1, xs) == [5, 5, 5, 6, 7, 7]
    assert P.pad_clamp(1, 1, [9]) == [9, 9, 9]
    x2 = P.pad_clamp2D(1, 1, [[1, 2], [3, 4]])
    assert x2 == [[1, 1, 2, 2], [1, 1, 2, 2], [3, 3, 4, 4], [3, 3, 4, 4]]


def test_transpose_involution():
    x = [[1, 2, 3], [4, 5, 6]]
    assert P.transpose(x) == [[1, 4], [2, 5], [3, 6]]
    assert P.transpose(P.transpose(x)) == x


def test_rewrite_rules_are_equalities():
    """Sec. 4.2: split-join, map fusion and fuseReduceMap preserve the value."""
    rng = random.Random(0)
    xs = [rng.uniform(-1, 1) for _ in range(24)]
    f = lambda v: 3.0 * v - 1.0
    g = lambda v: v * v
    # map(f) == split(n) >> map(map(f)) >> join        (exact: a permutation of the same work)
    assert P.map_(f, xs) == P.join(P.map_(lambda c: P.map_(f, c), P.split(6, xs)))
    # map(f) >> map(g) == map(f >> g)                  (exact)
    assert P.map_(g, P.map_(f, xs)) == P.map_(lambda v: g(f(v)), xs)
    # map(f) >> reduce(+, init) == reduceSeq(acc + f(y), init)   (exact: same fold order)
    assert P.reduce_(lambda a, b: a + b, 0.5, P.map_(f, xs)) == \
        P.reduce_seq(lambda acc, y: acc + f(y), 0.5, xs)


def test_reduce_associativity_within_rounding():
    """reduce's parallel reading assumes associativity: left, right and tree folds of + agree
    within the FP64 rounding bound (n-1) * eps * sum|x|."""
    rng = random.Random(1)
    xs = [rng.uniform(-1, 1) for _ in range(1000)]
    left = P.reduce_(lambda a, b: a + b, 0.0, xs)
    right = P.reduce_(lambda a, b: a + b, 0.0, xs[::-1])

    def tree(v):
        return v[0] if len(v) == 1 else tree(v[:len(v) // 2]) + tree(v[len(v) // 2:])
    bound = (len(xs) - 1) * 2.0 ** -53 * sum(abs(v) for v in xs)
    exact = math.fsum(xs)
    for s in (left, right, tree(xs)):
        assert abs(s - exact) <= bound


def test_mv_example_against_a_double_loop_and_numpy():
    """Sec. 4: mv and the optimised mvOpt compute y_i = sum_j M[i][j] x[j]."""
    rng = np.random.default_rng(3)
    n, m, s = 12, 7, 4
    M = rng.standard_normal((n, m))
    x = rng.standard_normal(m)
    y_hi = MV.mv(M.tolist(), x.tolist())
    y_opt = MV.mv_opt(M.tolist(), x.tolist(), s)
    loop = [sum(M[i][j] * x[j] for j in range(m)) for i in range(n)]
    assert y_hi == y_opt          # same fold order and operations -> bit-identical
    assert np.allclose(y_hi, loop, rtol=0, atol=1e-14)
    assert np.allclose(y_hi, M @ x, rtol=0, atol=1e-13)
    with pytest.raises(ValueError):
        MV.mv_opt(M.tolist(), x.tolist(), 5)     # split(5) of 12 rows is ill-typed


def test_mv_rows_equals_the_pattern_form():
    """The row-sampled MV (numpy dot as the row reduction) equals the list form of Sec. 4 to
    FP64 rounding, on every row and on a chosen subset, and its scale is sum |a x|."""
    rng = np.random.default_rng(11)
    n, m = 9, 33
    M = rng.standard_normal((n, m))
    x = rng.standard_normal(m)
    y = MV.mv(M.tolist(), x.tolist())
    scale = np.abs(M) @ np.abs(x)
    assert np.all(np.abs(MV.mv_rows(M, x) - y) <= 64 * 2.0 ** -53 * scale)
    rows = [7, 0, 3]
    assert np.array_equal(MV.mv_rows(M, x, rows), MV.mv_rows(M, x)[rows])
    assert np.allclose(MV.mv_abs_rows(M, x, rows), scale[rows], rtol=1e-15, atol=0)
    # closed forms: a row of ones against x sums x; a zero vector gives zeros
    ones = np.ones((2, m))
    assert np.allclose(MV.mv_rows(ones, x), [math.fsum(x)] * 2, rtol=0, atol=1e-14)
    assert np.array_equal(MV.mv_rows(M, np.zeros(m)), np.zeros(n))


def test_iterate_typing_and_value():
    """Sec. 6: iterate over Array[(n^k)*m] with a body that shrinks by n gives Array[m]."""
    n, k, m = 2, 3, 5
    xs = [float(i) for i in range(n ** k * m)]
    body = lambda arr: P.map_(lambda c: P.reduce_(lambda a, b: a + b, 0.0, c), P.split(n, arr))
    out = P.iterate(k, body, xs)
    assert len(out) == m
    # each output sums n^k consecutive inputs
    assert out == [sum(xs[i * n ** k:(i + 1) * n ** k]) for i in range(m)]


def _dot(a, b):
    return float(np.sum(np.asarray(a, np.float64) * np.asarray(b, np.float64)))


def test_adjoints_satisfy_the_dot_product_identity():
    """<A x, y> = <x, A^T y> for slide, slide2D and pad_clamp2D (their adjoints are the
    overlap-add and the clamp fold)."""
    rng = np.random.default_rng(4)
    x1 = rng.standard_normal(11).tolist()
    y1 = rng.standard_normal((9, 3)).tolist()
    assert abs(_dot(P.slide(3, 1, x1), y1) - _dot(x1, P.slide_vjp(3, 1, 11, y1, 0.0))) < 1e-12
    h, w = 6, 7
    x2 = rng.standard_normal((h, w)).tolist()
    y2 = rng.standard_normal((h - 2, w - 2, 3, 3)).tolist()
    assert abs(_dot(P.slide2D(3, 1, x2), y2) - _dot(x2, P.slide2D_vjp(3, 1, h, w, y2))) < 1e-12
    y3 = rng.standard_normal((h + 2, w + 2)).tolist()
    assert abs(_dot(P.pad_clamp2D(1, 1, x2), y3) - _dot(x2, P.pad_clamp2D_vjp(1, 1, h, w, y3))) < 1e-12


def test_iterate_sum_forms_agree_and_fix_the_tree():
    """Sec. 6 with the summing body: the numpy rounds equal the pattern composition bit for
    bit in float64 (same additions in the same order), every output is its group's tree sum,
    and all-ones inputs give n^k exactly."""
    from oracle import iterate_sum as IT
    rng = np.random.default_rng(4)
    for n, k, m in ((2, 3, 5), (3, 2, 4), (4, 3, 2), (5, 1, 7), (2, 0, 3)):
        x = rng.standard_normal(n ** k * m)
        a = IT.iterate_sum(x.tolist(), n, k)
        b = IT.iterate_sum_np(x, n, k)
        assert len(a) == m and np.array_equal(np.array(a), b)
        exact = [math.fsum(x[j * n ** k:(j + 1) * n ** k]) for j in range(m)]
        assert np.all(np.abs(b - exact) <= IT.tree_bound(x, n, k, 2.0 ** -53) + 1e-300)
        assert np.array_equal(IT.iterate_sum_np(np.ones(n ** k * m), n, k), np.full(m, float(n ** k)))
    # float32 rounds: the fold order matters, and the numpy form keeps the pattern's order
    x32 = np.array([1.0, 2.0 ** -24, 2.0 ** -24, 2.0 ** -24], dtype=np.float32)
    left = IT.iterate_sum_np(x32, 4, 1, np.float32)[0]
    assert left == np.float32(1.0)                       # ((1 + e) + e) + e rounds back to 1
    assert IT.iterate_sum_np(x32, 2, 2, np.float32)[0] == np.float32(1.0) + np.float32(2.0 ** -23)


def test_iterate_max_and_min_forms_agree_and_equal_the_group_extrema():
    """Sec. 6 with max / min bodies: the list form and the numpy form agree exactly, each output
    is its group's extremum, and a NaN operand is ignored (maxNum / minNum)."""
    from oracle import iterate_sum as IT
    rng = np.random.default_rng(8)
    for n, k, m in ((2, 3, 5), (3, 2, 4), (4, 1, 3)):
        x = rng.standard_normal(n ** k * m)
        for op, ref in (("max", np.max), ("min", np.min)):
            a = IT.iterate_fold(x.tolist(), n, k, op)
            b = IT.iterate_fold_np(x, n, k, op)
            assert np.array_equal(np.array(a), b)
            assert np.array_equal(b, ref(x.reshape(m, -1), axis=1))
    x = np.array([1.0, np.nan, -2.0, 0.5])
    assert IT.iterate_fold(x.tolist(), 2, 2, "max") == [1.0]
    assert IT.iterate_fold_np(x, 2, 2, "min")[0] == -2.0
