"""Data-parallel pattern semantics evaluated on nested Python lists in FP64.

ORACLE -- test infrastructure only. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import, call or run anything under ``oracle/``; the product
path (the CUDA library and its Python binding) never does.

Each function is the plain definition of one pattern, with no blocking, fusion or reordering.
Arrays are Python lists; a tuple value is a Python tuple; scalars are Python floats (FP64).

Where the definitions come from:

* ``map``, ``reduce``, ``zip``: the high-level RISE primitives (Sec. 4.1, the listing of
  functional data-parallel primitives): ``map: (s->t) -> Array[n,s] -> Array[n,t]``,
  ``reduce: (t->t->t) -> t -> Array[n,t] -> t``, ``zip: Array[n,s] -> Array[n,t] ->
  Array[n,(s,t)]``.
* ``reduce_seq``: the sequential fold ``reduceSeq`` (Sec. 4.3 and the DPIA functional
  primitives of Sec. 5.1): an accumulator initialised with ``init`` and updated once per
  element in index order.
* ``split``, ``join``, ``fst``, ``snd``, ``idx``: the DPIA functional primitives (Sec. 5.1):
  ``split(n): Array[n*m,t] -> Array[m, Array[n,t]]`` and ``join`` its inverse.
* ``iterate``: the extension primitive of Sec. 6 (``iterate(n, m, k, body)``: apply ``body``
  k times, each application shrinking the array by a factor n).
* ``slide``, ``slide2D``, ``pad_clamp``, ``transpose`` are not defined in the paper (it only
  cites the stencil work that introduced them); they take their standard meaning, fixed here:
  ``slide(k, s)`` makes the windows ``x[i*s : i*s+k]``, ``pad_clamp(l, r)`` reads index
  ``clamp(i - l, 0, n-1)``, ``slide2D = map(slide) >> slide >> map(transpose)``.
"""
from __future__ import annotations

from typing import Callable, Sequence


def map_(f: Callable, xs: Sequence) -> list:
    """map(f)(xs): apply f to every element; length is kept."""
    return [f(x) for x in xs]


def zip_(xs: Sequence, ys: Sequence) -> list:
    """zip(xs)(ys): pairs of equal-index elements; both arrays must have the same length n."""
    if len(xs) != len(ys):
        raise ValueError(f"zip of arrays of lengths {len(xs)} and {len(ys)}")
    return [(xs[i], ys[i]) for i in range(len(xs))]


def reduce_(f: Callable, init, xs: Sequence):
    """reduce(f)(init)(xs) as a left fold f(...f(f(init, x0), x1)..., x_{n-1}).

    The parallel reading of ``reduce`` assumes f associative (Sec. 4.2: the fused reduction
    "can no longer be parallelized" once f is not); for such f every bracketing gives the
    same value, and the left fold is the one the oracle fixes."""
    acc = init
    for x in xs:
        acc = f(acc, x)
    return acc


def reduce_seq(f: Callable, init, xs: Sequence):
    """reduceSeq: the sequential fold with an accumulator (Sec. 4.3, Sec. 5.1)."""
    acc = init
    for i in range(len(xs)):
        acc = f(acc, xs[i])
    return acc


def split(n: int, xs: Sequence) -> list:
    """split(n): Array[n*m, t] -> Array[m, Array[n, t]] (chunks of n consecutive elements)."""
    if n <= 0 or len(xs) % n != 0:
        raise ValueError(f"split({n}) of an array of length {len(xs)}")
    return [list(xs[i:i + n]) for i in range(0, len(xs), n)]


def join(xss: Sequence[Sequence]) -> list:
    """join: Array[m, Array[n, t]] -> Array[m*n, t] (concatenation in order)."""
    out = []
    for xs in xss:
        out.extend(xs)
    return out


def fst(p):
    return p[0]


def snd(p):
    return p[1]


def idx(i: int, xs: Sequence):
    """idx(i, arr): element i of an array of length n, 0 <= i < n."""
    if not 0 <= i < len(xs):
        raise IndexError(f"idx {i} of an array of length {len(xs)}")
    return xs[i]


def transpose(xss: Sequence[Sequence]) -> list:
    """transpose: Array[n, Array[m, t]] -> Array[m, Array[n, t]], out[j][i] = in[i][j]."""
    if len(xss) == 0:
        return []
    m = len(xss[0])
    return [[xss[i][j] for i in range(len(xss))] for j in range(m)]


def slide(k: int, s: int, xs: Sequence) -> list:
    """slide(k, s): Array[s*n + k - s, t] -> Array[n, Array[k, t]], window i = xs[i*s : i*s+k].

    For step 1 an array of length N gives N - k + 1 windows."""
    if k <= 0 or s <= 0 or len(xs) < k or (len(xs) - k) % s != 0:
        raise ValueError(f"slide({k},{s}) of an array of length {len(xs)}")
    n = (len(xs) - k) // s + 1
    return [list(xs[i * s:i * s + k]) for i in range(n)]


def pad_clamp(l: int, r: int, xs: Sequence) -> list:
    """pad_clamp(l, r): Array[n, t] -> Array[l + n + r, t], element i reads xs[clamp(i-l, 0, n-1)]."""
    n = len(xs)
    if n == 0:
        raise ValueError("pad_clamp of an empty array")
    return [xs[min(max(i - l, 0), n - 1)] for i in range(l + n + r)]


def slide2D(k: int, s: int, xss: Sequence[Sequence]) -> list:
    """slide2D(k, s) = map(slide(k, s)) >> slide(k, s) >> map(transpose).

    Window (i, j) is the k x k block with window[a][b] = xss[i*s + a][j*s + b]."""
    rows_windowed = map_(lambda row: slide(k, s, row), xss)        # [H][nw][k]
    blocks = slide(k, s, rows_windowed)                              # [nh][k][nw][k]
    return map_(transpose, blocks)                                   # [nh][nw][k][k]


def pad_clamp2D(l: int, r: int, xss: Sequence[Sequence]) -> list:
    """pad_clamp on both axes: map(pad_clamp(l, r)) >> pad_clamp(l, r)."""
    return pad_clamp(l, r, map_(lambda row: pad_clamp(l, r, row), xss))


def iterate(k: int, body: Callable, xs: Sequence) -> list:
    """iterate(k, body): apply body k times, feeding each output to the next step (Sec. 6)."""
    cur = list(xs)
    for _ in range(k):
        cur = body(cur)
    return cur


# ---------------------------------------------------------------------------------------------
# Adjoints (vector-Jacobian products) of the linear patterns, used by the oracle's reference
# gradient. Each takes the cotangent of the pattern's output and returns the cotangent of its
# input; all are the transposes of the definitions above.
# ---------------------------------------------------------------------------------------------

def zeros_like(x):
    if isinstance(x, (list, tuple)):
        return [zeros_like(e) for e in x]
    return 0.0


def add_into(acc, g):
    """acc += g, elementwise over nested lists (returns the new value)."""
    if isinstance(acc, list):
        return [add_into(a, b) for a, b in zip(acc, g)]
    return acc + g


def slide_vjp(k: int, s: int, n_in: int, g_windows: Sequence, zero) -> list:
    """Transpose of slide(k, s): overlap-add every window cotangent back onto its elements."""
    g = [zeros_like(zero) for _ in range(n_in)]
    for i, win in enumerate(g_windows):
        for a in range(k):
            g[i * s + a] = add_into(g[i * s + a], win[a])
    return g


def transpose_vjp(g: Sequence[Sequence]) -> list:
    """Transpose is a permutation, so its adjoint is transpose again."""
    return transpose(g)


def slide2D_vjp(k: int, s: int, h_in: int, w_in: int, g_windows: Sequence) -> list:
    """Adjoint of slide2D = map(slide) >> slide >> map(transpose), taken in reverse order."""
    g_blocks = map_(transpose_vjp, g_windows)                                  # [nh][k][nw][k]
    nw = len(g_windows[0]) if g_windows else 0
    zero_row = [[0.0] * k for _ in range(nw)]
    g_rows_windowed = slide_vjp(k, s, h_in, g_blocks, zero_row)                 # [H][nw][k]
    return map_(lambda gr: slide_vjp(k, s, w_in, gr, 0.0), g_rows_windowed)    # [H][W]


def pad_clamp_vjp(l: int, r: int, n: int, g_padded: Sequence, zero) -> list:
    """Adjoint of pad_clamp: each padded cotangent is added onto the index it was read from."""
    g = [zeros_like(zero) for _ in range(n)]
    for i, gi in enumerate(g_padded):
        j = min(max(i - l, 0), n - 1)
        g[j] = add_into(g[j], gi)
    return g


def pad_clamp2D_vjp(l: int, r: int, h: int, w: int, g_padded: Sequence[Sequence]) -> list:
    """Adjoint of pad_clamp2D = map(pad_clamp) >> pad_clamp, taken in reverse order."""
    g_rows = pad_clamp_vjp(l, r, h, g_padded, [0.0] * (w + l + r))
    return map_(lambda gr: pad_clamp_vjp(l, r, w, gr, 0.0), g_rows)
