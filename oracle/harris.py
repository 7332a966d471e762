"""Harris corner response written as a composition of data-parallel patterns, in FP64.

ORACLE -- test infrastructure only (see ``oracle/patterns.py`` for who may use it).

The pipeline, on an H x W x 3 image (HWC, channel fastest), with per-stage clamp padding in
CLAMP mode and no padding in VALID mode:

  A1  G  = map(map(px => reduce(+,0)(map(*)(zip(px, (0.299, 0.587, 0.114))))))(img)
  A2  Ix = map(map(nbh => reduce(+,0)(map(*)(zip(join nbh, join Wx)))))(slide2D(3,1)(pad(G)))
      Iy = same with Wy
  A3  P  = map(map((ix, iy) => (ix*ix, ix*iy, iy*iy)))(zip2D(Ix, Iy))
  A4  S  = map(map(nbh => reduce(+,0)(join nbh)))(slide2D(3,1)(pad(P_c)))   for each plane c
  A5  R  = map(map((sxx, sxy, syy) => sxx*syy - sxy*sxy - kappa*(sxx+syy)^2))(zip3(S))

``map``, ``zip`` and ``reduce`` are the RISE primitives (Sec. 4.1); the dot products are the
``zip >> map(*) >> reduce(+)`` shape of the paper's matrix-vector example (Sec. 4, MV
listing). Fusing ``map`` into ``reduce`` and ``map`` into ``map`` (the rewrite rules of
Sec. 4.2) changes no value in exact arithmetic, so this unfused composition is the definition
the fused kernels must reproduce. VALID needs H, W >= 5 and gives (H-4) x (W-4); CLAMP gives
H x W for any H, W >= 1.

The reference gradient ``harris_vjp`` is reverse mode through the same patterns, each replaced
by its adjoint: ``map`` -> pointwise chain rule, ``zip`` -> unzip, ``reduce(+)`` -> broadcast,
``join`` -> ``split``, ``slide2D`` -> overlap-add, ``pad_clamp2D`` -> fold onto the clamped
index, and a value shared by every ``map`` application (kappa, Wx, Wy) -> sum over them.
"""
from __future__ import annotations

from .patterns import (fst, join, map_, pad_clamp2D, pad_clamp2D_vjp, reduce_, slide2D,
                       slide2D_vjp, snd, split, zip_)

GRAY_COEF = (0.299, 0.587, 0.114)
VALID, CLAMP = "valid", "clamp"


def _add(a, b):
    return a + b


def dot(xs, ws):
    """zip >> map(*) >> reduce(+, 0): the dot-product shape of the MV example."""
    return reduce_(_add, 0.0, map_(lambda p: fst(p) * snd(p), zip_(xs, ws)))


def map2(f, xss):
    return map_(lambda row: map_(f, row), xss)


def zip2(xss, yss):
    return map_(lambda rows: zip_(fst(rows), snd(rows)), zip_(xss, yss))


def gray(img):
    """A1: luminance of every pixel."""
    return map2(lambda px: dot(px, GRAY_COEF), img)


def _pad(x, border):
    return pad_clamp2D(1, 1, x) if border == CLAMP else x


def stencil3(x, wt, border):
    """A2: 3x3 correlation with weights wt (slide2D + zip with the weights + reduce)."""
    w_flat = join(wt)
    return map2(lambda nbh: dot(join(nbh), w_flat), slide2D(3, 1, _pad(x, border)))


def box3(x, border):
    """A4: unnormalised 3x3 box sum (slide2D + reduce over the joined window)."""
    return map2(lambda nbh: reduce_(_add, 0.0, join(nbh)), slide2D(3, 1, _pad(x, border)))


def products(ix, iy):
    """A3: the structure-tensor entries (Ix^2, Ix*Iy, Iy^2)."""
    return map2(lambda t: (t[0] * t[0], t[0] * t[1], t[1] * t[1]), zip2(ix, iy))


def response(sxx, sxy, syy, kappa):
    """A5: det - kappa * trace^2 of the summed structure tensor."""
    s = zip2(zip2(sxx, sxy), syy)
    return map2(lambda t: (t[0][0] * t[1] - t[0][1] * t[0][1]
                           - kappa * (t[0][0] + t[1]) * (t[0][0] + t[1])), s)


def harris_stages(img, kappa, wx, wy, border):
    """Every intermediate of A1-A5, for the reverse pass and for stage-level tests."""
    if border not in (VALID, CLAMP):
        raise ValueError(border)
    g = gray(img)
    ix = stencil3(g, wx, border)
    iy = stencil3(g, wy, border)
    p = products(ix, iy)
    pxx = map2(lambda t: t[0], p)
    pxy = map2(lambda t: t[1], p)
    pyy = map2(lambda t: t[2], p)
    sxx, sxy, syy = box3(pxx, border), box3(pxy, border), box3(pyy, border)
    r = response(sxx, sxy, syy, kappa)
    return dict(G=g, Ix=ix, Iy=iy, Pxx=pxx, Pxy=pxy, Pyy=pyy, Sxx=sxx, Sxy=sxy, Syy=syy, R=r)


def harris(img, kappa, wx, wy, border):
    """R for one image; img is a nested list [H][W][3] of floats, wx/wy nested [3][3]."""
    return harris_stages(img, kappa, wx, wy, border)["R"]


# --------------------------------------------------------------------------------------------
# Reverse mode
# --------------------------------------------------------------------------------------------

def _unpad_vjp(g_padded, h, w, border):
    return pad_clamp2D_vjp(1, 1, h, w, g_padded) if border == CLAMP else g_padded


def box3_vjp(g_out, h, w, border):
    """Adjoint of box3: reduce(+) broadcasts, join -> split(3), then slide2D and pad adjoints."""
    g_win = map2(lambda gv: split(3, [gv] * 9), g_out)
    hp, wp = (h + 2, w + 2) if border == CLAMP else (h, w)
    return _unpad_vjp(slide2D_vjp(3, 1, hp, wp, g_win), h, w, border)


def stencil3_vjp(x, wt, g_out, border):
    """Adjoint of stencil3 with respect to its input x and to the shared weights wt."""
    h, w = len(x), len(x[0])
    w_flat = join(wt)
    g_win = map2(lambda gv: split(3, [gv * wf for wf in w_flat]), g_out)
    hp, wp = (h + 2, w + 2) if border == CLAMP else (h, w)
    gx = _unpad_vjp(slide2D_vjp(3, 1, hp, wp, g_win), h, w, border)
    # wt is closed over by every map application: its cotangent is the sum over all windows.
    windows = slide2D(3, 1, _pad(x, border))
    per_window = map2(lambda pair: [fst(pair) * v for v in join(snd(pair))],
                      zip2(g_out, windows))
    g_wt_flat = reduce_(lambda acc, v: [a + b for a, b in zip(acc, v)], [0.0] * 9,
                        join(per_window))
    return gx, split(3, g_wt_flat)


def harris_vjp(img, kappa, wx, wy, border, g):
    """Cotangents (d img [H][W][3], d kappa, d Wx [3][3], d Wy [3][3]) of L = sum(g * R)."""
    st = harris_stages(img, kappa, wx, wy, border)
    h, w = len(img), len(img[0])
    sxx, sxy, syy = st["Sxx"], st["Sxy"], st["Syy"]
    # A5 adjoint (pointwise chain over zip3; kappa is shared, so its cotangent is a sum).
    trio = zip2(zip2(zip2(sxx, sxy), syy), g)

    def local(t):
        (((a, b), c), gv) = t
        tr = a + c
        return (gv * (c - 2.0 * kappa * tr), -2.0 * gv * b, gv * (a - 2.0 * kappa * tr),
                -gv * tr * tr)
    loc = map2(local, trio)
    g_sxx = map2(lambda t: t[0], loc)
    g_sxy = map2(lambda t: t[1], loc)
    g_syy = map2(lambda t: t[2], loc)
    g_kappa = reduce_(_add, 0.0, join(map2(lambda t: t[3], loc)))
    # A4 adjoint.
    hi, wi = len(st["Ix"]), len(st["Ix"][0])
    g_pxx = box3_vjp(g_sxx, hi, wi, border)
    g_pxy = box3_vjp(g_sxy, hi, wi, border)
    g_pyy = box3_vjp(g_syy, hi, wi, border)
    # A3 adjoint (products -> unzip).
    q = zip2(zip2(zip2(st["Ix"], st["Iy"]), zip2(g_pxx, g_pxy)), g_pyy)
    g_i = map2(lambda t: (2.0 * t[0][0][0] * t[0][1][0] + t[0][0][1] * t[0][1][1],
                          t[0][0][0] * t[0][1][1] + 2.0 * t[0][0][1] * t[1]), q)
    g_ix = map2(lambda t: t[0], g_i)
    g_iy = map2(lambda t: t[1], g_i)
    # A2 adjoint.
    g_gx, g_wx = stencil3_vjp(st["G"], wx, g_ix, border)
    g_gy, g_wy = stencil3_vjp(st["G"], wy, g_iy, border)
    g_g = map2(lambda t: t[0] + t[1], zip2(g_gx, g_gy))
    # A1 adjoint.
    g_img = map2(lambda gv: [gv * c for c in GRAY_COEF], g_g)
    assert len(g_img) == h and len(g_img[0]) == w
    return g_img, g_kappa, g_wx, g_wy


# --------------------------------------------------------------------------------------------
# Conversions for tests (torch / numpy arrays <-> nested lists of Python floats)
# --------------------------------------------------------------------------------------------

def to_nested(a):
    """Any array-like with .tolist() (or nested sequence) -> nested lists of Python floats."""
    if hasattr(a, "double"):
        a = a.double()
    if hasattr(a, "tolist"):
        return a.tolist()
    return [to_nested(x) for x in a]
