"""Plant plausible mistakes in the pattern oracle (on the CPU) and check that the pins catch
every one of them, while the true oracle passes them all."""
import pytest

import oracle_pins as PINS
from oracle import harris as H
from oracle import patterns as P


def _resp_no_sxy(sxx, sxy, syy, kappa):
    s = H.zip2(H.zip2(sxx, sxy), syy)
    return H.map2(lambda t: t[0][0] * t[1] - kappa * (t[0][0] + t[1]) ** 2, s)


def _resp_kappa_sign(sxx, sxy, syy, kappa):
    return _orig_response(sxx, sxy, syy, -kappa)


def _stencil_convolution(x, wt, border):
    flipped = [row[::-1] for row in wt[::-1]]
    return _orig_stencil(x, flipped, border)


def _stencil_transposed(x, wt, border):
    return _orig_stencil(x, P.transpose(wt), border)


def _pad_once(x, border):
    # clamp only once (on the gray image) instead of before each stage: pad(1) here, and the
    # box stage sees an unpadded-but-same-size input by padding with zeros
    if border != H.CLAMP:
        return x
    h, w = len(x), len(x[0])
    z = [[0.0] * (w + 2)] + [[0.0] + list(r) + [0.0] for r in x] + [[0.0] * (w + 2)]
    return z


def _gray_swapped(img):
    return H.map2(lambda px: H.dot(px, (0.114, 0.587, 0.299)), img)


def _box_vjp_no_fold(g_out, h, w, border):
    g_win = H.map2(lambda gv: P.split(3, [gv] * 9), g_out)
    hp, wp = (h + 2, w + 2) if border == H.CLAMP else (h, w)
    g_pad = P.slide2D_vjp(3, 1, hp, wp, g_win)
    if border == H.CLAMP:
        return [row[1:-1] for row in g_pad[1:-1]]      # drops the clamp fold
    return g_pad


def _stencil_vjp_transposed_w(x, wt, g_out, border):
    gx, gw = _orig_stencil_vjp(x, wt, g_out, border)
    return gx, P.transpose(gw)


_orig_stencil = H.stencil3
_orig_response = H.response
_orig_stencil_vjp = H.stencil3_vjp

MUTANTS = {
    "response drops Sxy^2": [("response", _resp_no_sxy)],
    "kappa term sign": [("response", _resp_kappa_sign)],
    "convolution instead of correlation": [("stencil3", _stencil_convolution)],
    "weights transposed": [("stencil3", _stencil_transposed)],
    "zero pad instead of clamp in the box stage": [("box3", lambda x, b: _orig_box(_pad_once(x, b), "valid")
                                                    if b == H.CLAMP else _orig_box(x, b))],
    "gray coefficients swapped": [("gray", _gray_swapped)],
    "clamp fold dropped in the box adjoint": [("box3_vjp", _box_vjp_no_fold)],
    "weight gradient transposed": [("stencil3_vjp", _stencil_vjp_transposed_w)],
}
_orig_box = H.box3


def test_true_oracle_passes_every_pin():
    res = PINS.run_all(*PINS.pattern_oracle())
    assert all(not v for v in res.values()), res


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    for attr, fn in MUTANTS[name]:
        monkeypatch.setattr(H, attr, fn)
    res = PINS.run_all(*PINS.pattern_oracle())
    caught = [k for k, v in res.items() if v]
    assert caught, f"mutant '{name}' passed every pin"
