"""Checks that pin the oracle to facts other than itself.

Each pin takes an oracle given as two callables,

  fwd(img, kappa, wx, wy, border) -> R (numpy float64)
  vjp(img, g, kappa, wx, wy, border) -> (d img, d kappa, d wx, d wy)

and returns a list of failure messages (empty when the pin holds). The pins are:

* ``golden``        hand-derived worked examples in tests/golden/ (impulse, step edge);
* ``ramp``          closed form on a linear ramp: det = 0 and R = -kappa (576 (a^2+b^2))^2;
* ``constant``      R == 0 exactly on a constant image (the Sobel rows sum to 0);
* ``library``       torch.nn.functional.conv2d in float64 (a correlation) with replicate
                    padding before each stage, on random images and non-symmetric weights;
* ``homogeneity``   R(2 img) == 16 R(img) exactly (scaling by 2 is exact in binary FP);
* ``fd``            the reverse-mode gradient against FP64 central differences;
* ``euler``         degree-4 homogeneity: sum(img * d img) = 4 L and sum(W * d W) = 4 L.

They are chosen so that each plausible mistake (a dropped term, a flipped sign, a transposed
or flipped operand, a wrong padding or fold) fails at least one; tests/test_oracle_mutants.py
plants such mistakes and checks exactly that.
"""
from __future__ import annotations

import os

import numpy as np
import torch
import torch.nn.functional as F

import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = [s.strip() for s in line.split("=", 1)]
            vals[k] = v
    return vals


def rel(a, b) -> float:
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    den = max(np.abs(b).max(initial=0.0), 1e-300)
    return float(np.abs(a - b).max(initial=0.0) / den)


def _img_from_gray(gray: np.ndarray) -> torch.Tensor:
    g = torch.from_numpy(np.asarray(gray, np.float32))
    return torch.stack([g, g, g], dim=-1)


def pin_golden(fwd, vjp) -> list[str]:
    fails = []
    wx, wy = wl.sobel_weights()
    gi = read_golden("impulse_5x5.txt")
    kappa = float(gi["kappa"])
    img = torch.zeros(5, 5, 3)
    img[2, 2, :] = 1.0
    r = fwd(img, kappa, wx, wy, "valid")
    if r.shape != (1, 1) or abs(r[0, 0] - float(gi["R[0][0]"])) > 1e-9:
        fails.append(f"impulse valid R {r.tolist()} != {gi['R[0][0]']}")
    rc = fwd(img, kappa, wx, wy, "clamp")
    if abs(rc[2, 2] - float(gi["clamp_R[2][2]"])) > 1e-9:
        fails.append(f"impulse clamp R[2][2] {rc[2, 2]} != {gi['clamp_R[2][2]']}")
    _, gk, _, _ = vjp(img, torch.ones(1, 1), kappa, wx, wy, "valid")
    if abs(gk - float(gi["dkappa"])) > 1e-9:
        fails.append(f"impulse dkappa {gk} != {gi['dkappa']}")
    ge = read_golden("edge_5x5.txt")
    gray = np.zeros((5, 5))
    gray[:, 2:] = 1.0
    r = fwd(_img_from_gray(gray), float(ge["kappa"]), wx, wy, "clamp")
    for key in ("R[2][2]", "R[0][1]", "R[2][0]", "R[2][4]"):
        i, j = int(key[2]), int(key[5])
        if abs(r[i, j] - float(ge[key])) > 1e-9:
            fails.append(f"edge {key} {r[i, j]} != {ge[key]}")
    return fails


def pin_ramp(fwd, vjp) -> list[str]:
    fails = []
    wx, wy = wl.sobel_weights()
    kappa = 0.05
    for (a, b, h, w) in ((0.037, -0.021, 9, 11), (-0.011, 0.029, 8, 7)):
        y, x = np.mgrid[0:h, 0:w]
        gray = a * x + b * y + 0.5
        img = _img_from_gray(gray)
        # the f32 image is what the oracle sees: use its exact gray slope only through the
        # closed form's inputs a, b; the f32 rounding of the ramp is below 1e-7 relative.
        expect = -kappa * (576.0 * (a * a + b * b)) ** 2
        rv = fwd(img, kappa, wx, wy, "valid")
        rc = fwd(img, kappa, wx, wy, "clamp")[2:-2, 2:-2]
        for name, r in (("valid", rv), ("clamp interior", rc)):
            if r.shape != (h - 4, w - 4) or rel(r, np.full_like(r, expect)) > 1e-4:
                fails.append(f"ramp {name}: max rel {rel(r, np.full_like(r, expect))}")
    # the same closed form exactly, on a ramp whose f32 values are exact (integers / 8)
    y, x = np.mgrid[0:7, 0:9]
    gray = (3 * x - 2 * y + 40) / 8.0
    r = fwd(_img_from_gray(gray), kappa, wx, wy, "valid")
    # gray coefficients sum to 1 only to FP64 rounding, hence 1e-12 rather than 0
    expect = -kappa * (576.0 * ((3 / 8) ** 2 + (2 / 8) ** 2)) ** 2
    if rel(r, np.full_like(r, expect)) > 1e-12:
        fails.append(f"exact ramp: max rel {rel(r, np.full_like(r, expect))}")
    return fails


def pin_constant(fwd, vjp) -> list[str]:
    fails = []
    wx, wy = wl.sobel_weights()
    for border, (h, w) in (("valid", (6, 7)), ("clamp", (5, 3)), ("clamp", (1, 1))):
        img = torch.full((h, w, 3), 0.625)
        r = fwd(img, 0.04, wx, wy, border)
        if np.any(r != 0.0):
            fails.append(f"constant {border} {h}x{w}: max |R| {np.abs(r).max()}")
    return fails


def library_harris(img: torch.Tensor, kappa, wx, wy, border) -> np.ndarray:
    """The pipeline from torch's float64 conv2d (a cross-correlation) and replicate padding."""
    x = img.double()
    gray = x[..., 0] * 0.299 + x[..., 1] * 0.587 + x[..., 2] * 0.114
    g4 = gray[None, None]

    def stage(t, k):
        if border == "clamp":
            t = F.pad(t, (1, 1, 1, 1), mode="replicate")
        return F.conv2d(t, k)
    kx = torch.as_tensor(wx, dtype=torch.float64).reshape(1, 1, 3, 3)
    ky = torch.as_tensor(wy, dtype=torch.float64).reshape(1, 1, 3, 3)
    ix, iy = stage(g4, kx), stage(g4, ky)
    ones = torch.ones(1, 1, 3, 3, dtype=torch.float64)
    sxx, sxy, syy = stage(ix * ix, ones), stage(ix * iy, ones), stage(iy * iy, ones)
    r = sxx * syy - sxy * sxy - kappa * (sxx + syy) ** 2
    return r[0, 0].numpy()


def pin_library(fwd, vjp) -> list[str]:
    fails = []
    for seed, (h, w), border in ((1, (7, 9), "clamp"), (2, (8, 6), "valid"), (3, (2, 5), "clamp")):
        img = wl.random_image(h, w, seed)
        wx, wy = wl.random_weights(seed + 10)
        r = fwd(img, 0.06, wx, wy, border)
        ref = library_harris(img, 0.06, wx.double(), wy.double(), border)
        if r.shape != ref.shape or rel(r, ref) > 1e-12:
            fails.append(f"conv2d {border} {h}x{w}: shape {r.shape} vs {ref.shape}, "
                         f"rel {rel(r, ref) if r.shape == ref.shape else 'n/a'}")
    return fails


def pin_homogeneity(fwd, vjp) -> list[str]:
    fails = []
    img = wl.random_image(6, 8, 4)
    wx, wy = wl.random_weights(4)
    for border in ("clamp", "valid"):
        r1 = fwd(img, 0.04, wx, wy, border)
        r2 = fwd(img * 2, 0.04, wx, wy, border)
        if not np.array_equal(r2, 16.0 * r1):
            fails.append(f"homogeneity {border}: max |R(2x) - 16R(x)| {np.abs(r2 - 16 * r1).max()}")
    return fails


def _loss(fwd, img64, g, kappa, wx, wy, border) -> float:
    # both oracles take FP64 images, so the FD perturbations are not rounded away
    return float(np.sum(np.asarray(g, np.float64) * fwd(img64, kappa, wx, wy, border)))


def pin_fd(fwd, vjp) -> list[str]:
    fails = []
    for seed, (h, w), border in ((5, (5, 6), "clamp"), (6, (6, 7), "valid"), (7, (1, 3), "clamp")):
        img = wl.random_image(h, w, seed).double()
        wx, wy = wl.random_weights(seed)
        wx, wy = wx.double(), wy.double()
        kappa = 0.05
        ho, wo = (h, w) if border == "clamp" else (h - 4, w - 4)
        g = wl.random_cotangent(ho, wo, seed + 1).double()
        gimg, gk, gwx, gwy = vjp(img, g, kappa, wx, wy, border)

        def L(im=img, k=kappa, a=wx, b=wy):
            return _loss(fwd, im, g, k, a, b, border)
        eps = 1e-6
        fd_img = np.zeros((h, w, 3))
        for i in range(h):
            for j in range(w):
                for c in range(3):
                    p, m = img.clone(), img.clone()
                    p[i, j, c] += eps
                    m[i, j, c] -= eps
                    fd_img[i, j, c] = (L(im=p) - L(im=m)) / (2 * eps)
        fd_k = (L(k=kappa + eps) - L(k=kappa - eps)) / (2 * eps)
        fd_w = []
        for which in (0, 1):
            out = np.zeros((3, 3))
            for a in range(3):
                for b in range(3):
                    p = (wx if which == 0 else wy).clone()
                    m = p.clone()
                    p[a, b] += eps
                    m[a, b] -= eps
                    lp = L(a=p) if which == 0 else L(b=p)
                    lm = L(a=m) if which == 0 else L(b=m)
                    out[a, b] = (lp - lm) / (2 * eps)
            fd_w.append(out)
        for name, got, ref in (("img", gimg, fd_img), ("kappa", [gk], [fd_k]),
                               ("wx", gwx, fd_w[0]), ("wy", gwy, fd_w[1])):
            if rel(got, ref) > 1e-6:
                fails.append(f"fd {border} {h}x{w} d{name}: rel {rel(got, ref)}")
    return fails


def pin_euler(fwd, vjp) -> list[str]:
    fails = []
    for seed, (h, w), border in ((8, (7, 6), "clamp"), (9, (7, 8), "valid")):
        img = wl.random_image(h, w, seed)
        wx, wy = wl.random_weights(seed)
        ho, wo = (h, w) if border == "clamp" else (h - 4, w - 4)
        g = wl.random_cotangent(ho, wo, seed + 1)
        L = float(np.sum(g.double().numpy() * fwd(img, 0.04, wx, wy, border)))
        gimg, gk, gwx, gwy = vjp(img, g, 0.04, wx, wy, border)
        s_img = float(np.sum(img.double().numpy() * gimg))
        s_w = float(np.sum(wx.double().numpy() * gwx) + np.sum(wy.double().numpy() * gwy))
        if abs(s_img - 4 * L) > 1e-10 * abs(L):
            fails.append(f"euler img {border}: {s_img} vs 4L {4 * L}")
        if abs(s_w - 4 * L) > 1e-10 * abs(L):
            fails.append(f"euler weights {border}: {s_w} vs 4L {4 * L}")
    return fails


ALL_PINS = {
    "golden": pin_golden, "ramp": pin_ramp, "constant": pin_constant, "library": pin_library,
    "homogeneity": pin_homogeneity, "fd": pin_fd, "euler": pin_euler,
}


def run_all(fwd, vjp) -> dict[str, list[str]]:
    out = {}
    for name, pin in ALL_PINS.items():
        try:
            out[name] = pin(fwd, vjp)
        except Exception as e:  # a mutant may also break shapes; that is a failed pin too
            out[name] = [f"raised {type(e).__name__}: {e}"]
    return out


# ---------------------------------------------------------------------------------------------
# Adapters: the two oracles as (fwd, vjp)
# ---------------------------------------------------------------------------------------------

def pattern_oracle():
    from oracle import harris as H

    def fwd(img, kappa, wx, wy, border):
        return np.array(H.harris(H.to_nested(img), float(kappa), H.to_nested(wx),
                                 H.to_nested(wy), border), dtype=np.float64).reshape(
            (img.shape[0], img.shape[1]) if border == "clamp" else (img.shape[0] - 4, img.shape[1] - 4))

    def vjp(img, g, kappa, wx, wy, border):
        gi, gk, gwx, gwy = H.harris_vjp(H.to_nested(img), float(kappa), H.to_nested(wx),
                                        H.to_nested(wy), border, H.to_nested(g))
        return np.array(gi), float(gk), np.array(gwx), np.array(gwy)
    return fwd, vjp


def c_oracle():
    """The C reference (FP64 inputs and arithmetic) as (fwd, vjp)."""
    from oracle import cref

    def fwd(img, kappa, wx, wy, border):
        return cref.forward(img, kappa, wx, wy, border)

    def vjp(img, g, kappa, wx, wy, border):
        return cref.backward(img, g, kappa, wx, wy, border)
    return fwd, vjp
