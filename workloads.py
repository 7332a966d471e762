"""Seeded synthetic inputs for the Harris pattern pipeline.

This module only draws numbers: it holds none of the pipeline's arithmetic, so both the
FP64 oracle (``oracle/``) and the CUDA path use it without sharing any method code.
Every tensor is made on the host with the torch CPU generator, so the same seed gives the
same bits on any machine; storage-dtype casts are round-to-nearest-even (torch ``.to``).

Workloads (images are H x W x 3, HWC interleaved, channel fastest):

* ``plain_256``     one 256x256 image, uniform [0,1) from seed 0, kappa 0.04, VALID borders.
* ``salt_8192``     one 8192x8192 image, uniform [0,1) from seed 0, then a mask
                    ``rand(8192,8192) < 0.05`` drawn next from the same generator sets all
                    three channels of 5% of the pixels to 1.0; CLAMP borders.
* ``diff_2048``     image seed 0 ``rand(2048,2048,3)``, cotangent ``w = randn(2048,2048)``
                    from seed 1, CLAMP borders, loss = sum(w * R).
* ``prec_8192``     ``rand(8192,8192,3)`` seed 0 (no salt), cast to bf16 / fp16, and
                    ``w = randn(8192,8192)`` seed 1 cast the same way.
* ``batch_512``     seed 2: sizes ``round(exp(U(ln 64, ln 2048)))`` as a (512, 2) draw,
                    kappa_i ~ U(0.02, 0.08), then per image ``rand(H,W,3)`` and
                    ``randn(H,W)`` in order from the same generator; bf16 storage, every
                    row pitch (image and cotangent) rounded up to a multiple of 16 bytes.
"""
from __future__ import annotations

import math

import torch

KAPPA = 0.04
# Corner threshold of the salt workloads: about the top 1% of R on the salted uniform image
# (R quantiles there: 50% ~ 13, 90% ~ 41, 99% ~ 95); the corners are the local maxima above it.
CORNER_THRESHOLD = 100.0

# Default Sobel weights, applied as a correlation (window[a][b] * W[a][b]); x is the column.
SOBEL_X = [[-1.0, 0.0, 1.0], [-2.0, 0.0, 2.0], [-1.0, 0.0, 1.0]]
SOBEL_Y = [[-1.0, -2.0, -1.0], [0.0, 0.0, 0.0], [1.0, 2.0, 1.0]]

_DTYPES = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}


def storage_dtype(name: str) -> torch.dtype:
    return _DTYPES[name]


def sobel_weights() -> tuple[torch.Tensor, torch.Tensor]:
    """The default (wx, wy) as 3x3 float32 tensors."""
    return torch.tensor(SOBEL_X, dtype=torch.float32), torch.tensor(SOBEL_Y, dtype=torch.float32)


def random_weights(seed: int) -> tuple[torch.Tensor, torch.Tensor]:
    """Non-symmetric 3x3 weights, used to catch orientation and index mistakes."""
    g = torch.Generator().manual_seed(seed)
    wx = torch.randn(3, 3, generator=g, dtype=torch.float32)
    wy = torch.randn(3, 3, generator=g, dtype=torch.float32)
    return wx, wy


def random_image(h: int, w: int, seed: int, dtype: str = "f32") -> torch.Tensor:
    """Uniform [0,1) H x W x 3 image, cast to the storage dtype."""
    g = torch.Generator().manual_seed(seed)
    img = torch.rand(h, w, 3, generator=g, dtype=torch.float32)
    return img.to(_DTYPES[dtype])


def random_cotangent(h: int, w: int, seed: int, dtype: str = "f32") -> torch.Tensor:
    """N(0,1) H x W cotangent (the loss weights w), cast to the storage dtype."""
    g = torch.Generator().manual_seed(seed)
    return torch.randn(h, w, generator=g, dtype=torch.float32).to(_DTYPES[dtype])


def plain_256() -> dict:
    img = random_image(256, 256, seed=0)
    return {"img": img, "kappa": KAPPA, "border": "valid"}


def salt_image(h: int, w: int, seed: int = 0, frac: float = 0.05) -> torch.Tensor:
    """Uniform [0,1) image with a fraction of pixels forced to 1.0 in all channels."""
    g = torch.Generator().manual_seed(seed)
    img = torch.rand(h, w, 3, generator=g, dtype=torch.float32)
    mask = torch.rand(h, w, generator=g, dtype=torch.float32) < frac
    img[mask] = 1.0
    return img


def salt_8192() -> dict:
    return {"img": salt_image(8192, 8192), "kappa": KAPPA, "border": "clamp"}


def diff_2048() -> dict:
    return {
        "img": random_image(2048, 2048, seed=0),
        "w": random_cotangent(2048, 2048, seed=1),
        "kappa": KAPPA,
        "border": "clamp",
    }


def prec_8192(dtype: str) -> dict:
    return {
        "img": random_image(8192, 8192, seed=0, dtype=dtype),
        "w": random_cotangent(8192, 8192, seed=1, dtype=dtype),
        "kappa": KAPPA,
        "border": "clamp",
    }


def batch_sizes(n: int = 512, seed: int = 2, lo: int = 64, hi: int = 2048):
    """Image sizes and kappas of the uneven batch, plus the generator positioned after them."""
    g = torch.Generator().manual_seed(seed)
    u = torch.rand(n, 2, generator=g, dtype=torch.float64)
    hw = torch.round(torch.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).to(torch.int64)
    kappa = 0.02 + 0.06 * torch.rand(n, generator=g, dtype=torch.float64)
    return hw, kappa.to(torch.float32), g


def padded(t: torch.Tensor, row_bytes: int = 16) -> torch.Tensor:
    """The same values with every row (first dimension) padded to a multiple of row_bytes bytes:
    a strided view into a zero-filled buffer of whole padded rows."""
    h = t.shape[0]
    row = t.reshape(h, -1)
    esize = t.element_size()
    pitch = -(-row.shape[1] * esize // row_bytes) * row_bytes // esize
    store = torch.zeros(h, pitch, dtype=t.dtype, device=t.device)
    store[:, :row.shape[1]] = row
    strides = (pitch,) + tuple(t.stride()[1:])
    return store.as_strided(t.shape, strides)


def to_device(t: torch.Tensor, device) -> torch.Tensor:
    """Copy of a (possibly row-padded) tensor on `device` with the same strides."""
    h, pitch = t.shape[0], t.stride(0)
    return torch.as_strided(t, (h, pitch), (pitch, 1)).to(device).as_strided(t.shape, t.stride())


def empty_padded(shape, dtype: torch.dtype, device, row_bytes: int = 16) -> torch.Tensor:
    """An uninitialised tensor of `shape` whose rows are padded to a multiple of row_bytes bytes."""
    esize = torch.empty(0, dtype=dtype).element_size()
    row = 1
    for d in shape[1:]:
        row *= d
    pitch = -(-row * esize // row_bytes) * row_bytes // esize
    store = torch.empty(shape[0], pitch, dtype=dtype, device=device)
    strides, acc = [], 1
    for d in reversed(shape[1:]):
        strides.insert(0, acc)
        acc *= d
    return store.as_strided(tuple(shape), (pitch,) + tuple(strides))


def batch_512(n: int = 512, dtype: str = "bf16", seed: int = 2, lo: int = 64, hi: int = 2048,
              pad16: bool = True) -> dict:
    """The uneven batch: per-image images and cotangents drawn in order after the sizes; with
    pad16 every row pitch is rounded up to a multiple of 16 bytes (see padded, to_device)."""
    hw, kappa, g = batch_sizes(n, seed, lo, hi)
    imgs, ws = [], []
    for i in range(n):
        h, w = int(hw[i, 0]), int(hw[i, 1])
        img = torch.rand(h, w, 3, generator=g, dtype=torch.float32).to(_DTYPES[dtype])
        wi = torch.randn(h, w, generator=g, dtype=torch.float32).to(_DTYPES[dtype])
        imgs.append(padded(img) if pad16 else img)
        ws.append(padded(wi) if pad16 else wi)
    return {"hw": hw, "kappa": kappa, "imgs": imgs, "ws": ws, "border": "clamp"}


def sample_points(h: int, w: int, n: int, seed: int, border_rows: int = 3) -> torch.Tensor:
    """(n + edge) x 2 int64 (y, x) positions: random interior points plus the four corners and
    points on each border band, so that sampled checks always see the clamp folds."""
    g = torch.Generator().manual_seed(seed)
    ys = torch.randint(0, h, (n,), generator=g)
    xs = torch.randint(0, w, (n,), generator=g)
    edge = []
    for y in list(range(min(border_rows, h))) + list(range(max(h - border_rows, 0), h)):
        for x in (0, 1, 2, w // 2, w - 3, w - 2, w - 1):
            if 0 <= x < w:
                edge.append((y, x))
    for x in list(range(min(border_rows, w))) + list(range(max(w - border_rows, 0), w)):
        for y in (h // 3, h // 2, (2 * h) // 3):
            edge.append((y, x))
    pts = torch.cat([torch.stack([ys, xs], 1), torch.tensor(edge, dtype=torch.int64).reshape(-1, 2)])
    return pts


def mv_inputs(m: int, n: int, seed: int) -> tuple[torch.Tensor, torch.Tensor]:
    """Matrix-vector workload (the paper's running example): A ~ N(0,1) of shape (m, n), then
    x ~ N(0,1) of shape (n,), float32, from one generator in that order."""
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(m, n, generator=g)
    x = torch.randn(n, generator=g)
    return A, x


def iterate_inputs(m: int, n: int, k: int, seed: int) -> torch.Tensor:
    """Input of the iterate (tree-sum) workload: (n^k) m float32 values ~ U(-1, 1)."""
    g = torch.Generator().manual_seed(seed)
    return torch.rand(n ** k * m, generator=g) * 2.0 - 1.0


def iterate_stencil_inputs(h: int, w: int, seed: int, blur: bool = True) -> tuple[torch.Tensor, torch.Tensor]:
    """Iterated-stencil workload: x ~ U(0, 1) of shape (h, w), then 3 x 3 weights from one
    generator in that order: a blur (U(0, 1) weights scaled to sum 1, so repeated rounds stay
    in range) or, with blur=False, N(0, 1) weights."""
    g = torch.Generator().manual_seed(seed)
    x = torch.rand(h, w, generator=g)
    if blur:
        W = torch.rand(3, 3, generator=g)
        W = (W.double() / W.double().sum()).float()
    else:
        W = torch.randn(3, 3, generator=g)
    return x, W


def stencil_inputs(h: int, w: int, k: int, seed: int) -> tuple[torch.Tensor, torch.Tensor]:
    """Generalised-stencil workload: x ~ U(0, 1) of shape (h, w), then K x K weights ~ N(0, 1)
    (non-separable), float32, from one generator in that order."""
    g = torch.Generator().manual_seed(seed)
    x = torch.rand(h, w, generator=g)
    W = torch.randn(k, k, generator=g)
    return x, W


def separable_weights(k: int, seed: int) -> tuple[torch.Tensor, torch.Tensor]:
    """A K-tap Gaussian down the columns (sigma = K / 4) and K ~ N(0, 1) taps along the rows."""
    g = torch.Generator().manual_seed(seed + 7919)
    r = (k - 1) // 2
    t = torch.arange(-r, r + 1, dtype=torch.float64)
    sigma = max(k / 4.0, 0.5)
    wv = torch.exp(-0.5 * (t / sigma) ** 2)
    wv = (wv / wv.sum()).float()
    wh = torch.randn(k, generator=g)
    return wv, wh


def gaussian_window(k: int, sigma: float | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """Normalised K-tap Gaussian taps (sigma = K / 4 unless given) for both window axes."""
    r = (k - 1) // 2
    s = sigma if sigma is not None else max(k / 4.0, 0.5)
    t = torch.arange(-r, r + 1, dtype=torch.float64)
    w = torch.exp(-0.5 * (t / s) ** 2)
    w = (w / w.sum()).float()
    return w.clone(), w.clone()
