"""Autotuner of the batched plan's tile heights (rows per warp work item), per shape bucket.

    python -m paper_2201_03611_b300.tune --out tune_cache.txt [--n 512] [--dtype bf16]

For each shape bucket (ceil(log2(rows))) of a batch, coordinate descent over candidate band
heights: the whole batch is timed with CUDA events for each candidate of one bucket while the
other buckets keep their current choice, and the fastest is kept. Short bands balance the
persistent schedule's tail; long bands cut the recomputed vertical halo (4 rows forward, 8
forward+backward). The result is written as text lines
    <gpu key> <dtype> <border> <mode> <bucket> <band_rows>
which shine_plan_create reads when given the file.
"""
from __future__ import annotations

import argparse
import ctypes
import math
import os
import tempfile

import torch

from . import _lib as L
from .batched import BatchedPlan
from .ops import border_code, dtype_code

CANDIDATES = (16, 32, 64, 128, 256, 512, 1024, 2048)


def gpu_key() -> str:
    buf = ctypes.create_string_buffer(512)
    n = L.lib().shine_tune_key(buf, 512)
    if n < 0:
        raise RuntimeError("no CUDA device visible")
    return buf.value.decode()


def bucket_of(rows: int) -> int:
    return max(0, math.ceil(math.log2(rows))) if rows > 1 else 0


def _write(path: str, key: str, dt: int, border: int, mode: int, table: dict) -> None:
    with open(path, "w") as f:
        f.write("# gpu dtype border mode bucket band_rows\n")
        for b, r in sorted(table.items()):
            f.write(f"{key} {dt} {border} {mode} {b} {r}\n")


def time_batch(shapes, imgs, outs, gouts, gimgs, kappa, wx, wy, dtype, border, fwd_bwd, cache, reps=5) -> float:
    plan = BatchedPlan(shapes, dtype, border, fwd_bwd=fwd_bwd, tune_cache=cache)
    descs = plan.bind(imgs, outs, gouts, gimgs)
    ws = plan.new_workspace(imgs[0].device)
    n = len(shapes)
    gk = torch.empty(n, device=imgs[0].device) if fwd_bwd else None
    gwx = torch.empty(3, 3, device=imgs[0].device) if fwd_bwd else None
    gwy = torch.empty(3, 3, device=imgs[0].device) if fwd_bwd else None
    for _ in range(2):
        plan.run(descs, kappa, wx, wy, gk, gwx, gwy, ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record()
        plan.run(descs, kappa, wx, wy, gk, gwx, gwy, ws)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    plan.close()
    return best


def tune(shapes, imgs, outs, gouts, gimgs, kappa, wx, wy, dtype, border="clamp", fwd_bwd=True,
         out_path: str | None = None, candidates=CANDIDATES, verbose=False) -> dict:
    mode = L.SHINE_MODE_FWD_BWD if fwd_bwd else L.SHINE_MODE_FWD
    key = gpu_key()
    halo = 4 if border == "valid" and not fwd_bwd else 0
    buckets = sorted({bucket_of(h - halo) for h, _ in shapes})
    table = {}
    with tempfile.TemporaryDirectory() as td:
        cache = os.path.join(td, "tune.txt")
        for b in buckets:
            best, best_rows = float("inf"), None
            for c in candidates:
                if c > 2 ** b * 2:
                    continue
                trial = dict(table)
                trial[b] = c
                _write(cache, key, dtype_code(dtype), border_code(border), mode, trial)
                t = time_batch(shapes, imgs, outs, gouts, gimgs, kappa, wx, wy, dtype, border, fwd_bwd, cache)
                if verbose:
                    print(f"bucket {b} rows {c}: {t:.3f} ms")
                if t < best:
                    best, best_rows = t, c
            table[b] = best_rows
    if out_path:
        _write(out_path, key, dtype_code(dtype), border_code(border), mode, table)
    return table


def main():
    import workloads as wl
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--dtype", default="bf16")
    ap.add_argument("--fwd-only", action="store_true")
    args = ap.parse_args()
    b = wl.batch_512(n=args.n, dtype=args.dtype)
    imgs = [wl.to_device(t, "cuda") for t in b["imgs"]]
    gouts = [wl.to_device(t, "cuda") for t in b["ws"]]
    shapes = [tuple(t.shape[:2]) for t in imgs]
    outs = [wl.empty_padded((h, w), imgs[0].dtype, "cuda") for h, w in shapes]
    gimgs = [wl.empty_padded((h, w, 3), imgs[0].dtype, "cuda") for h, w in shapes]
    wx, wy = [t.cuda() for t in wl.sobel_weights()]
    table = tune(shapes, imgs, outs, None if args.fwd_only else gouts, None if args.fwd_only else gimgs,
                 b["kappa"].cuda(), wx, wy, imgs[0].dtype, "clamp", not args.fwd_only, args.out, verbose=True)
    print(table)


if __name__ == "__main__":
    main()
