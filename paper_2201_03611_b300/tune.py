"""Autotuner of the batched plan: tile heights per shape bucket and the plan's schedule.

    python -m paper_2201_03611_b300.tune --out tune_cache.txt [--n 512] [--dtype bf16]

Coordinate descent over the batch's time (CUDA events, best of a few runs): first the schedule
knobs one at a time -- the staging of interior segments (per-lane cp.async or bulk copies),
the order in which the persistent warps claim the tiles (longest first, image by image,
largest image first), the weight of an edge-segment row in that order's work estimate, and the
segment origin (which columns fall in edge segments, and the alignment of the staged spans) --
then the band height of each shape bucket (ceil(log2(rows))), then the schedule knobs once
more with the tuned heights. Short bands balance the persistent schedule's tail; long bands cut
the recomputed vertical halo (4 rows forward, 8 forward+backward). The result is written as
text lines
    <gpu key> <dtype> <border> <mode> <bucket> <band_rows>
    <gpu key> <dtype> <border> <mode> plan <order> <staging> <edge_w4> <origin>
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
ORDERS = (L.SHINE_ORDER_LONGEST_FIRST, L.SHINE_ORDER_IMAGE, L.SHINE_ORDER_LARGEST_IMAGE_FIRST)
EDGE_W4 = (4, 5, 6, 8, 10, 12)
ORIGINS = (0, -4, -28, -52, -76, -100)
DEFAULT_SCHEDULE = {"order": L.SHINE_ORDER_LONGEST_FIRST, "staging": 0, "edge_w4": 6, "origin": 0}


def gpu_key() -> str:
    buf = ctypes.create_string_buffer(512)
    n = L.lib().shine_tune_key(buf, 512)
    if n < 0:
        raise RuntimeError("no CUDA device visible")
    return buf.value.decode()


def bucket_of(rows: int) -> int:
    return max(0, math.ceil(math.log2(rows))) if rows > 1 else 0


def origin_ok(origin: int, staging: int, dtype) -> bool:
    """The plan's rule: a multiple of 4 columns, and 4 mod 8 for bulk-staged 16-bit images."""
    return origin % 4 == 0 and (staging == 0 or dtype == torch.float32 or origin % 8 == 4)


def _write(path: str, key: str, dt: int, border: int, mode: int, table: dict, sched: dict | None = None) -> None:
    with open(path, "w") as f:
        f.write("# gpu dtype border mode bucket band_rows | gpu dtype border mode plan order staging edge_w4 origin\n")
        for b, r in sorted(table.items()):
            f.write(f"{key} {dt} {border} {mode} {b} {r}\n")
        if sched is not None:
            f.write(f"{key} {dt} {border} {mode} plan {sched['order']} {sched['staging']} {sched['edge_w4']} "
                    f"{sched['origin']}\n")


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
         out_path: str | None = None, candidates=CANDIDATES, verbose=False) -> tuple[dict, dict]:
    """Returns (band rows per bucket, schedule) and writes them to out_path."""
    mode = L.SHINE_MODE_FWD_BWD if fwd_bwd else L.SHINE_MODE_FWD
    key = gpu_key()
    halo = 4 if border == "valid" and not fwd_bwd else 0
    buckets = sorted({bucket_of(h - halo) for h, _ in shapes})
    table: dict = {}
    sched = dict(DEFAULT_SCHEDULE)
    with tempfile.TemporaryDirectory() as td:
        cache = os.path.join(td, "tune.txt")

        def measure(tab, sc):
            _write(cache, key, dtype_code(dtype), border_code(border), mode, tab, sc)
            return time_batch(shapes, imgs, outs, gouts, gimgs, kappa, wx, wy, dtype, border, fwd_bwd, cache)

        def tune_schedule():
            knobs = (("staging", (0, 1) if fwd_bwd else (0,)), ("order", ORDERS), ("edge_w4", EDGE_W4),
                     ("origin", ORIGINS))
            for name, values in knobs:
                best, best_trial = float("inf"), dict(sched)
                for v in values:
                    trial = dict(sched)
                    trial[name] = v
                    if not origin_ok(trial["origin"], trial["staging"], dtype):
                        trial["origin"] = -4  # the nearest origin valid for both stagings
                    t = measure(table, trial)
                    if verbose:
                        print(f"schedule {trial}: {t:.3f} ms")
                    if t < best:
                        best, best_trial = t, trial
                sched.update(best_trial)

        tune_schedule()
        for b in buckets:
            best, best_rows = float("inf"), None
            for c in candidates:
                if c > 2 ** b * 2:
                    continue
                trial = dict(table)
                trial[b] = c
                t = measure(trial, sched)
                if verbose:
                    print(f"bucket {b} rows {c}: {t:.3f} ms")
                if t < best:
                    best, best_rows = t, c
            table[b] = best_rows
        tune_schedule()
    if out_path:
        _write(out_path, key, dtype_code(dtype), border_code(border), mode, table, sched)
    return table, sched


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
    table, sched = tune(shapes, imgs, outs, None if args.fwd_only else gouts, None if args.fwd_only else gimgs,
                        b["kappa"].cuda(), wx, wy, imgs[0].dtype, "clamp", not args.fwd_only, args.out, verbose=True)
    print(table, sched)


if __name__ == "__main__":
    main()
