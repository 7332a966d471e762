"""Build libshine.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

    python -m paper_2201_03611_b300.build [--force] [--verbose] [--debug | --all]

Each csrc/*.cu is compiled separately (in parallel) with nvcc for sm_103a only, then linked
into paper_2201_03611_b300/libshine.so with the CUDA runtime linked statically, so the
library needs nothing from the Python process but the driver. Objects go to _build/.
--debug builds libshine_debug.so instead: the same sources with SHINE_DEBUG_BOUNDS=1, whose
kernels check their index ranges and report violations (shine_debug_bounds_status); --all
builds both.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ_DIR = os.path.join(ROOT, "_build", "shine")
LIB = os.path.join(PKG, "libshine.so")
DEBUG_OBJ_DIR = os.path.join(ROOT, "_build", "shine_debug")
DEBUG_LIB = os.path.join(PKG, "libshine_debug.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def _deps(src: str) -> list[str]:
    return [src] + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, verbose: bool, obj_dir: str = OBJ_DIR, defs: tuple = ()) -> tuple[str, str]:
    obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, *defs, "-Xptxas", "-v", "-c", src, "-o", obj]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{p.stdout}\n{p.stderr}")
    return obj, (p.stderr if verbose else "")


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    obj_dir, lib = (DEBUG_OBJ_DIR, DEBUG_LIB) if debug else (OBJ_DIR, LIB)
    defs = ("-DSHINE_DEBUG_BOUNDS=1",) if debug else ()
    os.makedirs(obj_dir, exist_ok=True)
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    objs, todo = [], []
    for src in sources:
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _stale(obj, _deps(src)):
            todo.append(src)
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            for obj, log in ex.map(lambda s: _compile(s, verbose, obj_dir, defs), todo):
                if log:
                    sys.stderr.write(log)
    if force or todo or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [NVCC, *ARCH, "-shared", "-cudart", "static", "-Xcompiler", "-fvisibility=hidden", *objs,
               "-o", tmp]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
        os.replace(tmp, lib)
    return lib


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--debug", action="store_true", help="build libshine_debug.so (index checks)")
    ap.add_argument("--all", action="store_true", help="build both libraries")
    args = ap.parse_args()
    if args.all or not args.debug:
        print(build(args.force, args.verbose))
    if args.all or args.debug:
        print(build(args.force, args.verbose, debug=True))


if __name__ == "__main__":
    main()
