"""The index-checking build (libshine_debug.so, SHINE_DEBUG_BOUNDS=1): a stand-in for a memory
checker, which this pool does not offer. Its Harris kernels check the row and column ranges of
every global load, store and copy and of their shared-memory staging and record violations in a
device word instead of trapping. Here it runs the forward, the adjoint (all staging paths, both
adjoint layouts), the fused pass, the host-buffer pipeline and a batch under two schedules on
ragged shapes in a child process (with the eight-column adjoint allowed at every size), which
must report no violation and the same results, bit for bit, as the release build in this
process."""
import json
import os
import subprocess
import sys

import pytest
import torch

import gpu_util as U
import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEBUG_LIB = os.path.join(ROOT, "paper_2201_03611_b300", "libshine_debug.so")

SHAPES = [((1, 1), "clamp"), ((3, 5), "clamp"), ((37, 250), "clamp"), ((64, 256), "clamp"), ((130, 512), "clamp"),
          ((300, 264), "clamp"), ((9, 133), "valid"), ((70, 245), "valid"), ((257, 744), "clamp")]

CHILD = r"""
import json, os, sys, tempfile
sys.path.insert(0, {root!r}); sys.path.insert(0, os.path.join({root!r}, "tests"))
import torch
import paper_2201_03611_b300 as S
from paper_2201_03611_b300 import _lib as L
from paper_2201_03611_b300.tune import gpu_key
import workloads as wl
import gpu_util as U
import ctypes
assert L.LIB_PATH.endswith("libshine_debug.so"), L.LIB_PATH
out = {{}}
for (h, w), border in {shapes!r}:
    for dt in (torch.float32, torch.bfloat16):
        img = wl.random_image(h, w, seed=h + w).to(dt).cuda()
        ho, wo = S.output_shape(h, w, border)
        g = wl.random_cotangent(ho, wo, seed=h * w).to(dt).cuda()
        k, wx, wy = U.dev_params(0.05, *wl.random_weights(h))
        r = S.pipeline_fwd(img, k, wx, wy, border)
        gi = S.pipeline_bwd(img, g, k, wx, wy, border)[0]
        gi_u = S.pipeline_bwd(U.padded_image(img, 1), g, k, wx, wy, border)[0]
        fr, fgi = S.pipeline_fwd_bwd(img, g, k, wx, wy, border)[:2]
        torch.save([t.cpu() for t in (r, gi, gi_u, fr, fgi)], os.path.join({tmp!r}, f"{{h}}_{{w}}_{{border}}_{{dt}}.pt"))
# a batch under two schedules (per-lane and bulk staging)
b = wl.batch_512(n=8, dtype="bf16", seed=17, lo=40, hi=700)
imgs = [wl.to_device(t, "cuda") for t in b["imgs"]]
ws = [wl.to_device(t, "cuda") for t in b["ws"]]
shapes = [tuple(t.shape[:2]) for t in imgs]
kappa = b["kappa"].cuda()
wx, wy = [t.cuda() for t in wl.random_weights(5)]
for staging, origin in ((0, 0), (1, -76)):
    path = os.path.join({tmp!r}, "tune.txt")
    open(path, "w").write(f"{{gpu_key()}} 1 1 3 plan 0 {{staging}} 6 {{origin}}\n")
    plan = S.BatchedPlan(shapes, torch.bfloat16, "clamp", fwd_bwd=True, tune_cache=path)
    assert plan.schedule()["staging"] == staging
    outs = [wl.empty_padded((h, w), torch.bfloat16, "cuda") for h, w in shapes]
    gimgs = [wl.empty_padded((h, w, 3), torch.bfloat16, "cuda") for h, w in shapes]
    gk = torch.empty(len(imgs), device="cuda")
    gwx, gwy = torch.empty(3, 3, device="cuda"), torch.empty(3, 3, device="cuda")
    plan.run(plan.bind(imgs, outs, ws, gimgs), kappa, wx, wy, gk, gwx, gwy)
    torch.save([t.cpu() for t in outs + gimgs], os.path.join({tmp!r}, f"batch_{{staging}}.pt"))
    plan.close()
# the host-buffer pipeline
h, w, nb = 203, 517, 16
img_h = wl.random_image(h, w, seed=31).pin_memory()
g_h = wl.random_cotangent(h, w, seed=32).pin_memory()
k, wx, wy = U.dev_params(0.05, *wl.random_weights(31))
dev = [torch.empty(h, w, 3, device="cuda"), torch.empty(h, w, device="cuda"), torch.empty(h, w, device="cuda"),
       torch.empty(h, w, 3, device="cuda")]
ws_h = torch.empty(S.ops.host_workspace_bytes(h, w, "clamp", nb), dtype=torch.uint8, device="cuda")
out_h, gimg_h = torch.empty(h, w).pin_memory(), torch.empty(h, w, 3).pin_memory()
par = torch.empty(19, device="cuda")
S.ops.pipeline_host(img_h, g_h, k, wx, wy, *dev, ws_h, out_h=out_h, gimg_h=gimg_h, grad_params=par, nbands=nb)
torch.cuda.synchronize()
inst, bits = ctypes.c_int(), ctypes.c_uint()
L.check(L.lib().shine_debug_bounds_status(ctypes.byref(inst), ctypes.byref(bits), 1), "status")
print(json.dumps({{"instrumented": inst.value, "bits": bits.value}}))
"""


def test_debug_build_reports_no_violation_and_release_results(tmp_path):
    if not os.path.exists(DEBUG_LIB):
        pytest.fail("libshine_debug.so is not built (python -m paper_2201_03611_b300.build --debug)")
    import paper_2201_03611_b300 as S
    # the eight-column adjoint at every size, so that the small shapes reach it too
    env = dict(os.environ, SHINE_LIBRARY=DEBUG_LIB, SHINE_WIDE_BWD_MIN_PIXELS="0")
    script = CHILD.format(root=ROOT, shapes=SHAPES, tmp=str(tmp_path))
    p = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    status = json.loads(p.stdout.strip().splitlines()[-1])
    assert status == {"instrumented": 1, "bits": 0}, status
    # same bits as the release build
    for (h, w), border in SHAPES:
        for dt in (torch.float32, torch.bfloat16):
            img = wl.random_image(h, w, seed=h + w).to(dt).cuda()
            ho, wo = S.output_shape(h, w, border)
            g = wl.random_cotangent(ho, wo, seed=h * w).to(dt).cuda()
            k, wx, wy = U.dev_params(0.05, *wl.random_weights(h))
            ref = [S.pipeline_fwd(img, k, wx, wy, border), S.pipeline_bwd(img, g, k, wx, wy, border)[0]]
            got = torch.load(tmp_path / f"{h}_{w}_{border}_{dt}.pt")
            assert torch.equal(got[0], ref[0].cpu()) and torch.equal(got[1], ref[1].cpu()), ((h, w), border, dt)
            assert torch.equal(got[2], got[1]) and torch.equal(got[3], got[0]) and torch.equal(got[4], got[1])
    assert all(torch.equal(x, y) for x, y in zip(torch.load(tmp_path / "batch_0.pt"), torch.load(tmp_path / "batch_1.pt")))


def test_release_build_is_not_instrumented():
    import ctypes
    from paper_2201_03611_b300 import _lib as L
    inst, bits = ctypes.c_int(7), ctypes.c_uint(7)
    L.check(L.lib().shine_debug_bounds_status(ctypes.byref(inst), ctypes.byref(bits), 0), "status")
    assert inst.value == 0 and bits.value == 0
