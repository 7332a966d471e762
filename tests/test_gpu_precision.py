"""The precision workload (8192 x 8192 unsalted image, bf16 and fp16 storage, float32 arithmetic):
sampled outputs of the forward and backward passes against the FP64 oracle, with the error
statistics the workload asks to state printed as one JSON line per storage type (run with -s).

Comparisons (reading of the error metric: normwise max|x - ref| / max|ref| per output tensor):
  * R in storage precision against the oracle on the quantised input: gated at 2e-2;
  * R with float32 output from the same quantised input against that oracle: gated at 1e-5
    (the storage type only quantises the input and the stored result);
  * R against the oracle on the float32 input (total error, including input quantisation):
    reported, not gated;
  * d img in storage precision against the oracle's reverse pass on the quantised image and
    cotangent: gated at 2e-2.
"""
import json

import numpy as np
import pytest
import torch

import gpu_util as U
import workloads as wl
from oracle import cref

pytestmark = pytest.mark.gpu

SIZE = 8192


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


def _stats(got, ref) -> dict:
    g = np.asarray(got, np.float64).reshape(-1)
    r = np.asarray(ref, np.float64).reshape(-1)
    scale = max(np.abs(r).max(), 1e-300)
    d = np.abs(g - r)
    floor = np.maximum(np.abs(r), 1e-6 * scale)
    return {"normwise_max": float(d.max() / scale), "normwise_mean": float(d.mean() / scale),
            "pointwise_mean": float((d / floor).mean())}


@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_precision_workload_errors(shine, name):
    img32 = wl.random_image(SIZE, SIZE, seed=0)
    g32 = wl.random_cotangent(SIZE, SIZE, seed=1)
    wx, wy = wl.sobel_weights()
    k, dwx, dwy = U.dev_params(wl.KAPPA, wx, wy)
    dt = wl.storage_dtype(name)
    img_q, g_q = img32.to(dt), g32.to(dt)
    dimg, dg = img_q.cuda(), g_q.cuda()
    out = shine.pipeline_fwd(dimg, k, dwx, dwy, "clamp")
    out32 = shine.pipeline_fwd(dimg, k, dwx, dwy, "clamp", out_dtype=torch.float32)
    ws = torch.empty(shine.bwd_workspace_bytes(SIZE, SIZE, "clamp"), dtype=torch.uint8, device="cuda")
    gimg, _, _, _ = shine.pipeline_bwd(dimg, dg, k, dwx, dwy, "clamp", workspace=ws)
    pts = wl.sample_points(SIZE, SIZE, 2000, seed=7)
    ip, jp = pts[:, 0].cuda(), pts[:, 1].cuda()
    got = U.host(out[ip, jp])
    got32 = U.host(out32[ip, jp])
    ref_q = cref.forward_points(img_q, wl.KAPPA, wx, wy, "clamp", pts)
    ref32 = cref.forward_points(img32, wl.KAPPA, wx, wy, "clamp", pts)
    gpts = torch.cat([pts[:400], pts[-100:]])  # random points and border-band points
    gref = cref.backward_points(img_q, g_q, wl.KAPPA, wx, wy, "clamp", gpts)
    ggot = U.host(gimg[gpts[:, 0].cuda(), gpts[:, 1].cuda()])
    report = {
        "workload": f"{SIZE}x{SIZE} unsalted, {name} storage, float32 arithmetic",
        "R_vs_oracle_on_quantised_input": _stats(got, ref_q),
        "R_f32_output_vs_oracle_on_quantised_input": _stats(got32, ref_q),
        "R_vs_oracle_on_f32_input": _stats(got, ref32),
        "dimg_vs_oracle_on_quantised_inputs": _stats(ggot, gref),
        "sample": f"{pts.shape[0]} R outputs, {gpts.shape[0]} d img pixels (random, corners, border bands)",
    }
    print(json.dumps(report))
    assert report["R_vs_oracle_on_quantised_input"]["normwise_max"] <= U.TOL_16
    assert report["R_f32_output_vs_oracle_on_quantised_input"]["normwise_max"] <= U.TOL_F32
    assert report["dimg_vs_oracle_on_quantised_inputs"]["normwise_max"] <= U.TOL_16


@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_precision_workload_fused_pass(shine, name):
    """The fused single pass on the full precision workload, as the benchmark times it (the
    eight-column kernel, which 16-bit images of this size take): R equals the forward's and
    d img and the parameter cotangents equal the separate adjoint's, bit for bit."""
    dt = wl.storage_dtype(name)
    img = wl.random_image(SIZE, SIZE, seed=0).to(dt).cuda()
    g = wl.random_cotangent(SIZE, SIZE, seed=1).to(dt).cuda()
    wx, wy = wl.sobel_weights()
    k, dwx, dwy = U.dev_params(wl.KAPPA, wx, wy)
    r = shine.pipeline_fwd(img, k, dwx, dwy, "clamp")
    sep = shine.pipeline_bwd(img, g, k, dwx, dwy, "clamp")
    fused = shine.pipeline_fwd_bwd(img, g, k, dwx, dwy, "clamp")
    torch.cuda.synchronize()
    assert torch.equal(fused[0], r)
    for x, y in zip(fused[1:], sep):
        assert torch.equal(x, y)


@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_precision_workload_full_adjoint(shine, name):
    """The adjoint of the full precision workload in the benchmark's launch configuration (the
    eight-column kernel), every d img element against the oracle's reverse pass on the quantised
    image and cotangent, and the parameter cotangents on the summation scale."""
    dt = wl.storage_dtype(name)
    img = wl.random_image(SIZE, SIZE, seed=0).to(dt)
    g = wl.random_cotangent(SIZE, SIZE, seed=1).to(dt)
    wx, wy = wl.sobel_weights()
    k, dwx, dwy = U.dev_params(wl.KAPPA, wx, wy)
    dgi, dgk, dgwx, dgwy = shine.pipeline_bwd(img.cuda(), g.cuda(), k, dwx, dwy, "clamp")
    torch.cuda.synchronize()
    ref = cref.backward(img, g, wl.KAPPA, wx, wy, "clamp", with_abs=True)
    assert U.rel(U.host(dgi), ref[0]) <= U.TOL_16
    U.assert_params((dgk, dgwx, dgwy), ref[1:])


@pytest.mark.parametrize("name", ["bf16", "f16"])
def test_precision_workload_full_forward(shine, name):
    """The forward of the full precision workload, every element: R with float32 output from the
    16-bit image against the oracle on the quantised input at the float32 tolerance, and R in
    storage precision at the 16-bit one."""
    dt = wl.storage_dtype(name)
    img = wl.random_image(SIZE, SIZE, seed=0).to(dt)
    wx, wy = wl.sobel_weights()
    k, dwx, dwy = U.dev_params(wl.KAPPA, wx, wy)
    r32 = shine.pipeline_fwd(img.cuda(), k, dwx, dwy, "clamp", out_dtype=torch.float32)
    r16 = shine.pipeline_fwd(img.cuda(), k, dwx, dwy, "clamp")
    torch.cuda.synchronize()
    ref = cref.forward(img, wl.KAPPA, wx, wy, "clamp")
    assert U.rel(U.host(r32), ref) <= U.TOL_F32
    assert U.rel(U.host(r16), ref) <= U.TOL_16
