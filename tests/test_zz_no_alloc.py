"""shine_pipeline_bwd_noalloc: the backward pass for callers that cannot allocate device memory.

A caller that is only handed its input and output buffers (or that must not allocate after
start-up) cannot supply the workspace shine_pipeline_bwd asks for; this entry keeps the
partial sums in a fixed array inside the library instead. Here it is called through the C ABI
twice in a row, on different images, and each result must equal, bit for bit, the
workspace-taking entry point's on the same inputs: both run the same kernel with the same warp
count and the same fixed-order float64 finalize, so any difference would be a stale or shared
partial sum. A bounded wait that gave up would be reported through shine_wait_status, which
must stay clear. (The array's size limit, SHINE_ERR_UNSUPPORTED, needs a GPU with more than 256
SMs to reach and is not exercised here.) This file is collected last on purpose.
"""
import ctypes

import pytest
import torch

import gpu_util as U
import workloads as wl

pytestmark = pytest.mark.gpu


def _noalloc(img, g, k, wx, wy, border):
    from paper_2201_03611_b300 import _lib
    from paper_2201_03611_b300.ops import border_code, dtype_code
    L = _lib.lib()
    gimg = torch.empty_like(img)
    gk = torch.empty(1, device="cuda")
    gwx = torch.empty(3, 3, device="cuda")
    gwy = torch.empty(3, 3, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = L.shine_pipeline_bwd_noalloc(p(img), img.shape[0], img.shape[1], img.stride(0), dtype_code(img.dtype),
                                      border_code(border), p(k), p(wx), p(wy), p(g), g.stride(0),
                                      dtype_code(g.dtype), p(gimg), gimg.stride(0), p(gk), p(gwx), p(gwy), stream)
    assert rc == 0, _lib.status_string(rc)
    return gimg, gk, gwx, gwy


@pytest.mark.parametrize("calls", [[((517, 1030), "clamp", torch.float32), ((37, 250), "valid", torch.float32)],
                                   [((64, 124), "clamp", torch.bfloat16), ((300, 301), "clamp", torch.float32)]])
def test_noalloc_matches_workspace_entry_on_two_calls_in_a_row(calls):
    import paper_2201_03611_b300 as S
    S.ops.wait_failed(clear=True)  # start from a clear bounded-wait flag
    for n, ((h, w), border, dtype) in enumerate(calls):
        img = wl.random_image(h, w, seed=40 + n).to(dtype).cuda()
        ho, wo = S.output_shape(h, w, border)
        g = wl.random_cotangent(ho, wo, seed=50 + n).to(dtype).cuda()
        k, wx, wy = U.dev_params(0.05, *wl.random_weights(60 + n))
        got = _noalloc(img, g, k, wx, wy, border)
        ref = S.pipeline_bwd(img, g, k, wx, wy, border)
        torch.cuda.synchronize()
        for name, a, b in zip(("d img", "d kappa", "d Wx", "d Wy"), got, ref):
            assert torch.equal(a, b), (n, name)
    assert not S.ops.wait_failed(clear=True)
