"""The bounded waits of the kernels, exercised without any fault.

A wait that runs out must report, not hang: the self-test waits on a barrier that nothing
completes, with a small poll bound, and must come back with "gave up" and a usable context.
Normal runs of every kernel that stages by bulk copies must leave the failure flags clear.
"""
import pytest
import torch

import gpu_util as U
import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


def test_wait_that_runs_out_reports_and_the_context_survives(shine):
    from paper_2201_03611_b300 import _lib as L
    res = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    L.check(L.lib().shine_selftest_bounded_wait(1 << 12, res.data_ptr(), None), "shine_selftest_bounded_wait")
    torch.cuda.synchronize()
    assert int(res.item()) == 1                      # the wait gave up after its bound
    # the context is still usable and the kernels still compute
    img = wl.random_image(64, 256, seed=1).cuda()
    k, wx, wy = U.dev_params(0.04, *wl.random_weights(1))
    r = shine.pipeline_fwd(img, k, wx, wy, "clamp")
    torch.cuda.synchronize()
    assert torch.isfinite(r).all()


def test_selftest_rejects_bad_bounds(shine):
    from paper_2201_03611_b300 import _lib as L
    res = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.lib().shine_selftest_bounded_wait(0, res.data_ptr(), None) == L.SHINE_ERR_INVALID_ARG
    assert L.lib().shine_selftest_bounded_wait(1 << 23, res.data_ptr(), None) == L.SHINE_ERR_INVALID_ARG


def test_forward_type_kernels_leave_the_wait_flag_clear(shine):
    shine.ops.wait_failed(clear=True)
    img = wl.random_image(300, 1030, seed=2).cuda()          # 16-byte aligned rows: bulk staging
    k, wx, wy = U.dev_params(0.04, *wl.random_weights(2))
    shine.pipeline_fwd(img, k, wx, wy, "clamp")
    shine.corners(img, k, wx, wy, 10.0, "clamp")
    gv, gh = wl.gaussian_window(5)
    shine.harris_window(img, k, wx, wy, gv, gh)
    assert not shine.ops.wait_failed()
