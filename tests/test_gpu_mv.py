"""Parity of shine_mv (the paper's MV example as a GEMV kernel) with the FP64 oracle.

Tolerance: each y[i] is a float32 sum whose terms are rounded products; lane l sums at most
ceil(N / 32) of them in sequence, then 2 + 5 more additions join the accumulators and the
lanes, so |y - exact| <= (ceil(N / 32) + 8) * 2^-24 * sum_j |A[i][j] x[j]| (first-order bound).
The test uses that bound per row, relative to the oracle's sum |a x|.
"""
import math

import numpy as np
import pytest
import torch

import workloads as wl
from oracle import mv as MV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


def _tol(n):
    return (math.ceil(n / 32) + 8) * 2.0 ** -24


def _check(y, A_q, x, rows=None):
    """y (float32 result rows) against the oracle on the quantised matrix A_q (float64 rows of
    A, or only the given rows of it)."""
    ref = MV.mv_rows(A_q, x)
    scale = MV.mv_abs_rows(A_q, x)
    got = y.double().cpu().numpy() if rows is None else y.double().cpu().numpy()[np.asarray(rows)]
    err = np.abs(got - ref) / np.maximum(scale, np.finfo(np.float64).tiny)
    assert err.max() <= _tol(A_q.shape[1]), (err.max(), _tol(A_q.shape[1]))


@pytest.mark.parametrize("shape", [(1, 1), (5, 3), (37, 1000), (256, 4097), (1000, 64), (3, 8192)])
@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.float16])
def test_mv_matches_oracle(shine, shape, dtype):
    m, n = shape
    A, x = wl.mv_inputs(m, n, seed=m * 31 + n)
    Aq = A.to(dtype)
    y = shine.mv(Aq.cuda(), x.cuda())
    torch.cuda.synchronize()
    _check(y, Aq.double().numpy(), x.double().numpy())


def test_mv_small_against_the_pattern_form(shine):
    """Against the list form of the paper's mv itself (not only the numpy row reduction)."""
    A, x = wl.mv_inputs(13, 29, seed=4)
    y = shine.mv(A.cuda(), x.cuda()).double().cpu().numpy()
    ref = np.array(MV.mv(A.double().tolist(), x.double().tolist()))
    scale = MV.mv_abs_rows(A.double().numpy(), x.double().numpy())
    assert np.all(np.abs(y - ref) <= _tol(29) * scale)


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_mv_unaligned_rows_and_vector(shine, dtype):
    """Row pitch not a multiple of 16 bytes and x not 16-byte aligned: the element path."""
    m, n = 70, 1001
    A, x = wl.mv_inputs(m, n + 1, seed=9)
    Aq = A.to(dtype).cuda()[:, :n]            # pitch n + 1 elements
    xb = torch.cat([torch.zeros(1), x[:n]]).cuda()[1:]   # offset by one float
    y = shine.mv(Aq, xb)
    torch.cuda.synchronize()
    _check(y, Aq.double().cpu().numpy(), xb.double().cpu().numpy())


def test_mv_degenerate_shapes(shine):
    A = torch.empty(4, 0, device="cuda")
    y = shine.mv(A, torch.empty(0, device="cuda"))
    assert torch.equal(y.cpu(), torch.zeros(4))   # reduce(+, 0) of empty rows
    y = shine.mv(torch.empty(0, 7, device="cuda"), torch.ones(7, device="cuda"))
    assert y.shape == (0,)


def test_mv_deterministic(shine):
    A, x = wl.mv_inputs(300, 5000, seed=2)
    Ad, xd = A.cuda(), x.cuda()
    assert torch.equal(shine.mv(Ad, xd), shine.mv(Ad, xd))


def test_mv_rejects_bad_arguments(shine):
    from paper_2201_03611_b300 import _lib as L
    lib = L.lib()
    y = torch.empty(4, device="cuda")
    x = torch.empty(8, device="cuda")
    A = torch.empty(4, 8, device="cuda")
    assert lib.shine_mv(A.data_ptr(), 4, 8, 7, 0, x.data_ptr(), y.data_ptr(), None) == L.SHINE_ERR_INVALID_ARG
    assert lib.shine_mv(A.data_ptr(), -1, 8, 8, 0, x.data_ptr(), y.data_ptr(), None) == L.SHINE_ERR_INVALID_ARG
    assert lib.shine_mv(A.data_ptr() + 2, 4, 8, 8, 0, x.data_ptr(), y.data_ptr(), None) == L.SHINE_ERR_ALIGNMENT
    assert lib.shine_mv(A.data_ptr(), 4, 8, 8, 0, x.data_ptr(), None, None) == L.SHINE_ERR_INVALID_ARG


@pytest.mark.slow
def test_mv_full_size_sampled(shine):
    """The 16384 x 16384 float32 workload of the benchmark, in the launch configuration the
    benchmark times, on sampled rows (first, last, random)."""
    m = n = 16384
    A, x = wl.mv_inputs(m, n, seed=0)
    y = shine.mv(A.cuda(), x.cuda())
    torch.cuda.synchronize()
    rows = sorted(set([0, 1, m - 1] + torch.randint(0, m, (200,), generator=torch.Generator().manual_seed(5)).tolist()))
    _check(y, A[rows].double().numpy(), x.double().numpy(), rows)
