"""Parity of shine_iterate_sum (iterate with double buffering, Sec. 6) with the oracle.

Every addition of the kernel is one of the pattern's, in the pattern's order, so the float32
result must equal the oracle's float32 evaluation of the same definition bit for bit; it is
also checked against the FP64 oracle within the first-order tree-sum bound k (n-1) 2^-24 sum|x|.
"""
import numpy as np
import pytest
import torch

import workloads as wl
from oracle import iterate_sum as IT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shine():
    import paper_2201_03611_b300 as S
    return S


CASES = [(1, 1, 0), (5, 2, 3), (7, 4, 5), (1000, 4, 5), (33, 3, 4), (100, 16, 2), (9, 5, 1),
         (25, 2, 13), (2, 4, 7), (6145, 4, 1), (3000, 8, 3), (77, 1, 6)]


@pytest.mark.parametrize("m,n,k", CASES)
def test_iterate_sum_matches_oracle(shine, m, n, k):
    x = wl.iterate_inputs(m, n, k, seed=m + 10 * n + k)
    y = shine.iterate_sum(x.cuda(), n, k).cpu().numpy()
    x32 = x.numpy()
    assert np.array_equal(y, IT.iterate_sum_np(x32, n, k, np.float32))
    ref = IT.iterate_sum_np(x32, n, k, np.float64)
    assert np.all(np.abs(y - ref) <= IT.tree_bound(x32, n, k, 2.0 ** -24) + 1e-30)


def test_iterate_sum_small_against_the_pattern_form(shine):
    x = wl.iterate_inputs(3, 2, 4, seed=1)
    y = shine.iterate_sum(x.cuda(), 2, 4).cpu().numpy()
    ref = np.array(IT.iterate_sum(x.double().tolist(), 2, 4))
    assert np.all(np.abs(y - ref) <= IT.tree_bound(x.numpy(), 2, 4, 2.0 ** -24) + 1e-30)


def test_iterate_sum_unaligned_input(shine):
    """Input not 16-byte aligned: the scalar round-0 path, same bits."""
    m, n, k = 50, 4, 3
    x = wl.iterate_inputs(m, n, k, seed=3)
    xb = torch.cat([torch.zeros(1), x]).cuda()[1:]
    y = shine.iterate_sum(xb, n, k).cpu().numpy()
    assert np.array_equal(y, IT.iterate_sum_np(x.numpy(), n, k, np.float32))


def test_iterate_sum_limits(shine):
    from paper_2201_03611_b300 import _lib as L
    x = torch.ones(4 ** 8, device="cuda")
    out = torch.empty(1, device="cuda")
    # n^(k-1) = 4^7 = 16384 round-1 values do not fit one shared buffer
    assert L.lib().shine_iterate_sum(x.data_ptr(), 1, 4, 8, out.data_ptr(), None) == L.SHINE_ERR_UNSUPPORTED
    assert L.lib().shine_iterate_sum(x.data_ptr(), 1, 0, 2, out.data_ptr(), None) == L.SHINE_ERR_INVALID_ARG
    assert L.lib().shine_iterate_sum(x.data_ptr() + 2, 1, 4, 2, out.data_ptr(), None) == L.SHINE_ERR_ALIGNMENT
    # the largest supported group: n^(k-1) == 4096 <= 6144
    y = shine.iterate_sum(torch.ones(4 ** 7, device="cuda"), 4, 7)
    assert y.item() == 4.0 ** 7


def test_iterate_sum_full_size_sampled(shine):
    """The benchmark workload (m = 262144 groups of 4^5, 1 GiB of float32): every output
    against the float32 oracle."""
    m, n, k = 262144, 4, 5
    x = wl.iterate_inputs(m, n, k, seed=0)
    y = shine.iterate_sum(x.cuda(), n, k).cpu().numpy()
    assert np.array_equal(y, IT.iterate_sum_np(x.numpy(), n, k, np.float32))


@pytest.mark.parametrize("op", ["max", "min"])
@pytest.mark.parametrize("m,n,k", [(5, 2, 3), (1000, 4, 5), (33, 3, 4), (2, 4, 7), (6145, 4, 1)])
def test_iterate_max_min_match_oracle(shine, op, m, n, k):
    """max / min folds are exact: the kernel equals the oracle bit for bit, whatever the order."""
    x = wl.iterate_inputs(m, n, k, seed=m + n + k)
    y = shine.iterate_sum(x.cuda(), n, k, op=op).cpu().numpy()
    assert np.array_equal(y, IT.iterate_fold_np(x.numpy(), n, k, op, np.float32))


def test_iterate_max_ignores_nan_operands(shine):
    x = torch.tensor([1.0, float("nan"), -2.0, 0.5, float("nan"), float("nan"), 3.0, -1.0])
    y = shine.iterate_sum(x.cuda(), 2, 2, op="max").cpu().numpy()
    assert np.array_equal(y, IT.iterate_fold_np(x.numpy(), 2, 2, "max", np.float32))
    assert y[0] == 1.0 and y[1] == 3.0
