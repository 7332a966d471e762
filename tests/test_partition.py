"""The kernels' work partition (host logic, no GPU): every (segment, row) unit goes to exactly
one warp, for both layouts and any edge weight; the weighted layouts give the edge warps fewer
rows; the band-major layout keeps each warp on one segment."""
import ctypes
import random

import pytest

from paper_2201_03611_b300 import _lib as L


def _ranges(nseg, rows, t, band_major, ew4):
    lib = L.lib()
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    out = []
    for w in range(t):
        assert lib.shine_partition(nseg, rows, t, w, band_major, ew4, ctypes.byref(lo), ctypes.byref(hi)) == 0
        out.append((lo.value, hi.value))
    return out


@pytest.mark.parametrize("band_major", [0, 1])
@pytest.mark.parametrize("ew4", [4, 5, 6, 8])
def test_every_unit_exactly_once(band_major, ew4):
    rng = random.Random(band_major * 10 + ew4)
    for _ in range(150):
        nseg, rows, t = rng.randint(1, 75), rng.randint(1, 260), rng.randint(1, 2500)
        cover = [0] * (nseg * rows)
        for lo, hi in _ranges(nseg, rows, t, band_major, ew4):
            assert 0 <= lo <= hi <= nseg * rows
            for u in range(lo, hi):
                cover[u] += 1
        assert all(c == 1 for c in cover), (nseg, rows, t)


def test_band_major_warps_stay_on_one_segment_and_edges_get_shorter_bands():
    nseg, rows, t = 70, 8192, 2368
    rs = _ranges(nseg, rows, t, 1, 6)
    edge, inner = [], []
    for lo, hi in rs:
        if hi > lo:
            assert lo // rows == (hi - 1) // rows            # one segment per warp
            (edge if lo // rows in (0, nseg - 1) else inner).append(hi - lo)
    assert max(edge) < min(inner)                          # edge bands are shorter


def test_weighted_split_gives_edge_warps_fewer_rows():
    nseg, rows, t = 70, 8192, 1184
    rs = _ranges(nseg, rows, t, 0, 6)
    first = rs[0][1] - rs[0][0]                             # inside edge segment 0
    middle = rs[t // 2][1] - rs[t // 2][0]
    assert first * 6 == pytest.approx(middle * 4, rel=0.01)


def test_rejects_bad_arguments():
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    assert L.lib().shine_partition(0, 1, 1, 0, 0, 4, ctypes.byref(lo), ctypes.byref(hi)) == L.SHINE_ERR_INVALID_ARG
    assert L.lib().shine_partition(1, 1, 1, 1, 0, 4, ctypes.byref(lo), ctypes.byref(hi)) == L.SHINE_ERR_INVALID_ARG
