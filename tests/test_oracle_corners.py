"""Pins of the corner step's oracle (threshold + 3x3 non-maximum suppression) against hand
cases and brute force, independent of any kernel."""
import numpy as np
import pytest

from oracle import corners as C


def both(R, t):
    a, b = C.nms_loop(R, t), C.nms(R, t)
    assert np.array_equal(a, b)
    return a


def test_single_peak_in_a_flat_field():
    R = np.zeros((7, 9), dtype=np.float32)
    R[3, 4] = 5.0
    m = both(R, 1.0)
    assert m.sum() == 1 and m[3, 4] == 1


def test_threshold_is_strict():
    R = np.zeros((5, 5), dtype=np.float32)
    R[2, 2] = 1.0
    assert both(R, 1.0).sum() == 0
    assert both(R, np.nextafter(np.float32(1.0), np.float32(0.0))).sum() == 1


def test_ties_keep_every_tied_maximum():
    R = np.zeros((6, 6), dtype=np.float32)
    R[2:4, 2:4] = 3.0              # a 2 x 2 plateau: each cell >= all its neighbours
    m = both(R, 0.0)
    assert m.sum() == 4 and m[2:4, 2:4].all()
    R[2, 3] = 3.5                  # now one cell dominates its plateau neighbours
    m = both(R, 0.0)
    assert m.sum() == 1 and m[2, 3] == 1


def test_border_neighbours_outside_are_ignored():
    R = np.zeros((4, 5), dtype=np.float32)
    R[0, 0] = 2.0
    R[3, 4] = 2.0
    m = both(R, 0.0)
    assert m[0, 0] == 1 and m[3, 4] == 1 and m.sum() == 2


def test_ramp_keeps_only_its_last_column():
    R = np.tile(np.arange(6, dtype=np.float32), (4, 1))   # increasing along x, equal along y
    m = both(R, -1.0)
    assert m[:, -1].all() and m[:, :-1].sum() == 0


def test_nan_is_never_a_corner_and_constant_field_is_all_corners():
    R = np.full((3, 3), 1.0, dtype=np.float32)
    assert both(R, 0.0).sum() == 9
    R[1, 1] = np.nan
    m = both(R, 0.0)
    assert m[1, 1] == 0
    # no value is >= NaN: every pixel with the NaN among its neighbours is no corner either
    assert m.sum() == 0
    R = np.full((3, 5), 1.0, dtype=np.float32)
    R[1, 0] = np.nan
    assert both(R, 0.0)[:, 2:].all() and both(R, 0.0)[:, :2].sum() == 0


@pytest.mark.parametrize("seed", range(6))
def test_vector_form_equals_the_loops_on_random_values_with_ties(seed):
    rng = np.random.default_rng(seed)
    R = rng.integers(-3, 4, size=(13, 17)).astype(np.float32)   # many exact ties
    t = float(rng.integers(-2, 2))
    m = both(R, t)
    # brute-force restatement: the pixel equals the max of its clipped 3x3 window
    for y in range(13):
        for x in range(17):
            win = R[max(0, y - 1):y + 2, max(0, x - 1):x + 2]
            assert m[y, x] == (R[y, x] > t and R[y, x] == win.max())
