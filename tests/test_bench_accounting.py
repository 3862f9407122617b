"""The algorithmic work the bench's roofline line divides by, against direct enumeration.

One step l -> l + 1 of the recursion updates half rows A = 0 .. l (columns B = 0 .. A + 1) and
integer rows m = 0 .. l + 1 (columns n = 0 .. m); the sweep runs l = 0 .. L - 2."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


@pytest.mark.parametrize("L", [1, 2, 3, 7, 40, 129])
def test_recursion_update_counts(L):
    import bench
    half = sum(A + 2 for l in range(L - 1) for A in range(l + 1))
    integer = sum(m + 1 for l in range(L - 1) for m in range(l + 2))
    assert bench.recursion_updates(L) == (float(half), float(integer))


def test_contraction_macs_count_the_triangle():
    """Per field and direction: sum over l >= |s| (no coefficients below) of (2l + 1) orders m
    times (l + 1) columns m' >= 0."""
    import bench
    L, s = 37, -2
    direct = sum((2 * l + 1) * (l + 1) for l in range(abs(s), L))
    assert bench.contraction_macs(L, s) == pytest.approx(direct)


@pytest.mark.parametrize("L", [1, 2, 33, 64, 100])
def test_column_recursion_counts(L):
    """Column recursion: in degree l the lane of column m walks rows l down to 32 floor(m/32) (its
    block's first row) and updates once per row below the first.  Degree-lane recursion: the lane of
    degree l in the task of column m walks rows l down to m.  Entries: (l+1)^2 per degree."""
    import bench
    col = sum(l - 32 * (m // 32) for l in range(L) for m in range(l + 1))
    lane = sum(l - m for l in range(L) for m in range(l + 1))
    assert bench.column_updates(L) == float(col)
    assert bench.lane_updates(L) == float(lane)
    assert bench.quadrant_entries(L) == float(sum((l + 1) ** 2 for l in range(L)))


def test_torus_fft_length():
    import bench
    for L in (1, 2, 16, 33, 512, 1024, 2048):
        M = bench.torus_M(L)
        N = 2 * L - 1
        assert M >= 2 * N - 1 and M >= 128 and (M & (M - 1)) == 0 and (M // 2 < 2 * N - 1 or M == 128)
