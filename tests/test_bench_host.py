"""Host-side helpers of bench.py (no GPU)."""
from __future__ import annotations

import sys
from pathlib import Path

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))

import bench  # noqa: E402


def test_slice_bounds_cover_the_queries_in_growing_slices():
    for m in (0, 1, 3, 1000, 10_000_000):
        for nb in (1, 2, 4, 7):
            for g in (1.0, 1.5, 2.0):
                b = bench.slice_bounds(m, nb, g)
                assert len(b) == nb + 1 and b[0] == 0 and b[-1] == m
                assert all(x <= y for x, y in zip(b, b[1:]))
    assert bench.slice_bounds(10_000_000, 4, 1.0) == [0, 2_500_000, 5_000_000, 7_500_000, 10_000_000]
    assert bench.slice_bounds(15_000, 4, 2.0) == [0, 1000, 3000, 7000, 15_000]
