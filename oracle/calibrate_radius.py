"""Calibrate the radius of the large mixture workload with the CPU oracle.

The workload asks for a radius giving a mean of 32 neighbours per query.  This
script takes 1000 seeded calibration queries from the mixture, and finds the
smallest float32 r such that the exact mean count over those queries, against
all 10M points, is at least 32 (a binary search over float32 bit patterns, each
step an all-pairs count by the oracle).  It prints the bits, which are stored
as ``LARGE_RADIUS_BITS`` in the ``workloads`` package.

Run: python oracle/calibrate_radius.py [--n 10000000] [--target 32]
"""
from __future__ import annotations

import argparse
import sys
import time
from pathlib import Path

import numpy as np

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
import oracle  # noqa: E402
import workloads  # noqa: E402


def f2b(x: float) -> int:
    return int(np.array([x], np.float32).view(np.uint32)[0])


def b2f(b: int) -> np.float32:
    return np.array([b], np.uint32).view(np.float32)[0]


def calibrate(points: np.ndarray, queries: np.ndarray, target: float, lo: float, hi: float) -> int:
    m = len(queries)

    def mean_count(bits: int) -> float:
        return oracle.radius_count(points, queries, float(b2f(bits))).astype(np.int64).sum() / m

    lo_b, hi_b = f2b(lo), f2b(hi)
    assert mean_count(hi_b) >= target, "upper bracket too small"
    while hi_b - lo_b > 1:
        mid = (lo_b + hi_b) // 2
        t0 = time.time()
        c = mean_count(mid)
        print(f"  r={float(b2f(mid)):.9g} mean={c:.4f} ({time.time() - t0:.1f}s)", flush=True)
        if c >= target:
            hi_b = mid
        else:
            lo_b = mid
    return hi_b


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--target", type=float, default=32.0)
    ap.add_argument("--lo", type=float, default=1e-6)
    ap.add_argument("--hi", type=float, default=1e-1)
    a = ap.parse_args()
    wl = workloads.large_mixture(n=a.n, m=1)
    qs = workloads.large_mixture_calibration_queries(1000)
    bits = calibrate(wl["points"], qs, a.target, a.lo, a.hi)
    print(f"LARGE_RADIUS_BITS = 0x{bits:08x}  # r = {float(b2f(bits)):.9g}")


if __name__ == "__main__":
    main()
