"""GPU parity of the counting traversal's contained-subtree rule.

The count callbacks and the CRS count pass add the leaf count of an internal
child whose box lies inside the query's sphere (or box) instead of visiting
it.  Counts must still equal the oracle's brute-force counts exactly, for radii
from a few neighbours up to beyond the whole scene (r*r overflowing to +inf),
every dimension, the count-up-to limits, staged top levels (re-coded child
codes) and boxes on point and triangle trees (16-bit quantized nodes keep no
range ends and take the plain traversal).  The instrumented counting traversal gives closed forms:
with a radius beyond the scene every query fetches the root only and counts
all n leaves.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
import workloads
from crs_util import assert_crs_equal, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arbx():
    import paper_2507_23700_b300 as m
    return m


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def clustered(n, dim, seed):
    """Points in a few tight clusters plus a uniform background and exact
    duplicates (whole subtrees of equal points)."""
    rng = np.random.default_rng(seed)
    centers = rng.random((8, dim))
    lab = rng.integers(0, 8, n)
    pts = centers[lab] + rng.normal(0, 0.01, (n, dim))
    bg = rng.random((n // 4, dim))
    dup = np.repeat(rng.random((4, dim)), 200, axis=0)
    return np.concatenate([pts, bg, dup]).astype(np.float32)


TUNINGS = [None, dict(top_levels=255), dict(sort_queries=0, top_levels=1023)]


@pytest.mark.parametrize("dim", [2, 3, 6])
def test_counts_at_growing_radii(arbx, dim):
    pts = clustered(12000, dim, 40 + dim)
    rng = np.random.default_rng(50 + dim)
    qs = np.concatenate([pts[rng.integers(0, len(pts), 1500)], rng.random((500, dim))]).astype(np.float32)
    t = arbx.Tree(cu(pts))
    q = cu(qs)
    for r in (0.005, 0.03, 0.1, 0.4, 2.0 * math.sqrt(dim), 1e18, 3e19):
        ref = oracle.radius_count(pts, qs, r)
        for tu in TUNINGS:
            assert np.array_equal(to_np(t.count(q, r, tuning=tu)), ref), (dim, r, tu)
        for lim in (1, 7, 300):
            assert np.array_equal(to_np(t.count_up_to(q, r, lim)), np.minimum(ref, lim)), (dim, r, lim)
        assert np.array_equal(to_np(t.first_hit(q, r)), (ref >= 1).astype(np.int32))
    # CRS at a radius that contains whole clusters: the counted segments must
    # be exactly what the fill pass lists
    assert_crs_equal(t.radius(q, 0.1), oracle.radius(pts, qs, 0.1), what=f"radius {dim}D")


def test_per_query_radii_with_huge_and_zero(arbx):
    pts = clustered(20000, 3, 61)
    rng = np.random.default_rng(62)
    qs = pts[rng.integers(0, len(pts), 3000)]
    radii = np.where(rng.random(3000) < 0.3, rng.uniform(0.2, 3.0, 3000),
                     np.where(rng.random(3000) < 0.5, 0.0, rng.uniform(0, 0.05, 3000))).astype(np.float32)
    t = arbx.Tree(cu(pts))
    ref = oracle.radius_count(pts, qs, radii)
    assert np.array_equal(to_np(t.count(cu(qs), cu(radii))), ref)
    assert_crs_equal(t.radius(cu(qs), cu(radii)), oracle.radius(pts, qs, radii), what="mixed radii")


def test_big_boxes_on_points_and_triangles(arbx):
    pts = clustered(15000, 3, 71)
    rng = np.random.default_rng(72)
    c = rng.random((1500, 3)).astype(np.float32)
    h = rng.choice([0.02, 0.2, 0.6, 2.0], (1500, 1)).astype(np.float32) * np.ones((1, 3), np.float32)
    boxes = np.concatenate([c - h, c + h], 1).astype(np.float32)
    t = arbx.Tree(cu(pts))
    off, idx = t.box(cu(boxes))
    assert_crs_equal((off, idx, None), oracle.box_query(pts, oracle.POINT, boxes), check_d2=False,
                     what="big boxes on points")
    tris = workloads.heightfield_triangles(65, 33, seed=73)
    v = tris.reshape(-1, 3)
    lo, hi = v.min(0), v.max(0)
    cb = (lo + rng.random((800, 3)) * (hi - lo)).astype(np.float32)
    hb = (rng.choice([0.01, 0.1, 0.5], (800, 1)) * (hi - lo)).astype(np.float32)
    tboxes = np.concatenate([cb - hb, cb + hb], 1).astype(np.float32)
    ref = oracle.box_query(tris, oracle.TRIANGLE, tboxes)
    for quantized in (False, True, "parent"):
        tt = arbx.Tree(cu(tris), kind="triangle", quantized=quantized)
        toff, tidx = tt.box(cu(tboxes))
        assert_crs_equal((toff, tidx, None), ref, check_d2=False, what=f"big boxes on triangles q={quantized}")


def test_counting_stats_closed_forms(arbx):
    pts = clustered(10000, 3, 81)
    n = len(pts)
    rng = np.random.default_rng(82)
    qs = rng.random((777, 3)).astype(np.float32)
    t = arbx.Tree(cu(pts))
    q = cu(qs)
    full = t.stats(arbx.SPHERE, q, 1e18)
    cnt = t.stats(arbx.SPHERE, q, 1e18, counting=True)
    # a radius beyond the scene: the root's children are leaves or contained subtrees
    assert cnt["nodes"] == len(qs) and cnt["matches"] == len(qs) * n
    assert full["matches"] == len(qs) * n and full["nodes"] == len(qs) * (n - 1)
    for r in (0.01, 0.1):
        full = t.stats(arbx.SPHERE, q, r)
        cnt = t.stats(arbx.SPHERE, q, r, counting=True)
        assert cnt["matches"] == full["matches"] == int(oracle.radius_count(pts, qs, r).sum())
        assert cnt["nodes"] <= full["nodes"]
    with pytest.raises(Exception):
        t.stats(arbx.NEAREST, q, k=4, counting=True)
