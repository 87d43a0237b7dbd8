"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bit-exact bar: identical neighbour sets per query and bit-identical float32
squared distances (the method is exact; both sides round every operation the
same way), identical kNN lists including the (d2, index) order, identical
callback counts.  Sizes span several tiles and ragged tails; edge cases cover
empty, one-, two-point and duplicate-heavy inputs, k > n and every dimension
built.
"""
from __future__ import annotations

import json
import math
from pathlib import Path

import numpy as np
import pytest
import torch

import oracle
import workloads
from crs_util import assert_crs_equal, to_np

pytestmark = pytest.mark.gpu

GOLDEN = json.loads((Path(__file__).parent / "golden" / "hand_cases.json").read_text())


@pytest.fixture(scope="module")
def arbx():
    import paper_2507_23700_b300 as m
    return m


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def gpu_radius(arbx, pts, qs, r, **kw):
    t = arbx.Tree(cu(pts))
    off, idx, d2 = t.radius(cu(qs), r, **kw)
    return to_np(off), to_np(idx), to_np(d2)


# ------------------------------------------------------------------ golden

@pytest.mark.parametrize("case", GOLDEN["radius"], ids=lambda c: c["name"])
def test_golden_radius(arbx, case):
    dim = len(case["queries"][0])
    pts = np.asarray(case["points"], np.float32).reshape(-1, dim)
    off, idx, d2 = gpu_radius(arbx, pts, np.asarray(case["queries"], np.float32), case["radius"])
    for i, (ei, ed) in enumerate(zip(case["indices"], case["d2"])):
        seg = sorted(zip(idx[off[i]:off[i + 1]].tolist(), d2[off[i]:off[i + 1]].tolist()))
        assert [j for j, _ in seg] == ei
        assert [e for _, e in seg] == ed


@pytest.mark.parametrize("case", GOLDEN["knn"], ids=lambda c: c["name"])
def test_golden_knn(arbx, case):
    dim = len(case["queries"][0])
    t = arbx.Tree(cu(np.asarray(case["points"], np.float32).reshape(-1, dim)))
    idx, d2 = t.knn(cu(case["queries"]), case["k"])
    assert to_np(idx).tolist() == case["indices"]
    assert to_np(d2).tolist() == case["d2"]


@pytest.mark.parametrize("quantized", [False, True, "parent"])
def test_golden_rays(arbx, quantized):
    tris = np.asarray(GOLDEN["rays"]["triangles"], np.float32)
    rays = np.asarray([c["ray"] for c in GOLDEN["rays"]["cases"]], np.float32)
    t = arbx.Tree(cu(tris), kind="triangle", quantized=quantized)
    hit, tt = t.ray_nearest(cu(rays))
    for c, h, v in zip(GOLDEN["rays"]["cases"], to_np(hit), to_np(tt)):
        assert h == c["hit"], c["name"]
        assert float(v) == (math.inf if c["t"] == "inf" else c["t"]), c["name"]


@pytest.mark.parametrize("case", GOLDEN["boxes"], ids=lambda c: c["name"])
def test_golden_boxes(arbx, case):
    kind = case["kind"]
    prims = np.asarray(case["prims"], np.float32)
    for q in ([False, True, "parent"] if kind == "triangle" else [False]):
        t = arbx.Tree(cu(prims), kind=kind, quantized=q)
        off, idx = t.box(cu(case["boxes"]))
        off, idx = to_np(off), to_np(idx)
        for i, e in enumerate(case["indices"]):
            assert sorted(idx[off[i]:off[i + 1]].tolist()) == e


# ------------------------------------------------------------------ tiny uniform workload

@pytest.fixture(scope="module")
def tiny():
    wl = workloads.tiny_uniform()
    wl["ref_radius"] = oracle.radius(wl["points"], wl["queries"], wl["radius"])
    wl["ref_knn"] = oracle.knn(wl["points"], wl["queries"], wl["k"])
    return wl


def test_tiny_radius_crs(arbx, tiny):
    t = arbx.Tree(cu(tiny["points"]))
    off, idx, d2 = t.radius(cu(tiny["queries"]), tiny["radius"])
    assert_crs_equal((off, idx, d2), tiny["ref_radius"], what="tiny radius")
    # two-phase form into torch-allocated buffers gives the same bytes
    off2, idx2, d22 = t.offsets_fill(arbx.SPHERE, cu(tiny["queries"]), tiny["radius"])
    assert torch.equal(off, off2) and torch.equal(idx, idx2) and torch.equal(d2, d22)


def test_tiny_callbacks(arbx, tiny):
    t = arbx.Tree(cu(tiny["points"]))
    q = cu(tiny["queries"])
    cnt = np.diff(tiny["ref_radius"][0])
    assert np.array_equal(to_np(t.count(q, tiny["radius"])), cnt)
    for lim in (0, 1, 5, 16, 1000):
        got = to_np(t.count_up_to(q, tiny["radius"], lim))
        assert np.array_equal(got, oracle.radius_count_up_to(tiny["points"], tiny["queries"], tiny["radius"], lim))
        assert np.array_equal(got, np.minimum(cnt, lim))
    assert np.array_equal(to_np(t.first_hit(q, tiny["radius"])), (cnt >= 1).astype(np.int32))


def test_tiny_knn(arbx, tiny):
    t = arbx.Tree(cu(tiny["points"]))
    idx, d2 = t.knn(cu(tiny["queries"]), tiny["k"])
    ridx, rd2 = tiny["ref_knn"]
    assert np.array_equal(to_np(idx), ridx)
    assert np.array_equal(to_np(d2).view(np.uint32), rd2.view(np.uint32))
    crs = t.query_crs(arbx.NEAREST, cu(tiny["queries"]), k=tiny["k"])
    assert np.array_equal(to_np(crs.offsets), np.arange(len(ridx) + 1) * tiny["k"])
    assert np.array_equal(to_np(crs.indices), ridx.reshape(-1))


TUNINGS = [dict(block=b, sort_queries=s, top_levels=tl) for b in (64, 256) for s in (0, 1) for tl in (0, 255, 1023)]


def test_tuning_invariance(arbx, tiny):
    """Every launch shape, query order and shared-memory staging gives
    byte-identical output, including the order within each segment."""
    t = arbx.Tree(cu(tiny["points"]), wide=True)
    q = cu(tiny["queries"])
    base = t.radius(q, tiny["radius"], tuning=TUNINGS[0])
    kbase = t.knn(q, 16, tuning=TUNINGS[0])
    for tu in TUNINGS[1:] + [dict(grid_per_sm=1), dict(warp_refill=0), dict(warp_refill=1),
                             dict(warp_refill=0, top_levels=1023, block=128), dict(stackless=1),
                             dict(stackless=1, top_levels=0), dict(stackless=1, top_levels=255, warp_refill=1),
                             dict(stackless=0), dict(single_pass=0), dict(single_pass=0, stackless=1),
                             dict(single_pass=1, top_levels=1023, block=64), dict(lanes_per_query=1),
                             dict(lanes_per_query=2), dict(lanes_per_query=4, block=128),
                             dict(lanes_per_query=8, warp_refill=1), dict(lanes_per_query=8, top_levels=255),
                             dict(wide_nodes=0), dict(wide_nodes=1, block=64), dict(wide_nodes=1, warp_refill=1),
                             dict(wide_nodes=1, sort_queries=0), dict(wide_nodes=0, top_levels=0),
                             dict(warp_packets=1), dict(warp_packets=1, sort_queries=0, block=128),
                             dict(query_runs=1), dict(query_runs=4, block=64), dict(query_runs=8, top_levels=255),
                             dict(query_runs=8, sort_queries=0)]:
        got = t.radius(q, tiny["radius"], tuning=tu)
        assert all(torch.equal(a, b) for a, b in zip(base, got)), tu
        kg = t.knn(q, 16, tuning=tu)
        assert torch.equal(kbase[0], kg[0]) and torch.equal(kbase[1], kg[1]), tu


def test_leaf_order_is_morton_order(arbx, tiny):
    """Within each segment the matches come in left-to-right leaf order, which
    is the order of the tree's sorted leaves."""
    t = arbx.Tree(cu(tiny["points"]))
    ex = t.export()
    nodes = ex["nodes"].view(node_dtype(3))
    leaf_orig = {}
    for c in range(2):
        lc = nodes["child"][:, c] < 0
        leaf_orig.update(zip((~nodes["child"][lc, c]).tolist(), nodes["orig"][lc, c].tolist()))
    rank = np.empty(len(tiny["points"]), np.int64)
    for pos, o in leaf_orig.items():
        rank[o] = pos
    off, idx, _ = (to_np(x) for x in t.radius(cu(tiny["queries"]), tiny["radius"]))
    r = rank[idx]
    seg = np.repeat(np.arange(len(off) - 1), np.diff(off))
    inner = seg[1:] == seg[:-1]
    assert np.all(r[1:][inner] > r[:-1][inner])


# ------------------------------------------------------------------ sizes, dims, edges

@pytest.mark.parametrize("dim", [2, 3, 6])
@pytest.mark.parametrize("n,m", [(1, 5), (2, 7), (3, 33), (31, 64), (4097, 1000), (20011, 3001)])
def test_sizes_and_dims(arbx, dim, n, m):
    rng = np.random.default_rng(n * 10 + dim)
    pts = rng.random((n, dim), dtype=np.float32)
    qs = rng.random((m, dim), dtype=np.float32)
    r = float((12.0 / (workloads.unit_ball_volume(dim) * max(n, 1))) ** (1.0 / dim))
    t = arbx.Tree(cu(pts))
    assert t.size() == n
    assert_crs_equal(t.radius(cu(qs), r), oracle.radius(pts, qs, r), what=f"radius n={n} d={dim}")
    for k in (1, 3, 8, 32):
        idx, d2 = t.knn(cu(qs), k)
        ridx, rd2 = oracle.knn(pts, qs, k)
        assert np.array_equal(to_np(idx), ridx), (k, n, dim)
        assert np.array_equal(to_np(d2).view(np.uint32), rd2.view(np.uint32)), (k, n, dim)
    lo, hi = t.bounds()
    assert np.array_equal(np.float32(lo), pts.min(0)) and np.array_equal(np.float32(hi), pts.max(0))


@pytest.mark.parametrize("dim", [2, 3, 6])
@pytest.mark.parametrize("n", [50, 7001])
def test_knn_long_lists(arbx, dim, n):
    """32 < k <= 256: lists spread over lane groups of k/8 lanes (k = 33 and
    100 use the 64- and 128-key lists with the columns below k written);
    k > n gives n columns."""
    rng = np.random.default_rng(1000 + n + dim)
    pts = rng.random((n, dim), dtype=np.float32)
    pts[n // 3: n // 3 + 9] = pts[0]  # duplicates: ties broken by index
    qs = rng.random((613, dim), dtype=np.float32)
    t = arbx.Tree(cu(pts))
    for k in (33, 64, 100, 128, 200, 256):
        ridx, rd2 = oracle.knn(pts, qs, k)
        for tu in (None, dict(query_runs=1), dict(query_runs=8)):  # lane runs of the groups (default 4 in 2D/3D)
            idx, d2 = t.knn(cu(qs), k, tuning=tu)
            assert idx.shape == (len(qs), min(k, n))
            assert np.array_equal(to_np(idx), ridx), (k, n, dim, tu)
            assert np.array_equal(to_np(d2).view(np.uint32), rd2.view(np.uint32)), (k, n, dim, tu)


@pytest.mark.parametrize("scale", [1.0, 1e30, 1e-30, 1e3])
def test_knn_query_runs_edge_cases(arbx, scale):
    """Lane runs carry an upper bound on the k-th distance from a lane's
    previous query (rounded up, widened for float32 rounding and underflow).
    The bound must never prune a true neighbour: huge, tiny (subnormal d2) and
    offset coordinates, exact duplicates (ties), NaN queries between ordinary
    ones and k above n all give the oracle's rows under runs of 1, 4 and 8."""
    rng = np.random.default_rng(606)
    pts = rng.random((3001, 3)).astype(np.float64)
    pts[200:260] = pts[5]  # ties
    qs = rng.random((2500, 3))
    qs[1000:1100] = pts[5]
    if scale == 1e3:
        pts, qs = pts + 1e3, qs + 1e3
    else:
        pts, qs = pts * scale, qs * scale
    pts, qs = pts.astype(np.float32), qs.astype(np.float32)
    qs[7::97] = np.nan
    for tp, ks in ((pts, (1, 5, 16, 32)), (pts[:20], (8, 32))):  # the second: k above n
        t = arbx.Tree(cu(tp), wide=True)
        for k in ks:
            ridx, rd2 = oracle.knn(tp, qs, k)
            for r in (1, 4, 8):
                for wd in (0, 1):
                    idx, d2 = t.knn(cu(qs), k, tuning=dict(query_runs=r, wide_nodes=wd, warp_packets=0))
                    assert np.array_equal(to_np(idx), ridx), (scale, k, r, wd)
                    assert np.array_equal(to_np(d2).view(np.uint32), rd2.view(np.uint32)), (scale, k, r, wd)


@pytest.mark.parametrize("dim", [2, 3, 6])
def test_knn_lanes_per_query(arbx, dim):
    """Every lane-group size, and the four-wide records, give the oracle's
    rows for every list size; the wide records also give the oracle's counts."""
    rng = np.random.default_rng(77 + dim)
    pts = rng.random((9001, dim), dtype=np.float32)
    pts[100:140] = pts[7]  # duplicates
    qs = rng.random((1777, dim), dtype=np.float32)
    t = arbx.Tree(cu(pts), wide=True)
    for k in (1, 2, 3, 5, 8, 13, 16, 17, 32):
        ridx, rd2 = oracle.knn(pts, qs, k)
        for tu in [dict(lanes_per_query=L, warp_refill=rf) for L in (1, 2, 4, 8) for rf in (0, 1)] + \
                  [dict(wide_nodes=w, warp_refill=rf) for w in (0, 1) for rf in (0, 1)] + \
                  [dict(warp_packets=pk, block=b) for pk in (0, 1) for b in (64, 256)] + \
                  [dict(query_runs=r, block=b) for r in (1, 4, 8) for b in (64, 256)]:
            idx, d2 = t.knn(cu(qs), k, tuning=tu)
            assert np.array_equal(to_np(idx), ridx), (k, tu, dim)
            assert np.array_equal(to_np(d2).view(np.uint32), rd2.view(np.uint32)), (k, tu, dim)
    r = float((20.0 / (workloads.unit_ball_volume(dim) * len(pts))) ** (1.0 / dim))
    roff = oracle.radius(pts, qs, r)[0]
    for w in (0, 1):
        assert np.array_equal(to_np(t.count(cu(qs), r, tuning=dict(wide_nodes=w))), np.diff(roff)), w
        assert np.array_equal(to_np(t.count_up_to(cu(qs), r, 7, tuning=dict(wide_nodes=w))),
                              np.minimum(np.diff(roff), 7)), w
        off, _, _ = t.radius(cu(qs), r, tuning=dict(wide_nodes=w))
        assert np.array_equal(to_np(off), roff), w


def test_shared_query_order(arbx, tiny):
    """One Morton order (arbx_query_order) shared by several calls: it is a
    permutation, and every call given it returns the bytes it returns when it
    sorts the queries itself."""
    t = arbx.Tree(cu(tiny["points"]))
    q = cu(tiny["queries"])
    order = t.query_order(arbx.SPHERE, q, tiny["radius"])
    assert torch.equal(torch.sort(order.to(torch.int64)).values, torch.arange(q.shape[0], device="cuda"))
    korder = t.query_order(arbx.NEAREST, q, k=tiny["k"])
    assert torch.equal(order, korder)  # the same centres give the same order
    base = t.radius(q, tiny["radius"])
    got = t.radius(q, tiny["radius"], order=order)
    assert all(torch.equal(a, b) for a, b in zip(base, got))
    kb = t.knn(q, tiny["k"])
    kg = t.knn(q, tiny["k"], order=order)
    assert torch.equal(kb[0], kg[0]) and torch.equal(kb[1], kg[1])
    assert torch.equal(t.count(q, tiny["radius"]),
                       t.callback(arbx.SPHERE, q, arbx.CB_COUNT, tiny["radius"], order=order))
    # a reversed order is another permutation: still the same bytes
    rev = torch.flip(order, [0]).contiguous()
    got = t.radius(q, tiny["radius"], order=rev)
    assert all(torch.equal(a, b) for a, b in zip(base, got))
    # one query, and an empty tree
    assert to_np(t.query_order(arbx.SPHERE, q[:1], 0.1)).tolist() == [0]
    e = arbx.Tree(torch.zeros((0, 3), device="cuda"))
    assert to_np(e.query_order(arbx.SPHERE, q[:5], 0.1)).tolist() == [0, 1, 2, 3, 4]


STACKLESS = dict(stackless=1)


@pytest.mark.parametrize("dim", [2, 3, 6])
@pytest.mark.parametrize("n,m", [(1, 5), (2, 7), (3, 33), (31, 64), (4097, 1000), (20011, 3001)])
def test_stackless_sizes_and_dims(arbx, dim, n, m):
    """The stackless traversal against the oracle: radius CRS (sets, d2 bits
    and leaf order equal to the stack traversal's), count-up-to and boxes."""
    rng = np.random.default_rng(n * 10 + dim + 1)
    pts = rng.random((n, dim), dtype=np.float32)
    qs = rng.random((m, dim), dtype=np.float32)
    r = float((12.0 / (workloads.unit_ball_volume(dim) * max(n, 1))) ** (1.0 / dim))
    t = arbx.Tree(cu(pts))
    got = t.radius(cu(qs), r, tuning=STACKLESS)
    assert_crs_equal(got, oracle.radius(pts, qs, r), what=f"stackless radius n={n} d={dim}")
    ref = t.radius(cu(qs), r, tuning=dict(stackless=0))
    assert all(torch.equal(a, b) for a, b in zip(got, ref))
    for lim in (0, 1, 7):
        c = to_np(t.count_up_to(cu(qs), r, lim, tuning=STACKLESS))
        assert np.array_equal(c, oracle.radius_count_up_to(pts, qs, r, lim)), lim
    h = rng.uniform(0, 2 * r, (m, dim)).astype(np.float32)
    boxes = np.concatenate([qs - h, qs + h], 1)
    off, idx = t.box(cu(boxes), tuning=STACKLESS)
    roff, ridx = oracle.box_query(pts, oracle.POINT, boxes)
    assert_crs_equal((off, idx, None), (roff, ridx, None), check_d2=False, what="stackless boxes")
    arbx.stream_check()


def test_stackless_duplicates_and_triangles(arbx):
    """Tied Morton codes (index tie-break), per-query radii, and box queries on
    a float32 triangle tree, stackless."""
    p = np.tile(np.float32([0.3, 0.7, 0.1]), (1000, 1))
    t = arbx.Tree(cu(p))
    off, idx, d2 = t.radius(cu(p[:3]), 0.0, tuning=STACKLESS)
    assert to_np(off).tolist() == [0, 1000, 2000, 3000]
    assert all(sorted(to_np(idx)[i * 1000:(i + 1) * 1000].tolist()) == list(range(1000)) for i in range(3))
    rng = np.random.default_rng(9)
    pts = rng.random((30000, 3), dtype=np.float32)
    qs = rng.random((2000, 3), dtype=np.float32)
    radii = rng.uniform(0, 0.05, 2000).astype(np.float32)
    t = arbx.Tree(cu(pts))
    assert_crs_equal(t.radius(cu(qs), cu(radii), tuning=STACKLESS), oracle.radius(pts, qs, radii),
                     what="stackless per-query radii")
    tris = workloads.heightfield_triangles(65, 33, seed=3)
    tt = arbx.Tree(cu(tris), kind="triangle")
    c = np.concatenate([rng.uniform(0, 64 * workloads.HF_SPACING, (1500, 1)),
                        rng.uniform(0, 32 * workloads.HF_SPACING, (1500, 1)),
                        rng.uniform(0, 0.2, (1500, 1))], 1).astype(np.float32)
    hh = rng.uniform(0.002, 0.02, (1500, 3)).astype(np.float32)
    boxes = np.concatenate([c - hh, c + hh], 1)
    off, idx = tt.box(cu(boxes), tuning=STACKLESS)
    roff, ridx = oracle.box_query(tris, oracle.TRIANGLE, boxes)
    assert_crs_equal((off, idx, None), (roff, ridx, None), check_d2=False, what="stackless triangle boxes")


def test_single_pass_overflow_rerun(arbx):
    """Single-pass storage whose pool, sized from a sampled count pass, is far
    too small: the sampled (even) queries see no points, the others see
    hundreds, so most of them are re-run by the fill pass.  Same bytes as the
    two-pass form, and the oracle's on a subset."""
    rng = np.random.default_rng(12)
    pts = (0.5 + 0.01 * rng.standard_normal((20000, 3))).astype(np.float32)
    m = 131072
    qs = rng.random((m, 3), dtype=np.float32) * 0.2 + 0.8
    qs[1::2] = (0.5 + 0.005 * rng.standard_normal((m // 2, 3))).astype(np.float32)
    t = arbx.Tree(cu(pts))
    one = t.radius(cu(qs), 0.01, tuning=dict(single_pass=1))
    two = t.radius(cu(qs), 0.01, tuning=dict(single_pass=0))
    assert all(torch.equal(a, b) for a, b in zip(one, two))
    cnt = np.diff(to_np(one[0]))
    assert cnt[0::2].sum() == 0 and (cnt[1::2] > 8 * 32).mean() > 0.5
    sub = np.arange(3000)
    off = to_np(one[0])
    sel = np.concatenate([np.arange(off[i], off[i + 1]) for i in sub])
    sub_off = np.concatenate([[0], np.cumsum(cnt[sub])])
    assert_crs_equal((sub_off, to_np(one[1])[sel], to_np(one[2])[sel]), oracle.radius(pts, qs[sub], 0.01),
                     what="overflow re-run subset")
    off_b, idx_b = t.box(cu(np.concatenate([qs - 0.01, qs + 0.01], 1)), tuning=dict(single_pass=1))
    off_c, idx_c = t.box(cu(np.concatenate([qs - 0.01, qs + 0.01], 1)), tuning=dict(single_pass=0))
    assert torch.equal(off_b, off_c) and torch.equal(idx_b, idx_c)
    arbx.stream_check()


def test_empty_tree_and_empty_queries(arbx):
    t = arbx.Tree(torch.zeros((0, 3), device="cuda"))
    assert t.empty() and t.size() == 0
    q = cu(np.random.default_rng(0).random((10, 3)))
    off, idx, d2 = t.radius(q, 0.5)
    assert to_np(off).tolist() == [0] * 11 and idx.numel() == 0
    assert to_np(t.count(q, 0.5)).tolist() == [0] * 10
    ki, kd = t.knn(q, 4)
    assert ki.shape == (10, 0)
    t2 = arbx.Tree(cu(np.random.default_rng(1).random((100, 3))))
    off, idx, d2 = t2.radius(torch.zeros((0, 3), device="cuda"), 0.5)
    assert to_np(off).tolist() == [0]
    ki, kd = t2.knn(torch.zeros((0, 3), device="cuda"), 4)
    assert ki.shape == (0, 4)


def test_duplicates(arbx):
    """1000 identical points (the tree's codes all tie; the index breaks ties)
    and a two-cluster cloud of exact duplicates."""
    p = np.tile(np.float32([0.3, 0.7, 0.1]), (1000, 1))
    t = arbx.Tree(cu(p))
    off, idx, d2 = t.radius(cu(p[:1]), 0.0)
    assert sorted(to_np(idx).tolist()) == list(range(1000)) and not to_np(d2).any()
    ki, kd = t.knn(cu(p[:1]), 8)
    assert to_np(ki).tolist() == [list(range(8))]
    rng = np.random.default_rng(5)
    two = np.where(rng.random((5000, 1)) < 0.5, np.float32([0.25, 0.25, 0.25]), np.float32([0.75, 0.5, 0.25]))
    two = two.astype(np.float32)
    qs = rng.random((300, 3), dtype=np.float32)
    t = arbx.Tree(cu(two))
    assert_crs_equal(t.radius(cu(qs), 0.3), oracle.radius(two, qs, 0.3), what="two clusters")
    idx, d2 = t.knn(cu(qs), 32)
    ridx, rd2 = oracle.knn(two, qs, 32)
    assert np.array_equal(to_np(idx), ridx)


def test_per_query_radii_and_boxes_on_points(arbx):
    rng = np.random.default_rng(8)
    pts = rng.random((30000, 3), dtype=np.float32)
    qs = rng.random((2000, 3), dtype=np.float32)
    radii = rng.uniform(0, 0.05, 2000).astype(np.float32)
    t = arbx.Tree(cu(pts))
    assert_crs_equal(t.radius(cu(qs), cu(radii)), oracle.radius(pts, qs, radii), what="per-query radii")
    c = rng.random((2000, 3), dtype=np.float32)
    h = rng.uniform(0, 0.03, (2000, 3)).astype(np.float32)
    boxes = np.concatenate([c - h, c + h], 1)
    off, idx = t.box(cu(boxes))
    roff, ridx = oracle.box_query(pts, oracle.POINT, boxes)
    assert_crs_equal((off, idx, None), (roff, ridx, None), check_d2=False, what="box on points")


def test_nonfinite_rejected(arbx):
    p = np.random.default_rng(2).random((1000, 3)).astype(np.float32)
    p[123, 1] = np.nan
    with pytest.raises(arbx.ArbxError) as e:
        arbx.Tree(cu(p))
    assert e.value.status == arbx.ERR_NONFINITE
    p[123, 1] = np.inf
    with pytest.raises(arbx.ArbxError):
        arbx.Tree(cu(p))
    # the library stays usable
    t = arbx.Tree(cu(np.random.default_rng(3).random((100, 3))))
    assert t.size() == 100


def test_invalid_queries(arbx):
    t = arbx.Tree(cu(np.random.default_rng(3).random((100, 3))))
    q = cu(np.random.default_rng(4).random((10, 3)))
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(arbx.ArbxError):
            t.radius(q, bad)
    with pytest.raises(arbx.ArbxError):
        t.knn(q, 0)
    with pytest.raises(arbx.ArbxError) as e:
        t.knn(q, 257)
    assert e.value.status == arbx.ERR_UNSUPPORTED
    with pytest.raises(arbx.ArbxError) as e:
        t.knn(q, 8, tuning=dict(lanes_per_query=3))
    assert e.value.status == arbx.ERR_INVALID
    with pytest.raises(arbx.ArbxError):
        t.radius(cu(np.zeros((4, 2))), 0.1)  # dimension mismatch


# ------------------------------------------------------------------ tree structure

def node_dtype(dim):
    return np.dtype([("lo0", "<f4", dim), ("hi0", "<f4", dim), ("lo1", "<f4", dim), ("hi1", "<f4", dim),
                     ("child", "<i4", 2), ("orig", "<i4", 2)])


@pytest.mark.parametrize("dim", [2, 3, 6])
def test_tree_structure(arbx, dim):
    """Every leaf is reached exactly once, every internal node except the root
    has one parent, each child box equals the union of its subtree, leaf boxes
    are the points, the root covers the scene, and building twice gives
    identical node bytes."""
    rng = np.random.default_rng(40 + dim)
    n = 5003
    pts = rng.random((n, dim), dtype=np.float32)
    pts[100:140] = pts[7]  # duplicates
    t = arbx.Tree(cu(pts))
    ex = t.export()
    nodes = ex["nodes"].view(node_dtype(dim))
    assert len(nodes) == n - 1
    ch = nodes["child"]
    leaves = np.sort(~ch[ch < 0])
    assert np.array_equal(leaves, np.arange(n))
    internal = np.sort(ch[ch >= 0])
    assert np.array_equal(internal, np.setdiff1d(np.arange(n - 1), [ex["root"]]))
    origs = nodes["orig"][ch < 0]
    assert np.array_equal(np.sort(origs), np.arange(n))
    # leaf boxes are the points
    for c in range(2):
        lc = ch[:, c] < 0
        lo = nodes["lo0" if c == 0 else "lo1"][lc]
        hi = nodes["hi0" if c == 0 else "hi1"][lc]
        assert np.array_equal(lo, pts[nodes["orig"][lc, c]]) and np.array_equal(hi, lo)
    # child box of an internal child = union of that child's two child boxes
    for c in range(2):
        ic = ch[:, c] >= 0
        kid = nodes[ch[ic, c]]
        ulo = np.minimum(kid["lo0"], kid["lo1"])
        uhi = np.maximum(kid["hi0"], kid["hi1"])
        assert np.array_equal(nodes["lo0" if c == 0 else "lo1"][ic], ulo)
        assert np.array_equal(nodes["hi0" if c == 0 else "hi1"][ic], uhi)
    # an internal child's orig slot holds its range end: the largest sorted
    # leaf position below it (the link the stackless traversal follows)
    c1 = ch[:, 1].astype(np.int64)
    end = np.where(c1 < 0, ~c1, -1)
    for _ in range(n):  # end(g) = end(right child of g), resolved bottom-up
        todo = end < 0
        if not todo.any():
            break
        end[todo] = end[c1[todo]]
    assert (end >= 0).all()
    for c in range(2):
        ic = ch[:, c] >= 0
        assert np.array_equal(nodes["orig"][ic, c], end[ch[ic, c]])
    r = nodes[ex["root"]]
    assert np.array_equal(np.minimum(r["lo0"], r["lo1"]), pts.min(0))
    assert np.array_equal(np.maximum(r["hi0"], r["hi1"]), pts.max(0))
    ex2 = arbx.Tree(cu(pts)).export()
    assert np.array_equal(ex["nodes"], ex2["nodes"]) and ex["root"] == ex2["root"]


def test_shared_memory_sizes_in_any_order(arbx):
    """Trees whose staged top levels need different amounts of shared memory
    above the 48 KB default, queried large, smaller, then large again."""
    rng = np.random.default_rng(77)
    for n in (5000, 1000, 900, 5000, 20000):
        pts = rng.random((n, 3), dtype=np.float32)
        qs = rng.random((200, 3), dtype=np.float32)
        t = arbx.Tree(cu(pts))
        for tl in (1023, 255):
            got = t.radius(cu(qs), 0.1, tuning=dict(top_levels=tl))
            assert_crs_equal(got, oracle.radius(pts, qs, 0.1), what=f"n={n} top={tl}")
        arbx.stream_check()


def test_concurrent_streams(arbx, tiny):
    """Queries on two streams at once give the same results as alone
    (section 2.1: concurrent searches on execution spaces)."""
    t = arbx.Tree(cu(tiny["points"]))
    q = cu(tiny["queries"])
    alone = t.count(q, tiny["radius"])
    k_alone = t.knn(q, 8)
    torch.cuda.synchronize()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with torch.cuda.stream(s1):
        c1 = t.count(q, tiny["radius"], stream=s1)
    with torch.cuda.stream(s2):
        k2 = t.knn(q, 8, stream=s2)
    torch.cuda.synchronize()
    assert torch.equal(alone, c1) and torch.equal(k_alone[0], k2[0])
    arbx.stream_check()


def test_autotune_keeps_results(arbx, tiny, tmp_path):
    """The searched launch setting is one of the candidates, is recorded for
    the (tree, predicate) key, and calls that then run under it return the
    oracle's bytes."""
    t = arbx.Tree(cu(tiny["points"]))
    q = cu(tiny["queries"])
    arbx.autotune_clear()
    try:
        best, ms = t.autotune(arbx.SPHERE, q, tiny["radius"], sample=700)
        assert best["block"] in (128, 256) and best["sort_queries"] in (0, 1)
        assert best["top_levels"] in (0, 255, 1023) and best["warp_refill"] in (0, 1) and ms > 0
        kbest, _ = t.autotune(arbx.NEAREST, q, k=tiny["k"])
        assert kbest["block"] in (128, 256)
        assert_crs_equal(t.radius(q, tiny["radius"]), tiny["ref_radius"], what="autotuned radius")
        idx, d2 = t.knn(q, tiny["k"])
        assert np.array_equal(to_np(idx), tiny["ref_knn"][0])
        assert np.array_equal(to_np(d2).view(np.uint32), tiny["ref_knn"][1].view(np.uint32))
        path = tmp_path / "tune.txt"
        arbx.autotune_save(path)
        lines = [ln.split() for ln in path.read_text().splitlines() if not ln.startswith("#")]
        assert len(lines) == 2 and {int(ln[1]) for ln in lines} == {arbx.SPHERE, arbx.NEAREST}
        arbx.autotune_clear()
        arbx.autotune_load(path)
        assert_crs_equal(t.radius(q, tiny["radius"]), tiny["ref_radius"], what="loaded radius")
        # rays on a small terrain
        tris = workloads.heightfield_triangles(65, 33, seed=5)
        rays = workloads.heightfield_rays(3000, seed=6, extent_x=64 * workloads.HF_SPACING,
                                          extent_y=32 * workloads.HF_SPACING)
        tt = arbx.Tree(cu(tris), kind="triangle")
        rbest, _ = tt.autotune(arbx.RAY_NEAREST, cu(rays))
        assert rbest["top_levels"] in (0, 255, 1023)
        hit, tval = tt.ray_nearest(cu(rays))
        rhit, rt = oracle.ray_nearest(tris, rays)
        assert np.array_equal(to_np(hit), rhit)
        assert np.array_equal(to_np(tval).view(np.uint32), rt.view(np.uint32))
    finally:
        arbx.autotune_clear()


# ------------------------------------------------------------------ ray predicates (section 2.5)

def ordered_segments(off, idx, t):
    """Each CRS segment sorted by (t, index), +0 and -0 equal."""
    off, idx, t = to_np(off), to_np(idx), to_np(t)
    oi, ot = idx.copy(), t.copy()
    for i in range(len(off) - 1):
        a, b = off[i], off[i + 1]
        o = np.lexsort((idx[a:b], t[a:b] + np.float32(0)))
        oi[a:b], ot[a:b] = idx[a:b][o], t[a:b][o]
    return off, oi, ot


def ray_scenes():
    rng = np.random.default_rng(31)
    hf = workloads.heightfield_triangles(65, 33, seed=5)
    hf_rays = workloads.heightfield_rays(2500, seed=6, extent_x=64 * workloads.HF_SPACING,
                                         extent_y=32 * workloads.HF_SPACING)
    # grazing rays along the terrain meet several triangles
    o = np.stack([rng.uniform(0, 0.06, 800), rng.uniform(0, 0.03, 800), rng.uniform(0.0, 0.2, 800)], 1)
    d = np.concatenate([rng.normal(0, 1, (800, 2)), rng.normal(-0.05, 0.05, (800, 1))], 1)
    hf_rays = np.concatenate([hf_rays, np.concatenate([o, d], 1).astype(np.float32)])
    lay = workloads.layered_triangles(64)
    lay_rays = np.concatenate([workloads.layered_rays(600, seed=8), workloads.layered_rays(600, seed=9, tilt=0.3),
                               workloads.layered_rays(100, seed=10, z0=0.5)])
    lay_rays[:50, 1] = lay_rays[:50, 0]  # on the diagonal: two triangles per layer
    return [("heightfield", hf, hf_rays), ("layered", lay, lay_rays)]


@pytest.mark.parametrize("quantized", [False, True, "parent"])
def test_ray_intersect_and_ordered(arbx, quantized):
    for name, tris, rays in ray_scenes():
        t = arbx.Tree(cu(tris), kind="triangle", quantized=quantized)
        roff, ridx, rt = oracle.ray_all(tris, rays)
        q = cu(rays)
        # ordered_intersect: the oracle's bytes
        off, idx, tt = t.ray_intersect(q, ordered=True)
        assert np.array_equal(to_np(off), roff), name
        assert np.array_equal(to_np(idx), ridx), name
        assert np.array_equal(to_np(tt).view(np.uint32), rt.view(np.uint32)), name
        # intersect: the same hits per ray, in leaf order
        off2, idx2, t2 = t.ray_intersect(q, ordered=False)
        s_off, s_idx, s_t = ordered_segments(off2, idx2, t2)
        assert np.array_equal(s_off, roff) and np.array_equal(s_idx, ridx), name
        assert np.array_equal(s_t.view(np.uint32), rt.view(np.uint32)), name
        # callbacks count hits; two-phase fill gives the same bytes
        cnt = np.diff(roff)
        assert np.array_equal(to_np(t.callback(arbx.RAY_INTERSECT, q, arbx.CB_COUNT)), cnt)
        assert np.array_equal(to_np(t.callback(arbx.RAY_INTERSECT, q, arbx.CB_COUNT_UP_TO, limit=2)),
                              np.minimum(cnt, 2))
        assert np.array_equal(to_np(t.callback(arbx.RAY_ORDERED, q, arbx.CB_FIRST_HIT)), (cnt > 0).astype(np.int32))
        o3, i3, t3 = t.offsets_fill(arbx.RAY_ORDERED, q)
        assert torch.equal(o3, off) and torch.equal(i3, idx) and torch.equal(t3, tt)
        o4, i4, _ = t.offsets_fill(arbx.RAY_INTERSECT, q, want_d2=False)
        assert torch.equal(o4, off2) and torch.equal(i4, idx2)
        o5, i5, t5 = t.ray_intersect(q, ordered=True, tuning=dict(single_pass=1, sort_queries=0))
        assert torch.equal(o5, off) and torch.equal(i5, idx) and torch.equal(t5, tt)
        assert (cnt > 1).any(), name
    arbx.stream_check()


@pytest.mark.parametrize("quantized", [False, True, "parent"])
def test_ray_nearest_k(arbx, quantized):
    """nearest(ray, k): the first k hits of the oracle's ordered list, padded
    with -1 / +inf; the CRS form holds the hits found."""
    for name, tris, rays in ray_scenes():
        t = arbx.Tree(cu(tris), kind="triangle", quantized=quantized)
        roff, ridx, rt = oracle.ray_all(tris, rays)
        q = cu(rays)
        for k in (1, 2, 3, 8, 32):
            hit, tt = t.ray_nearest(q, k=k)
            hit, tt = to_np(hit).reshape(len(rays), -1), to_np(tt).reshape(len(rays), -1)
            assert hit.shape[1] == k
            for i in range(len(rays)):
                c = min(k, roff[i + 1] - roff[i])
                assert np.array_equal(hit[i, :c], ridx[roff[i]:roff[i] + c]), (name, k, i)
                assert np.array_equal(tt[i, :c].view(np.uint32), rt[roff[i]:roff[i] + c].view(np.uint32))
                assert (hit[i, c:] == -1).all() and np.isinf(tt[i, c:]).all()
            crs = t.query_crs(arbx.RAY_NEAREST, q, k=k)
            cnt = np.minimum(np.diff(roff), k)
            assert np.array_equal(np.diff(to_np(crs.offsets)), cnt)
            sel = np.concatenate([np.arange(roff[i], roff[i] + cnt[i]) for i in range(len(rays))])
            assert np.array_equal(to_np(crs.indices), ridx[sel])
    arbx.stream_check()


def test_crs_buffers_freed_without_garbage_collection(arbx, tiny):
    """A library CRS goes back to the device pool as soon as the result and
    its tensor views are dropped (no reference cycle waits for the collector)."""
    import gc
    from cuda.bindings import runtime as rt
    _, pool = rt.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())

    def used():
        torch.cuda.synchronize()
        _, v = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)
        return int(v)

    t = arbx.Tree(cu(tiny["points"]))
    q = cu(tiny["queries"])
    gc.disable()
    try:
        base = None
        for i in range(6):
            off, idx, d2 = t.radius(q, tiny["radius"] * 4)
            assert idx.numel() > 100000
            del off, idx, d2
            u = used()
            base = u if base is None else base
            assert u <= base, (i, u, base)
    finally:
        gc.enable()
