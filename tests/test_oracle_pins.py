"""Pins of the CPU oracle against things other than itself.

Each test ties the oracle to a value fixed by the paper's definitions and by
mathematics: hand-worked cases (tests/golden/hand_cases.json), exact rational
arithmetic with explicit binary32 rounding, library routines (scipy's k-d tree,
numpy's float64 linear solver), a closed-form expected count, and invariants
(symmetry, kNN-radius consistency, callback saturation).  A dropped term, a
wrong sign or index, a transposed operand, a contracted multiply-add or a
changed summation order each fails at least one of them.
"""
from __future__ import annotations

import json
import math
from fractions import Fraction
from pathlib import Path

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
import workloads

GOLDEN = json.loads((Path(__file__).parent / "golden" / "hand_cases.json").read_text())


def _arr(x, cols):
    a = np.asarray(x, dtype=np.float32)
    return a.reshape(-1, cols)


# ------------------------------------------------------------ hand-worked cases

@pytest.mark.parametrize("case", GOLDEN["radius"], ids=lambda c: c["name"])
def test_hand_radius(case):
    dim = len(case["queries"][0])
    off, idx, d2 = oracle.radius(_arr(case["points"], dim), _arr(case["queries"], dim), case["radius"])
    for i, (ei, ed) in enumerate(zip(case["indices"], case["d2"])):
        assert idx[off[i]:off[i + 1]].tolist() == ei
        assert d2[off[i]:off[i + 1]].tolist() == ed
    cnt = oracle.radius_count(_arr(case["points"], dim), _arr(case["queries"], dim), case["radius"])
    assert cnt.tolist() == [len(e) for e in case["indices"]]


@pytest.mark.parametrize("case", GOLDEN["knn"], ids=lambda c: c["name"])
def test_hand_knn(case):
    dim = len(case["queries"][0])
    idx, d2 = oracle.knn(_arr(case["points"], dim), _arr(case["queries"], dim), case["k"])
    assert idx.tolist() == case["indices"]
    assert d2.tolist() == case["d2"]


@pytest.mark.parametrize("case", GOLDEN["rays"]["cases"], ids=lambda c: c["name"])
def test_hand_rays(case):
    tris = np.asarray(GOLDEN["rays"]["triangles"], np.float32)
    hit, t = oracle.ray_nearest(tris, np.asarray([case["ray"]], np.float32))
    assert hit[0] == case["hit"]
    exp_t = math.inf if case["t"] == "inf" else case["t"]
    assert float(t[0]) == exp_t


@pytest.mark.parametrize("case", GOLDEN["boxes"], ids=lambda c: c["name"])
def test_hand_boxes(case):
    if case["kind"] == "triangle":
        prims, kind = np.asarray(case["prims"], np.float32), oracle.TRIANGLE
    else:
        prims, kind = np.asarray(case["prims"], np.float32), oracle.POINT
    off, idx = oracle.box_query(prims, kind, np.asarray(case["boxes"], np.float32))
    for i, e in enumerate(case["indices"]):
        assert idx[off[i]:off[i + 1]].tolist() == e


def test_identical_points():
    """1000 copies of one point: radius 0 finds all of them at d2 = 0; kNN k=8
    returns indices 0..7 (ties go to the lower index)."""
    p = np.tile(np.float32([0.3, 0.7, 0.1]), (1000, 1))
    off, idx, d2 = oracle.radius(p, p[:1], 0.0)
    assert idx.tolist() == list(range(1000)) and not d2.any()
    ki, kd = oracle.knn(p, p[:1], 8)
    assert ki.tolist() == [list(range(8))] and not kd.any()


def test_empty_index_knn():
    idx, d2 = oracle.knn(np.zeros((0, 3), np.float32), np.zeros((5, 3), np.float32), 4)
    assert idx.shape == (5, 0)


# ------------------------------------------------- exact binary32 arithmetic

def rn32(x: Fraction) -> Fraction:
    """Round an exact rational to the nearest binary32 value, ties to even
    (normal range only)."""
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    while Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    ulp = Fraction(2) ** (e - 23)
    q, r = divmod(a, ulp)
    if 2 * r > ulp or (2 * r == ulp and q % 2 == 1):
        q += 1
    return s * q * ulp


def exact_d2_sequential(q, p):
    """d2 by the contract: dx = rn(q - p), then rn(acc + rn(dx*dx)), left to right."""
    acc = None
    for qa, pa in zip(q, p):
        dx = rn32(Fraction(float(qa)) - Fraction(float(pa)))
        sq = rn32(dx * dx)
        acc = sq if acc is None else rn32(acc + sq)
    return acc


def test_d2_rounding_contract():
    """The oracle's d2 equals the exactly-rounded step sequence on random inputs."""
    r = np.random.default_rng(7)
    for _ in range(300):
        dim = int(r.choice([2, 3, 6]))
        q = r.random(dim, dtype=np.float32)
        p = r.random(dim, dtype=np.float32)
        assert Fraction(float(oracle.sq_dist(q, p))) == exact_d2_sequential(q, p)


def test_d2_left_to_right_order():
    """(1, 2^-12, 2^-12): summed left to right the tiny squares are absorbed one
    at a time (ties to even), d2 = 1; in the reverse order d2 = 1 + 2^-23."""
    a = np.float32(2.0 ** -12)
    zero = np.zeros(3, np.float32)
    assert float(oracle.sq_dist(np.float32([1.0, a, a]), zero)) == 1.0
    assert float(oracle.sq_dist(np.float32([a, a, 1.0]), zero)) == 1.0 + 2.0 ** -23


def test_d2_no_fused_multiply_add():
    """Find inputs where a fused multiply-add of the second square would round
    differently; the oracle must give the separately rounded value."""
    r = np.random.default_rng(11)
    found = 0
    for _ in range(20000):
        q = (1.0 + r.random(2, dtype=np.float32)).astype(np.float32)
        a, b = Fraction(float(q[0])), Fraction(float(q[1]))
        sep = rn32(rn32(a * a) + rn32(b * b))
        fused = rn32(rn32(a * a) + b * b)
        if sep != fused:
            assert Fraction(float(oracle.sq_dist(q, np.zeros(2, np.float32)))) == sep
            found += 1
            if found >= 5:
                break
    assert found >= 5


def test_d2_error_bound_vs_float64():
    """Relative error of the float32 d2 against float64 is within gamma_6."""
    r = np.random.default_rng(3)
    q = r.random((2000, 3), dtype=np.float32)
    p = r.random((2000, 3), dtype=np.float32)
    d64 = ((q.astype(np.float64) - p.astype(np.float64)) ** 2).sum(1)
    d32 = np.array([oracle.sq_dist(q[i], p[i]) for i in range(len(q))], np.float64)
    u = 2.0 ** -24
    gamma6 = 6 * u / (1 - 6 * u)
    assert np.all(np.abs(d32 - d64) <= gamma6 * d64 + 1e-38)


# ------------------------------------------------------------ library routines

@pytest.mark.parametrize("dim,n,m,r", [(2, 4000, 300, 0.03), (3, 4000, 300, 0.08), (6, 3000, 200, 0.35)])
def test_radius_vs_kdtree(dim, n, m, r):
    """Neighbour sets equal scipy's float64 k-d tree ball query, except for pairs
    within a relative 1e-5 of the boundary, where float32 rounding may decide."""
    rng = np.random.default_rng(dim)
    pts = rng.random((n, dim), dtype=np.float32)
    qs = rng.random((m, dim), dtype=np.float32)
    off, idx, d2 = oracle.radius(pts, qs, r)
    tree = cKDTree(pts.astype(np.float64))
    balls = tree.query_ball_point(qs.astype(np.float64), r)
    d64 = np.sqrt(((qs[:, None, :].astype(np.float64) - pts[None].astype(np.float64)) ** 2).sum(-1))
    for i in range(m):
        mine = set(idx[off[i]:off[i + 1]].tolist())
        ref = set(balls[i])
        for j in mine ^ ref:
            assert abs(d64[i, j] - r) < 1e-5 * r, (i, j)
        assert list(idx[off[i]:off[i + 1]]) == sorted(mine)


@pytest.mark.parametrize("dim,k", [(2, 8), (3, 16), (6, 8)])
def test_knn_vs_kdtree(dim, k):
    """kNN lists equal scipy's float64 k-d tree, on queries whose k+1 nearest
    float64 distances are separated by more than a relative 1e-5."""
    rng = np.random.default_rng(100 + dim)
    pts = rng.random((3000, dim), dtype=np.float32)
    qs = rng.random((300, dim), dtype=np.float32)
    idx, d2 = oracle.knn(pts, qs, k)
    dd, ii = cKDTree(pts.astype(np.float64)).query(qs.astype(np.float64), k + 1)
    checked = 0
    for i in range(len(qs)):
        if np.all(np.diff(dd[i]) > 1e-5 * dd[i, 1:]):
            assert idx[i].tolist() == ii[i, :k].tolist()
            checked += 1
    assert checked > 250
    assert np.allclose(np.sqrt(d2.astype(np.float64)), dd[:, :k], rtol=1e-6)


def test_tiny_uniform_mean_count_closed_form():
    """For a ball of radius r centred uniformly in the unit cube, the expected
    volume inside the cube is (4/3)pi r^3 - (3/2)pi r^4 + (8/5) r^5 - r^6/6
    (integral of prod(1-|z_a|) over the ball).  With 16384 uniform points the
    mean count of the tiny workload must match 16384 times that."""
    wl = workloads.tiny_uniform()
    c = oracle.radius_count(wl["points"], wl["queries"], wl["radius"])
    r = wl["radius"]
    ev = 4 / 3 * math.pi * r ** 3 - 1.5 * math.pi * r ** 4 + 1.6 * r ** 5 - r ** 6 / 6
    assert abs(c.mean() - 16384 * ev) < 0.25


def test_ray_vs_linear_solve():
    """Moller-Trumbore hit/miss and t equal a float64 solve of
    o + t d = v0 + u e1 + v e2 wherever the decision is clear by 1e-4."""
    rng = np.random.default_rng(5)
    n = 400
    v0 = rng.random((n, 3)).astype(np.float32)
    tris = np.stack([v0, v0 + rng.normal(0, 0.3, (n, 3)).astype(np.float32),
                     v0 + rng.normal(0, 0.3, (n, 3)).astype(np.float32)], 1).astype(np.float32)
    rays = np.concatenate([rng.random((300, 3)), rng.normal(0, 1, (300, 3))], 1).astype(np.float32)
    clear_hits = 0
    for ry in rays[:60]:
        o, d = ry[:3].astype(np.float64), ry[3:].astype(np.float64)
        for tri in tris:
            a, b, c = tri.astype(np.float64)
            A = np.stack([-d, b - a, c - a], 1)
            if abs(np.linalg.det(A)) < 1e-6:
                continue
            t, u, v = np.linalg.solve(A, o - a)
            hit, tt = oracle.moller_trumbore(ry, tri)
            eps = 1e-4
            if u > eps and v > eps and u + v < 1 - eps and t > eps:
                assert hit and abs(float(tt) - t) <= 1e-4 * max(1.0, abs(t))
                clear_hits += 1
            elif u < -eps or v < -eps or u + v > 1 + eps or t < -eps:
                assert not hit
    assert clear_hits > 100


def test_ray_nearest_is_first_of_all_hits():
    rng = np.random.default_rng(9)
    tris = workloads.heightfield_triangles(40, 20, seed=77)
    o = np.stack([rng.uniform(0, 39 / 1023, 500), rng.uniform(0, 19 / 1023, 500), np.full(500, 0.25)], 1)
    d = np.concatenate([rng.normal(0, 0.01, (500, 2)), -np.ones((500, 1))], 1)
    rays = np.concatenate([o, d], 1).astype(np.float32)
    hit, t = oracle.ray_nearest(tris, rays)
    off, idx, tt = oracle.ray_all(tris, rays)
    for i in range(len(rays)):
        if off[i + 1] > off[i]:
            assert hit[i] == idx[off[i]] and t[i] == tt[off[i]]
            seg = list(zip(tt[off[i]:off[i + 1]].tolist(), idx[off[i]:off[i + 1]].tolist()))
            assert seg == sorted(seg)
        else:
            assert hit[i] == -1 and math.isinf(t[i])
    assert (hit >= 0).mean() > 0.8   # near-vertical rays from above the surface


def test_ray_all_layered_closed_form():
    """Vertical rays through 64 stacked unit squares (two triangles each) and
    a duplicated layer: a ray at (x, y) off the diagonal meets exactly one
    triangle per layer, at t = z0 - z, top layer first; the duplicate ties
    with its original at the same t and follows it (higher index).  A ray
    whose origin lies on a layer meets it at t = 0.  On the diagonal a ray
    meets both triangles of each layer (closed barycentric bounds)."""
    L = 64
    tris = workloads.layered_triangles(L, duplicate_layer=7)
    rays = workloads.layered_rays(300, seed=3)
    rays[0, :2] = [0.25, 0.25]          # on the diagonal
    rays[1, 2] = 0.5                    # origin on layer 32
    off, idx, t = oracle.ray_all(tris, rays)
    for i, ry in enumerate(rays):
        x, y, z0 = (float(v) for v in ry[:3])
        seg_i = idx[off[i]:off[i + 1]].tolist()
        seg_t = t[off[i]:off[i + 1]].tolist()
        layers = [l for l in range(L - 1, -1, -1) if l / L <= z0]
        if i == 0:
            want = [2 * l + b for l in layers for b in (0, 1)]
            want[want.index(15) + 1:want.index(15) + 1] = [2 * L, 2 * L + 1]
        else:
            b = 1 if y > x else 0
            want = [2 * l + b for l in layers]
            want.insert(want.index(2 * 7 + b) + 1, 2 * L + b)
        assert seg_i == want, i
        zs = [float(tris[j][0][2]) for j in seg_i]
        assert all(abs(tt - (z0 - z)) <= 1e-6 for tt, z in zip(seg_t, zs))
        assert seg_t == sorted(seg_t)
    assert t[off[1] + 0] == 0.0 and idx[off[1]] in (64, 65)
    hit, tn = oracle.ray_nearest(tris, rays)
    assert np.array_equal(hit, idx[off[:-1]])


# ------------------------------------------------------------------ invariants

def test_radius_symmetry():
    """Queries = points: j in R(i) iff i in R(j), with bit-identical d2, since
    fl(a - b) = -fl(b - a)."""
    rng = np.random.default_rng(21)
    p = rng.random((1500, 3), dtype=np.float32)
    off, idx, d2 = oracle.radius(p, p, 0.07)
    pairs = {}
    for i in range(len(p)):
        for j, e in zip(idx[off[i]:off[i + 1]], d2[off[i]:off[i + 1]]):
            pairs[(i, int(j))] = e.view(np.uint32)
    for (i, j), bits in pairs.items():
        assert pairs[(j, i)] == bits
    assert all(pairs[(i, i)] == 0 for i in range(len(p)))


def test_knn_equals_sorted_radius_prefix():
    """Whenever a query has at least k neighbours within r, its kNN list is the
    k smallest (d2, index) pairs of its radius list; otherwise the radius list
    is a prefix of the kNN list and the rest lies outside r."""
    rng = np.random.default_rng(31)
    pts = rng.random((5000, 3), dtype=np.float32)
    qs = rng.random((400, 3), dtype=np.float32)
    r, k = 0.06, 8
    off, idx, d2 = oracle.radius(pts, qs, r)
    ki, kd = oracle.knn(pts, qs, k)
    r2 = np.float32(r) * np.float32(r)
    for i in range(len(qs)):
        seg = sorted(zip(d2[off[i]:off[i + 1]].tolist(), idx[off[i]:off[i + 1]].tolist()))
        mine = list(zip(kd[i].tolist(), ki[i].tolist()))
        if len(seg) >= k:
            assert mine == seg[:k]
        else:
            assert mine[:len(seg)] == seg
            assert all(e > r2 for e, _ in mine[len(seg):])
        assert mine == sorted(mine) and len(set(ki[i].tolist())) == k


def test_counts_and_callbacks():
    """offsets deltas = count; count-up-to(n) = min(count, n); first hit =
    count-up-to(1) = [count >= 1]."""
    rng = np.random.default_rng(41)
    pts = rng.random((3000, 3), dtype=np.float32)
    qs = rng.random((500, 3), dtype=np.float32)
    off, idx, d2 = oracle.radius(pts, qs, 0.05)
    cnt = oracle.radius_count(pts, qs, 0.05)
    assert np.array_equal(np.diff(off), cnt)
    for lim in (0, 1, 3, 10, 1000):
        assert np.array_equal(oracle.radius_count_up_to(pts, qs, 0.05, lim), np.minimum(cnt, lim))
    assert np.array_equal(oracle.radius_count_up_to(pts, qs, 0.05, 1), (cnt >= 1).astype(np.int32))


def test_per_query_radii():
    rng = np.random.default_rng(51)
    pts = rng.random((2000, 3), dtype=np.float32)
    qs = rng.random((100, 3), dtype=np.float32)
    radii = rng.uniform(0.0, 0.1, 100).astype(np.float32)
    off, idx, d2 = oracle.radius(pts, qs, radii)
    for i in range(0, 100, 7):
        o1, i1, e1 = oracle.radius(pts, qs[i:i + 1], float(radii[i]))
        assert idx[off[i]:off[i + 1]].tolist() == i1.tolist()


def test_box_degenerate_and_universal():
    """A box collapsed onto point j finds exactly the points equal to it; an
    all-covering box finds everything; growing a box never loses a hit; the
    overlap test equals the interval-intersection form max(lo) <= min(hi)."""
    rng = np.random.default_rng(61)
    pts = np.round(rng.random((800, 3)) * 16).astype(np.float32) / 16
    boxes = np.concatenate([pts[:50], pts[:50]], 1)
    off, idx = oracle.box_query(pts, oracle.POINT, boxes)
    for i in range(50):
        exp = np.nonzero(np.all(pts == pts[i], 1))[0].tolist()
        assert idx[off[i]:off[i + 1]].tolist() == exp
    big = np.float32([[-1, -1, -1, 2, 2, 2]])
    off, idx = oracle.box_query(pts, oracle.POINT, big)
    assert idx.tolist() == list(range(800))
    tris = workloads.heightfield_triangles(30, 20, seed=5)
    c = rng.random((200, 3)).astype(np.float32) * np.float32([29 / 1023, 19 / 1023, 0.2])
    h = np.float32(0.01)
    small = np.concatenate([c - h, c + h], 1)
    large = np.concatenate([c - 2 * h, c + 2 * h], 1)
    o1, i1 = oracle.box_query(tris, oracle.TRIANGLE, small)
    o2, i2 = oracle.box_query(tris, oracle.TRIANGLE, large)
    tlo, thi = tris.min(1), tris.max(1)
    for i in range(200):
        s1, s2 = set(i1[o1[i]:o1[i + 1]].tolist()), set(i2[o2[i]:o2[i + 1]].tolist())
        assert s1 <= s2
        exp = np.nonzero(np.all(np.maximum(small[i, :3], tlo) <= np.minimum(small[i, 3:], thi), 1))[0]
        assert sorted(s1) == exp.tolist()


# ------------------------------------------------------------------ DBSCAN (section 2.4)

def test_dbscan_hand_case():
    """Points on a line, eps = 1, minPts = 3 (self included): 0,1,2 form a
    cluster labelled 1 (1 is core with 3 neighbours; 0 and 2 have 2 and are
    border); 5 is noise; 10..13 are a cluster labelled 5, the index of 11
    (11 and 12 are core, 10 and 13 border); 14.5 is noise (its only point
    within eps is itself)."""
    x = np.float32([0, 1, 2, 5, 10, 11, 12, 13, 14.5])
    pts = np.stack([x, np.zeros_like(x)], 1)
    labels, nc = oracle.dbscan(pts, 1.0, 3)
    assert labels.tolist() == [1, 1, 1, -1, 5, 5, 5, 5, -1] and nc == 2


def test_dbscan_vs_sklearn():
    """The same core points, the same partition of core points and the same
    noise as scikit-learn's DBSCAN (eps inclusive, min_samples counting the
    point itself) on clustered data with no pair distance near eps; each
    border point lies in a cluster of one of its core neighbours."""
    from sklearn.cluster import DBSCAN
    rng = np.random.default_rng(21)
    centres = rng.random((12, 3))
    pts = (centres[rng.integers(0, 12, 3000)] + 0.03 * rng.standard_normal((3000, 3))).astype(np.float32)
    pts = np.concatenate([pts, rng.random((300, 3)).astype(np.float32)])
    eps, min_pts = 0.05, 6
    d = np.sqrt(((pts[:, None, :].astype(np.float64) - pts[None, :, :]) ** 2).sum(-1))
    near = np.abs(d - eps) < 1e-5             # drop points with a decision near the boundary
    keep = ~near.any(1)
    pts, d = pts[keep], d[keep][:, keep]
    assert len(pts) > 3000
    labels, nc = oracle.dbscan(pts, eps, min_pts)
    sk = DBSCAN(eps=eps, min_samples=min_pts).fit(pts.astype(np.float64))
    core = np.zeros(len(pts), bool)
    core[sk.core_sample_indices_] = True
    nb = d <= eps
    assert np.array_equal(core, nb.sum(1) >= min_pts)
    assert np.array_equal(labels == -1, sk.labels_ == -1)
    # partition of core points: a bijection between label sets
    pairs = set(zip(labels[core].tolist(), sk.labels_[core].tolist()))
    assert len(pairs) == len(set(labels[core].tolist())) == len(set(sk.labels_[core].tolist())) == nc
    # labels are the smallest core index of each cluster
    for lab in set(labels[core].tolist()):
        assert lab == np.flatnonzero(core & (labels == lab)).min()
    # border points: the smallest label among their core neighbours
    for i in np.flatnonzero(~core & (labels >= 0)):
        assert labels[i] == labels[nb[i] & core].min()
    assert nc > 5 and (labels == -1).sum() > 50 and (~core & (labels >= 0)).sum() > 20


def test_dbscan_degenerate():
    """minPts = 1: every point is core, clusters are the eps-graph's
    components; eps = 0 clusters exact duplicates only."""
    rng = np.random.default_rng(4)
    pts = rng.random((500, 2)).astype(np.float32)
    pts[100:110] = pts[3]
    labels, nc = oracle.dbscan(pts, 0.0, 2)
    assert (labels[[3, *range(100, 110)]] == 3).all() and nc == 1
    assert (np.delete(labels, [3, *range(100, 110)]) == -1).all()
    labels1, nc1 = oracle.dbscan(pts, 0.0, 1)
    assert nc1 == 500 - 10 and (labels1 >= 0).all()
