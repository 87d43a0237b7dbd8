"""Full-size GPU parity, in the launch configuration bench.py times.

* Large mixture (N = M = 10M): radius CRS with d2 and kNN k=16 compared bit for bit
  with the oracle on the seeded 10k-query subset; over all 10M queries, the count
  callback equals the CRS offset deltas, every kNN row is strictly increasing in
  (d2, index), and kNN agrees with the radius result: its first min(count, 16)
  pairs are the smallest pairs of the radius list and any further pair lies
  outside the radius.
* Heightfield (4,188,162 triangles, 4M rays, 4M boxes), float32 and 16-bit nodes:
  both node formats give identical results on all queries; 10k-ray and 10k-box
  subsets equal the oracle; rays aimed at triangle vertices and edge midpoints
  (where culling is closest to wrong) equal the oracle; every decoded 16-bit child
  box contains its exact child box.
* Heightfield rays, intersect and ordered_intersect: ordered_intersect equals the
  oracle on the 10k-ray subset; intersect holds the same hits per ray on all 4M
  rays; nearest(ray, k) rows are the first k entries of the ordered lists.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arbx():
    import paper_2507_23700_b300 as m
    return m


def segments(off: torch.Tensor, sel: torch.Tensor):
    """Positions of the CRS entries of the selected queries, and their lengths."""
    start = off[sel]
    lens = off[sel + 1] - start
    base = torch.repeat_interleave(start, lens)
    first = torch.repeat_interleave(torch.cumsum(lens, 0) - lens, lens)
    pos = base + (torch.arange(int(lens.sum()), device=off.device) - first)
    return pos, lens


@pytest.fixture(scope="module")
def large():
    wl = workloads.large_mixture()
    wl["sub"] = workloads.subset_indices(len(wl["queries"]), 10_000)
    return wl


def test_large_mixture_subset_vs_oracle(arbx, large):
    pts = torch.from_numpy(large["points"]).cuda()
    qs = torch.from_numpy(large["queries"]).cuda()
    r, k, sub = large["radius"], large["k"], large["sub"]
    tree = arbx.Tree(pts)
    off, idx, d2 = tree.radius(qs, r)
    subt = torch.from_numpy(sub).cuda()
    pos, lens = segments(off, subt)
    g_off = np.zeros(len(sub) + 1, np.int64)
    np.cumsum(lens.cpu().numpy(), out=g_off[1:])
    g_idx = idx[pos].cpu().numpy()
    g_d2 = d2[pos].cpu().numpy()
    r_off, r_idx, r_d2 = oracle.radius(large["points"], large["queries"][sub], r)
    from crs_util import assert_crs_equal
    assert_crs_equal((g_off, g_idx, g_d2), (r_off, r_idx, r_d2), what="10M radius subset")
    kidx, kd2 = tree.knn(qs, k)
    ridx, rd2 = oracle.knn(large["points"], large["queries"][sub], k)
    assert np.array_equal(kidx[subt].cpu().numpy(), ridx)
    assert np.array_equal(kd2[subt].cpu().numpy().view(np.uint32), rd2.view(np.uint32))


def test_large_mixture_shared_order_lanes_and_k64(arbx, large):
    """In the bench's launch form: one query order shared by the radius and kNN
    calls gives the same bytes as each call sorting for itself; kNN k=16 under
    every lane-group size equals the one-lane rows on all 10M queries; k=64 (a
    lane group of 8 per query) equals the oracle on the 10k subset."""
    pts = torch.from_numpy(large["points"]).cuda()
    qs = torch.from_numpy(large["queries"]).cuda()
    r, k, sub = large["radius"], large["k"], large["sub"]
    tree = arbx.Tree(pts, wide=True)
    order = tree.query_order(arbx.SPHERE, qs, r)
    base = tree.radius(qs, r)
    got = tree.radius(qs, r, order=order)
    assert all(torch.equal(a, b) for a, b in zip(base, got))
    del base, got
    k1 = tree.knn(qs, k, tuning=dict(lanes_per_query=1))
    for tu in (dict(lanes_per_query=2), dict(lanes_per_query=4), dict(lanes_per_query=8), dict(wide_nodes=1),
               dict(warp_packets=1), dict(query_runs=1), dict(query_runs=8)):
        kg = tree.knn(qs, k, tuning=tu, order=order)
        assert torch.equal(k1[0], kg[0]) and torch.equal(k1[1], kg[1]), tu
    del k1, kg
    cnt = tree.count(qs, r)
    assert torch.equal(cnt, tree.count(qs, r, tuning=dict(wide_nodes=1)))
    del cnt
    subt = torch.from_numpy(sub).cuda()
    kidx, kd2 = tree.knn(qs, 64, order=order)
    ridx, rd2 = oracle.knn(large["points"], large["queries"][sub], 64)
    assert np.array_equal(kidx[subt].cpu().numpy(), ridx)
    assert np.array_equal(kd2[subt].cpu().numpy().view(np.uint32), rd2.view(np.uint32))
    arbx.stream_check()


def test_large_mixture_to_host_in_chunks(arbx, large):
    """The 10M radius query (351M matches) filled into host memory in ranges
    of at most 256 MB of results equals the device CRS byte for byte."""
    pts = torch.from_numpy(large["points"]).cuda()
    qs = torch.from_numpy(large["queries"]).cuda()
    tree = arbx.Tree(pts)
    off, idx, d2 = tree.radius(qs, large["radius"])
    h_off, h_idx, h_d2 = tree.query_crs_host(arbx.SPHERE, qs, large["radius"], chunk_bytes=256 << 20)
    assert np.array_equal(off.cpu().numpy(), h_off)
    assert np.array_equal(idx.cpu().numpy(), h_idx)
    assert np.array_equal(d2.cpu().numpy().view(np.uint32), h_d2.view(np.uint32))


def test_large_mixture_full_invariants(arbx, large):
    pts = torch.from_numpy(large["points"]).cuda()
    qs = torch.from_numpy(large["queries"]).cuda()
    r, k = large["radius"], large["k"]
    m = qs.shape[0]
    tree = arbx.Tree(pts)
    off, idx, d2 = tree.radius(qs, r)
    cnt = off[1:] - off[:-1]
    assert int(off[0]) == 0 and bool((cnt >= 0).all())
    assert torch.equal(tree.count(qs, r).to(torch.int64), cnt)
    assert torch.equal(tree.count_up_to(qs, r, 5).to(torch.int64), torch.clamp(cnt, max=5))
    kidx, kd2 = tree.knn(qs, k)
    # rows strictly increasing in (d2, index)
    a, b = kd2[:, :-1], kd2[:, 1:]
    ia, ib = kidx[:, :-1], kidx[:, 1:]
    assert bool(((b > a) | ((b == a) & (ib > ia))).all())
    # radius list sorted by (d2, index) within each query
    seg = torch.repeat_interleave(torch.arange(m, device="cuda", dtype=torch.int64), cnt)
    o1 = torch.sort(idx.to(torch.int64), stable=True).indices
    key = (seg[o1] << 32) | d2[o1].view(torch.int32).to(torch.int64)
    o2 = torch.sort(key, stable=True).indices
    order = o1[o2]
    s_idx, s_d2 = idx[order], d2[order]
    r2 = torch.tensor(np.float32(r) * np.float32(r), device="cuda")
    for j in range(k):
        has = cnt > j
        p = off[:-1][has] + j
        assert torch.equal(s_idx[p], kidx[has, j]), j
        assert torch.equal(s_d2[p].view(torch.int32), kd2[has, j].view(torch.int32)), j
        assert bool((kd2[~has, j] > r2).all()), j
    arbx.stream_check()


# ------------------------------------------------------------------ heightfield

@pytest.fixture(scope="module")
def hf():
    tris = workloads.heightfield_triangles()
    rays = workloads.heightfield_rays(4_000_000)
    boxes = workloads.heightfield_boxes(4_000_000)
    return dict(tris=tris, rays=rays, boxes=boxes, sub=workloads.subset_indices(4_000_000, 10_000))


def test_heightfield_rays_and_boxes(arbx, hf):
    tris = torch.from_numpy(hf["tris"].reshape(-1, 9)).cuda()
    rays = torch.from_numpy(hf["rays"]).cuda()
    boxes = torch.from_numpy(hf["boxes"]).cuda()
    sub = hf["sub"]
    subt = torch.from_numpy(sub).cuda()
    t32 = arbx.Tree(tris.view(-1, 3, 3), kind="triangle")
    t16 = arbx.Tree(tris.view(-1, 3, 3), kind="triangle", quantized=True)
    tp = arbx.Tree(tris.view(-1, 3, 3), kind="triangle", quantized="parent")
    assert t32.layout()["node_stride"] == 64 and t16.layout()["node_stride"] == 48
    assert tp.layout()["node_stride"] == 32
    h32, tt32 = t32.ray_nearest(rays)
    for tq in (t16, tp):
        h16, tt16 = tq.ray_nearest(rays)
        assert torch.equal(h32, h16) and torch.equal(tt32.view(torch.int32), tt16.view(torch.int32))
    rh, rt = oracle.ray_nearest(hf["tris"], hf["rays"][sub])
    assert np.array_equal(h32[subt].cpu().numpy(), rh)
    assert np.array_equal(tt32[subt].cpu().numpy().view(np.uint32), rt.view(np.uint32))
    o32, i32 = t32.box(boxes)
    for tq in (t16, tp):
        o16, i16 = tq.box(boxes)
        assert torch.equal(o32, o16) and torch.equal(i32, i16)
    pos, lens = segments(o32, subt)
    g_off = np.zeros(len(sub) + 1, np.int64)
    np.cumsum(lens.cpu().numpy(), out=g_off[1:])
    r_off, r_idx = oracle.box_query(hf["tris"], oracle.TRIANGLE, hf["boxes"][sub])
    from crs_util import assert_crs_equal
    assert_crs_equal((g_off, i32[pos].cpu().numpy(), None), (r_off, r_idx, None), check_d2=False,
                     what="heightfield boxes")
    arbx.stream_check()


def test_heightfield_ray_intersect_and_k_nearest(arbx, hf):
    """Full-size terrain, both node formats: ordered_intersect equals the
    oracle on the 10k-ray subset (indices and t bits); intersect holds the
    same hits per ray as ordered_intersect on all 4M rays; nearest(ray, 4)
    rows are the first hits of the ordered lists, and nearest(ray, 1) their
    first entries."""
    tris = torch.from_numpy(hf["tris"].reshape(-1, 9)).cuda().view(-1, 3, 3)
    rays = torch.from_numpy(hf["rays"]).cuda()
    sub = hf["sub"]
    subt = torch.from_numpy(sub).cuda()
    r_off, r_idx, r_t = oracle.ray_all(hf["tris"], hf["rays"][sub])
    from crs_util import assert_crs_equal
    for q in (False, True, "parent"):
        t = arbx.Tree(tris, kind="triangle", quantized=q)
        off, idx, tt = t.ray_intersect(rays, ordered=True)
        pos, lens = segments(off, subt)
        g_off = np.zeros(len(sub) + 1, np.int64)
        np.cumsum(lens.cpu().numpy(), out=g_off[1:])
        assert np.array_equal(g_off, r_off), q
        assert np.array_equal(idx[pos].cpu().numpy(), r_idx), q
        assert np.array_equal(tt[pos].cpu().numpy().view(np.uint32), r_t.view(np.uint32)), q
        off2, idx2, t2 = t.ray_intersect(rays, ordered=False)
        assert torch.equal(off2, off)
        # same multiset per segment: sort both by (segment, index)
        seg = torch.repeat_interleave(torch.arange(len(off) - 1, device=off.device), off[1:] - off[:-1])
        k1 = seg.to(torch.int64) * (1 << 31) + idx.to(torch.int64)
        k2 = seg.to(torch.int64) * (1 << 31) + idx2.to(torch.int64)
        assert torch.equal(torch.sort(k1).values, torch.sort(k2).values)
        h4, t4 = t.ray_nearest(rays, k=4)
        cnt = (off[1:] - off[:-1]).clamp(max=4)
        assert torch.equal((h4 >= 0).sum(1).to(cnt.dtype), cnt)
        rows = torch.arange(4, device=off.device)[None, :] < cnt[:, None]
        src = (off[:-1, None] + torch.arange(4, device=off.device)[None, :]).clamp(max=max(int(off[-1]) - 1, 0))
        assert torch.equal(h4[rows], idx[src][rows])
        assert torch.equal(t4[rows].view(torch.int32), tt[src][rows].view(torch.int32))
        h1, t1 = t.ray_nearest(rays)
        assert torch.equal(h1, h4[:, 0]) and torch.equal(t1.view(torch.int32), t4[:, 0].view(torch.int32))
    arbx.stream_check()


def test_rays_at_vertices_and_edges(arbx):
    """Rays aimed exactly at triangle vertices and edge midpoints, where a
    rounded Moller-Trumbore hit can fall just outside the exact triangle box;
    the padded culling must keep every such hit."""
    rng = np.random.default_rng(17)
    n = 5000
    v0 = rng.random((n, 3))
    tris = np.stack([v0, v0 + rng.normal(0, 0.02, (n, 3)), v0 + rng.normal(0, 0.02, (n, 3))], 1).astype(np.float32)
    tgt = []
    for t in tris[:2000]:
        tgt += [t[0], t[1], t[2], (t[0] + t[1]) / 2, (t[1] + t[2]) / 2, (t[0] + t[2]) / 2]
    tgt = np.asarray(tgt, np.float64)
    org = rng.random((len(tgt), 3)) * 1.4 - 0.2
    d = tgt - org
    rays = np.concatenate([org, d], 1).astype(np.float32)
    for q in (False, True, "parent"):
        tree = arbx.Tree(torch.from_numpy(tris).cuda(), kind="triangle", quantized=q)
        h, tt = tree.ray_nearest(torch.from_numpy(rays).cuda())
        rh, rt = oracle.ray_nearest(tris, rays)
        assert np.array_equal(h.cpu().numpy(), rh), q
        assert np.array_equal(tt.cpu().numpy().view(np.uint32), rt.view(np.uint32)), q
    assert (rh >= 0).mean() > 0.5


QNODE = np.dtype([("origin", "<f4", 3), ("exps", "i1", 3), ("pad", "u1"), ("q", "<u2", (2, 2, 3)),
                  ("child", "<i4", 2)])
TRILEAF = np.dtype([("v", "<f4", 9), ("orig", "<i4"), ("pad", "<i4", 2)])


def test_quantized_boxes_contain_children(arbx):
    tris = workloads.heightfield_triangles(129, 65, seed=21)
    tree = arbx.Tree(torch.from_numpy(tris.reshape(-1, 9)).cuda().view(-1, 3, 3), kind="triangle", quantized=True)
    ex = tree.export()
    nodes = ex["nodes"].view(QNODE)
    leaves = ex["leaves"].view(TRILEAF)
    assert len(nodes) == len(tris) - 1 and len(leaves) == len(tris)
    lv = leaves["v"].reshape(-1, 3, 3).astype(np.float64)
    leaf_lo, leaf_hi = lv.min(1), lv.max(1)
    lo = np.full((len(nodes), 3), np.inf)
    hi = np.full((len(nodes), 3), -np.inf)
    # exact boxes bottom-up (iterative post-order from the root)
    stack, seen = [ex["root"]], set()
    while stack:
        g = stack[-1]
        kids = [c for c in nodes["child"][g] if c >= 0 and c not in seen]
        if kids:
            stack.extend(kids)
            continue
        stack.pop()
        seen.add(g)
        for c in nodes["child"][g]:
            clo, chi = (leaf_lo[~c], leaf_hi[~c]) if c < 0 else (lo[c], hi[c])
            lo[g] = np.minimum(lo[g], clo)
            hi[g] = np.maximum(hi[g], chi)
    assert len(seen) == len(nodes)
    step = np.ldexp(1.0, nodes["exps"].astype(np.int64))
    for ci in range(2):
        c = nodes["child"][:, ci]
        clo = np.where((c < 0)[:, None], leaf_lo[np.where(c < 0, ~c, 0)], lo[np.where(c >= 0, c, 0)])
        chi = np.where((c < 0)[:, None], leaf_hi[np.where(c < 0, ~c, 0)], hi[np.where(c >= 0, c, 0)])
        dlo = nodes["origin"].astype(np.float64) + nodes["q"][:, ci, 0, :] * step
        dhi = nodes["origin"].astype(np.float64) + nodes["q"][:, ci, 1, :] * step
        assert np.all(dlo <= clo) and np.all(dhi >= chi)
        # and the codes are tight: within one step (plus one float32 ulp of the
        # coordinate, from the outward-rounded difference the encoder starts from)
        ulp = np.spacing(np.abs(clo).astype(np.float32)).astype(np.float64)
        assert np.all(clo - dlo <= step + ulp)
        ulp = np.spacing(np.abs(chi).astype(np.float32)).astype(np.float64)
        assert np.all(dhi - chi <= step + ulp)


PNODE = np.dtype([("q", "<u2", (2, 2, 3)), ("child", "<i4", 2)])


def _round_f32(x, up):
    """float64 values (exact sums here) rounded to float32 toward +inf or -inf."""
    f = x.astype(np.float32)
    if up:
        return np.where(f.astype(np.float64) < x, np.nextafter(f, np.float32(np.inf)), f)
    return np.where(f.astype(np.float64) > x, np.nextafter(f, np.float32(-np.inf)), f)


def _p16_exp(ext):
    """Smallest e in [-126, 127] with 65535 * 2^e >= ext (per element)."""
    _, x = np.frexp(ext.astype(np.float64))  # ext = m * 2^x, m in [0.5, 1)
    e = np.maximum(-126, x - 1 - 15)
    e = np.where(65535.0 * np.ldexp(1.0, e) < ext, e + 1, e)
    return np.where(ext > 0, e, -126)


def test_parent_relative_boxes_contain_children(arbx):
    """The 32-byte parent-relative nodes, decoded top-down on the CPU from the
    exact root box with directed float32 rounding: every decoded child box
    holds the exact child box (leaf boxes from the triangles' vertices,
    internal boxes their unions) and lies within one step of it, and every
    node is reached once."""
    tris = workloads.heightfield_triangles(129, 65, seed=21)
    tree = arbx.Tree(torch.from_numpy(tris.reshape(-1, 9)).cuda().view(-1, 3, 3), kind="triangle",
                     quantized="parent")
    ex = tree.export()
    assert ex["node_stride"] == 32
    nodes = ex["nodes"].view(PNODE)
    leaves = ex["leaves"].view(TRILEAF)
    nn = len(nodes)
    assert nn == len(tris) - 1
    lv = leaves["v"].reshape(-1, 3, 3).astype(np.float64)
    leaf_lo, leaf_hi = lv.min(1), lv.max(1)
    # exact internal boxes, children before parents (reversed pre-order)
    lo = np.full((nn, 3), np.inf)
    hi = np.full((nn, 3), -np.inf)
    order, stack = [], [ex["root"]]
    while stack:
        g = stack.pop()
        order.append(g)
        stack.extend(c for c in nodes["child"][g] if c >= 0)
    assert sorted(order) == list(range(nn))
    for g in reversed(order):
        for c in nodes["child"][g]:
            clo, chi = (leaf_lo[~c], leaf_hi[~c]) if c < 0 else (lo[c], hi[c])
            lo[g] = np.minimum(lo[g], clo)
            hi[g] = np.maximum(hi[g], chi)
    # top-down decode, one level at a time
    root = ex["root"]
    f_lo = lo[root][None, :].astype(np.float32)
    f_e = _p16_exp(_round_f32(hi[root][None, :] - lo[root][None, :], up=True))
    level = np.array([root])
    seen = 0
    while len(level):
        seen += len(level)
        step = np.ldexp(1.0, f_e)
        nxt, nxt_lo, nxt_e = [], [], []
        for ci in range(2):
            c = nodes["child"][level, ci]
            q = nodes["q"][level, ci].astype(np.float64)  # [k][lo/hi][axis]
            dlo = _round_f32(f_lo.astype(np.float64) + q[:, 0] * step, up=False)
            dhi = _round_f32(f_lo.astype(np.float64) + q[:, 1] * step, up=True)
            leaf = (c < 0)[:, None]
            clo = np.where(leaf, leaf_lo[np.where(c < 0, ~c, 0)], lo[np.where(c >= 0, c, 0)])
            chi = np.where(leaf, leaf_hi[np.where(c < 0, ~c, 0)], hi[np.where(c >= 0, c, 0)])
            assert np.all(dlo <= clo) and np.all(dhi >= chi)
            ulp = np.spacing(np.abs(clo).astype(np.float32)).astype(np.float64)
            assert np.all(clo - dlo <= step + ulp)
            ulp = np.spacing(np.abs(chi).astype(np.float32)).astype(np.float64)
            assert np.all(dhi - chi <= step + ulp)
            inner = c >= 0
            nxt.append(c[inner])
            nxt_lo.append(dlo[inner])
            nxt_e.append(_p16_exp(_round_f32(dhi[inner].astype(np.float64) - dlo[inner].astype(np.float64),
                                             up=True)))
        level = np.concatenate(nxt)
        f_lo = np.concatenate(nxt_lo).astype(np.float32)
        f_e = np.concatenate(nxt_e)
    assert seen == nn
