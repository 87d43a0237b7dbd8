"""Visit counts of the instrumented traversals against a CPU walk of the exported tree.

The roofline's algorithmic bytes count node records: for a spatial predicate the
nodes whose box passes the predicate, for a nearest query the nodes whose box lies
within the final k-th distance (the set every exact best-first search must open,
section 2.1 nearest predicates).  These tests export small trees (arbx_tree_export),
walk them on the CPU with the box distance computed in float32 in the library's
operation order (per axis fl(q - clamp(q)) squared, summed in dimension order, no
fused multiply-add -- numpy float32 arithmetic rounds every operation), and require
the GPU counters to equal the walk exactly:

* arbx_query_stats (the fill pass's walk): every internal node whose box passes;
* arbx_query_count_stats (the count pass's walk): the same, except that an internal
  child whose box lies wholly inside the sphere is counted whole, not visited;
* arbx_query_stats_r2 with the kNN's final k-th squared distances: every internal
  node whose box distance is <= that distance; the kNN kernel's own fetch count
  (arbx_query_stats with a nearest predicate) is never below it.

The counting and nearest traversals can open four-wide records instead (tuning
wide_nodes; record g holds binary node g's grandchildren, so one step descends two
levels); their counters are checked against the same walk over records simulated
from the binary export, and with wide_nodes=0 against the binary walk.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import workloads
from crs_util import to_np

pytestmark = pytest.mark.gpu

NULL_CHILD = np.int32(-(2 ** 31))


@pytest.fixture(scope="module")
def arbx():
    import paper_2507_23700_b300 as m
    return m


def node_dtype(dim):
    return np.dtype([("lo0", "<f4", dim), ("hi0", "<f4", dim), ("lo1", "<f4", dim), ("hi1", "<f4", dim),
                     ("child", "<i4", 2), ("orig", "<i4", 2)])


def box_d2(q, lo, hi):
    """Squared distance from q to the box, float32, axis terms summed in order."""
    c = np.minimum(np.maximum(q, lo), hi)
    d = (q - c).astype(np.float32)
    s = (d * d).astype(np.float32)
    acc = s[:, 0].copy()
    for a in range(1, q.shape[1]):
        acc = (acc + s[:, a]).astype(np.float32)
    return acc


def far_d2(q, lo, hi):
    """Squared distance to the box's farthest corner, per axis the larger face term."""
    d0 = (q - lo).astype(np.float32)
    d1 = (q - hi).astype(np.float32)
    s = np.maximum((d0 * d0).astype(np.float32), (d1 * d1).astype(np.float32))
    acc = s[:, 0].copy()
    for a in range(1, q.shape[1]):
        acc = (acc + s[:, a]).astype(np.float32)
    return acc


def cpu_walk(nodes, root, qs, r2, contain=False):
    """Breadth-first walk over (query, node) pairs: returns (internal nodes
    fetched, leaf children matched) summed over all queries.  r2 is one float32
    per query."""
    qidx = np.arange(len(qs))
    cur = np.full(len(qs), root, np.int64)
    fetched = 0
    matched = 0
    while len(qidx):
        fetched += len(qidx)
        nd = nodes[cur]
        q = qs[qidx]
        rq = r2[qidx]
        nxt_q, nxt_n = [], []
        for c in (0, 1):
            lo, hi = nd[f"lo{c}"], nd[f"hi{c}"]
            child = nd["child"][:, c]
            valid = child != NULL_CHILD
            hit = valid & (box_d2(q, lo, hi) <= rq)
            leaf = hit & (child < 0)
            matched += int(leaf.sum())
            inner = hit & (child >= 0)
            if contain:
                inner &= ~(far_d2(q, lo, hi) <= rq)
            nxt_q.append(qidx[inner])
            nxt_n.append(child[inner].astype(np.int64))
        qidx = np.concatenate(nxt_q)
        cur = np.concatenate(nxt_n)
    return fetched, matched


def cpu_walk_wide(nodes, root, qs, r2, contain=False):
    """The same walk over four-wide records: record g holds the children of
    g's internal children and g's leaf children (one step descends two binary
    levels).  Returns the records fetched summed over all queries."""
    qidx = np.arange(len(qs))
    cur = np.full(len(qs), root, np.int64)
    fetched = 0
    while len(qidx):
        fetched += len(qidx)
        nd = nodes[cur]
        nxt_q, nxt_n = [], []
        entries = []  # (query index, lo, hi, code) per candidate entry
        for c in (0, 1):
            child = nd["child"][:, c]
            leaf = (child < 0) & (child != NULL_CHILD)
            entries.append((qidx[leaf], nd[f"lo{c}"][leaf], nd[f"hi{c}"][leaf], child[leaf]))
            inner = child >= 0
            ch = nodes[child[inner].astype(np.int64)]
            for gc in (0, 1):
                code = ch["child"][:, gc]
                ok = code != NULL_CHILD
                entries.append((qidx[inner][ok], ch[f"lo{gc}"][ok], ch[f"hi{gc}"][ok], code[ok]))
        for eq, lo, hi, code in entries:
            if len(eq) == 0:
                continue
            q = qs[eq]
            rq = r2[eq]
            go = (code >= 0) & (box_d2(q, lo, hi) <= rq)
            if contain:
                go &= ~(far_d2(q, lo, hi) <= rq)
            nxt_q.append(eq[go])
            nxt_n.append(code[go].astype(np.int64))
        qidx = np.concatenate(nxt_q) if nxt_q else np.zeros(0, np.int64)
        cur = np.concatenate(nxt_n) if nxt_n else np.zeros(0, np.int64)
    return fetched


# one traversal per query (warp packets, the default for k = 1, count one
# fetch per warp)
BINARY = dict(wide_nodes=0, warp_packets=0)
WIDE = dict(wide_nodes=1, warp_packets=0)


def exported(tree, dim):
    ex = tree.export()
    assert ex["node_stride"] == node_dtype(dim).itemsize
    return ex["nodes"].view(node_dtype(dim)), ex["root"]


@pytest.mark.parametrize("dim", [2, 3, 6])
@pytest.mark.parametrize("n", [2, 37, 5003])
def test_spatial_visit_counts(arbx, dim, n):
    rng = np.random.default_rng(40 + dim * 7 + n)
    pts = rng.random((n, dim), dtype=np.float32)
    pts[n // 2:n // 2 + min(5, n // 2)] = pts[0]
    qs = rng.random((431, dim), dtype=np.float32)
    r = float((24.0 / (workloads.unit_ball_volume(dim) * n)) ** (1.0 / dim))
    tree = arbx.Tree(torch.from_numpy(pts).cuda(), wide=True)
    nodes, root = exported(tree, dim)
    q = torch.from_numpy(qs).cuda()
    r2 = np.full(len(qs), np.float32(r) * np.float32(r), np.float32)
    total = int(oracle.radius(pts, qs, r)[0][-1])
    st = tree.stats(arbx.SPHERE, q, r)
    f, mt = cpu_walk(nodes, root, qs, r2)
    assert (st["nodes"], st["matches"]) == (f, mt) and mt == total
    cs = tree.stats(arbx.SPHERE, q, r, counting=True, tuning=BINARY)
    fc, _ = cpu_walk(nodes, root, qs, r2, contain=True)
    assert (cs["nodes"], cs["matches"]) == (fc, total)
    assert fc <= f
    # the count pass over four-wide records
    cw = tree.stats(arbx.SPHERE, q, r, counting=True, tuning=WIDE)
    assert (cw["nodes"], cw["matches"]) == (cpu_walk_wide(nodes, root, qs, r2, contain=True), total)
    # the same walks with the squared radii passed per query
    r2d = torch.from_numpy(r2).cuda()
    s2 = tree.stats_r2(q, r2d, tuning=BINARY)
    assert (s2["nodes"], s2["matches"]) == (f, total)
    s2w = tree.stats_r2(q, r2d, tuning=WIDE)
    assert (s2w["nodes"], s2w["matches"]) == (cpu_walk_wide(nodes, root, qs, r2), total)
    # box predicates: the counting walk over four-wide records
    h = np.float32(r)
    boxes = np.concatenate([qs - h, qs + h], 1).astype(np.float32)
    bw = tree.stats(arbx.BOX_PRED, torch.from_numpy(boxes).cuda(), counting=True, tuning=WIDE)
    assert bw["matches"] == int(oracle.box_query(pts, oracle.POINT, boxes)[0][-1])


@pytest.mark.parametrize("dim", [2, 3, 6])
@pytest.mark.parametrize("k", [1, 8, 16, 64])
def test_knn_visit_set(arbx, dim, k):
    rng = np.random.default_rng(90 + dim * 11 + k)
    n = 4099
    pts = rng.random((n, dim), dtype=np.float32)
    qs = np.concatenate([rng.random((300, dim), dtype=np.float32),
                         pts[:60] + np.float32(1e-4)]).astype(np.float32)
    tree = arbx.Tree(torch.from_numpy(pts).cuda(), wide=True)
    nodes, root = exported(tree, dim)
    q = torch.from_numpy(qs).cuda()
    _, d2 = tree.knn(q, k)
    kth = d2[:, -1].contiguous()
    st = tree.stats_r2(q, kth, tuning=BINARY)
    f, mt = cpu_walk(nodes, root, qs, to_np(kth))
    assert st["nodes"] == f
    # matches: the points within the k-th distance, ties included (at least k each)
    assert st["matches"] == mt and mt >= k * len(qs)
    fetched = tree.stats(arbx.NEAREST, q, k=k, tuning=dict(BINARY, query_runs=1, sort_queries=1))["nodes"]
    assert fetched >= f
    # lane runs prune with a carried bound that never drops below the k-th
    # distance: still every node of the optimal set
    for r in (4, 8):
        assert tree.stats(arbx.NEAREST, q, k=k, tuning=dict(BINARY, query_runs=r))["nodes"] >= f
    # a warp packet fetches each record once for its 32 (Morton-sorted, so
    # neighbouring) queries: at least the optimal set of its busiest query, at
    # most the sum over its queries
    pk = tree.stats(arbx.NEAREST, q, k=k, tuning=dict(warp_packets=1, sort_queries=1))["nodes"]
    assert f / 32 <= pk <= fetched
    # over four-wide records (k <= 32)
    sw = tree.stats_r2(q, kth, tuning=WIDE)
    fw = cpu_walk_wide(nodes, root, qs, to_np(kth))
    assert sw["nodes"] == fw and sw["matches"] == mt
    if k <= 32:
        for r in (1, 4, 8):
            assert tree.stats(arbx.NEAREST, q, k=k, tuning=dict(WIDE, query_runs=r))["nodes"] >= fw


def test_knn_visit_set_k_above_n(arbx):
    """k > n: the list never fills, the k-th distance is +inf and every node is opened."""
    pts = np.random.default_rng(5).random((40, 3), dtype=np.float32)
    qs = np.random.default_rng(6).random((17, 3), dtype=np.float32)
    tree = arbx.Tree(torch.from_numpy(pts).cuda(), wide=True)
    r2 = torch.full((17,), float("inf"), device="cuda")
    st = tree.stats_r2(torch.from_numpy(qs).cuda(), r2, tuning=BINARY)
    assert st["nodes"] == 17 * 39 and st["matches"] == 17 * 40
    assert tree.stats(arbx.NEAREST, torch.from_numpy(qs).cuda(), k=64)["nodes"] == 17 * 39
    nodes, root = exported(tree, 3)
    fw = cpu_walk_wide(nodes, root, qs, np.full(17, np.inf, np.float32))
    assert tree.stats_r2(torch.from_numpy(qs).cuda(), r2, tuning=WIDE)["nodes"] == fw
    # the four-wide nearest traversal with k > n opens every record too
    small = arbx.Tree(torch.from_numpy(pts[:20]).cuda(), wide=True)
    nodes, root = exported(small, 3)
    fw = cpu_walk_wide(nodes, root, qs, np.full(17, np.inf, np.float32))
    assert small.stats(arbx.NEAREST, torch.from_numpy(qs).cuda(), k=32, tuning=WIDE)["nodes"] == fw
