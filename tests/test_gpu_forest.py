"""GPU parity of forests (many independent trees built and queried together).

* A small mixed forest (dims 2/3/6, empty, one-point and ragged sets, sets
  without queries): every query's radius CRS (sets + d2 bits) and kNN list equal
  the oracle run on that query's own set.
* The captured CUDA graph of a batch (radius count/scan/fill + kNN) replays to
  the same bytes.
* The full forest workload (4096 sets, dims uniform over {2,3,6}, sizes
  log-uniform 1e3..1e6, 0.5-2x queries, per-set radius for ~16 neighbours,
  k=8), in the configuration bench.py times: 4 sampled queries per set equal the
  oracle; every CRS segment count equals the count pass.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import workloads
from crs_util import assert_crs_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arbx():
    import paper_2507_23700_b300 as m
    return m


def small_forest(seed=5):
    rng = np.random.default_rng(seed)
    sizes = [0, 1, 2, 3, 7, 31, 1000, 4113, 20000] + list(rng.integers(1, 6000, 39))
    sets, queries, radii = [], [], []
    for i, n in enumerate(sizes):
        d = [2, 3, 6][i % 3]
        sets.append(rng.random((int(n), d), dtype=np.float32))
        m = 0 if i % 11 == 5 else int(rng.integers(1, 700))
        queries.append(rng.random((m, d), dtype=np.float32))
        radii.append(float(np.float32((12.0 / (workloads.unit_ball_volume(d) * max(n, 1))) ** (1.0 / d))))
    return sets, queries, radii


def pack(arrs):
    return torch.from_numpy(np.concatenate([a.reshape(-1) for a in arrs])).cuda() if arrs else None


def test_small_forest_every_query(arbx):
    sets, queries, radii = small_forest()
    forest = arbx.Forest([torch.from_numpy(s).cuda() for s in sets])
    assert forest.info() == (len(sets), sum(len(s) for s in sets))
    batch = arbx.ForestBatch(forest, [len(q) for q in queries], radii)
    qd = pack(queries)
    off, idx, d2 = batch.radius(qd)
    k = 8
    kidx, kd2 = batch.knn(qd, k)
    off, idx, d2 = off.cpu().numpy(), idx.cpu().numpy(), d2.cpu().numpy()
    kidx, kd2 = kidx.cpu().numpy(), kd2.cpu().numpy()
    g = 0
    for s, (pts, qs, r) in enumerate(zip(sets, queries, radii)):
        m = len(qs)
        if m == 0:
            continue
        seg = slice(g, g + m)
        lo = off[g]
        sub_off = off[g:g + m + 1] - lo
        sub = (sub_off, idx[lo:off[g + m]], d2[lo:off[g + m]])
        assert_crs_equal(sub, oracle.radius(pts, qs, r), what=f"set {s} (n={len(pts)}, d={pts.shape[1]})")
        ridx, rd2 = oracle.knn(pts, qs, k)
        kk = ridx.shape[1]
        assert np.array_equal(kidx[seg, :kk], ridx), s
        assert np.array_equal(kd2[seg, :kk].view(np.uint32), rd2.view(np.uint32)), s
        assert np.all(kidx[seg, kk:] == -1) and np.all(np.isinf(kd2[seg, kk:])), s
        g += m
    assert g == batch.total


FOREST_TUNINGS = [dict(block=b, chunk=c, sort_queries=sq) for b in (128, 256) for c in (32, 64)
                  for sq in ([1, 1, 1], [0, 0, 0], [1, 0, 1])]


def test_forest_tunings_same_bytes_and_autotune(arbx, tmp_path):
    """Every batched launch setting (block size, chunk size, query ordering per
    dimension group) gives the same bytes as the defaults, which equal the
    oracle (test above); the autotuner's choice becomes the batch's setting,
    is recorded for new batches of the same shape, and survives save/load."""
    sets, queries, radii = small_forest(seed=13)
    forest = arbx.Forest([torch.from_numpy(s).cuda() for s in sets])
    batch = arbx.ForestBatch(forest, [len(q) for q in queries], radii)
    qd = pack(queries)
    assert batch.tuning() == {"block": 256, "chunk": 32, "sort_queries": [1, 1, 1]}
    base = batch.radius(qd) + batch.knn(qd, 8)
    for tu in FOREST_TUNINGS:
        batch.set_tuning(tu)
        assert batch.tuning() == tu
        got = batch.radius(qd) + batch.knn(qd, 8)
        assert all(torch.equal(a, b) for a, b in zip(base, got)), tu
    with pytest.raises(arbx.ArbxError):
        batch.set_tuning(dict(block=96))
    with pytest.raises(arbx.ArbxError):
        batch.set_tuning(dict(chunk=48))
    arbx.autotune_clear()
    best, ms = batch.autotune(qd, 8)
    assert ms > 0 and best == batch.tuning() and best["block"] in (128, 256) and best["chunk"] in (32, 64)
    got = batch.radius(qd) + batch.knn(qd, 8)
    assert all(torch.equal(a, b) for a, b in zip(base, got))
    # a new batch of the same shape starts from the recorded setting
    assert arbx.ForestBatch(forest, [len(q) for q in queries], radii).tuning() == best
    f = tmp_path / "tune.txt"
    arbx.autotune_save(f)
    assert any(ln.startswith("forest ") for ln in f.read_text().splitlines())
    arbx.autotune_clear()
    assert arbx.ForestBatch(forest, [len(q) for q in queries], radii).tuning()["chunk"] == 32
    arbx.autotune_load(f)
    assert arbx.ForestBatch(forest, [len(q) for q in queries], radii).tuning() == best
    arbx.autotune_clear()
    # the graph captures the batch's setting at capture time
    batch.set_tuning(dict(block=128, chunk=64, sort_queries=[0, 1, 0]))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        off = torch.empty(batch.total + 1, dtype=torch.int64, device="cuda")
        cap = int(base[0][-1])
        idx = torch.empty(cap, dtype=torch.int32, device="cuda")
        d2 = torch.empty(cap, dtype=torch.float32, device="cuda")
        kidx = torch.empty((batch.total, 8), dtype=torch.int32, device="cuda")
        kd2 = torch.empty((batch.total, 8), dtype=torch.float32, device="cuda")
        g = batch.graph(qd, off, idx, d2, cap, None, 8, kidx, kd2, stream)
        g.launch(stream)
    stream.synchronize()
    for a, b in zip(base, (off, idx, d2, kidx, kd2)):
        assert torch.equal(a, b)
    g.close()


def test_forest_graph_replay(arbx):
    sets, queries, radii = small_forest(seed=9)
    forest = arbx.Forest([torch.from_numpy(s).cuda() for s in sets])
    batch = arbx.ForestBatch(forest, [len(q) for q in queries], radii)
    qd = pack(queries)
    off, idx, d2 = batch.radius(qd)
    kidx, kd2 = batch.knn(qd, 8)
    nnz = int(off[-1])
    s = torch.cuda.Stream()
    g_off = torch.empty_like(off)
    g_idx = torch.full((nnz,), -5, dtype=torch.int32, device="cuda")
    g_d2 = torch.empty(nnz, dtype=torch.float32, device="cuda")
    g_nnz = torch.zeros(1, dtype=torch.int64, device="cuda")
    g_kidx = torch.empty_like(kidx)
    g_kd2 = torch.empty_like(kd2)
    torch.cuda.synchronize()
    graph = batch.graph(qd, g_off, g_idx, g_d2, nnz, g_nnz, 8, g_kidx, g_kd2, stream=s)
    for _ in range(2):
        graph.launch(stream=s)
        s.synchronize()
        assert int(g_nnz.item()) == nnz
        assert torch.equal(g_off, off) and torch.equal(g_idx, idx) and torch.equal(g_d2, d2)
        assert torch.equal(g_kidx, kidx) and torch.equal(g_kd2, kd2)
        g_idx.fill_(-5)
    graph.close()


def test_full_forest_sampled(arbx):
    plan = workloads.forest_plan()
    dims = np.array([p[0] for p in plan], np.int32)
    ns = np.array([p[1] for p in plan], np.int64)
    ms = np.array([p[2] for p in plan], np.int64)
    pfl = int((ns * dims).sum())
    qfl = int((ms * dims).sum())
    pts_d = torch.empty(pfl, dtype=torch.float32, device="cuda")
    qs_d = torch.empty(qfl, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(123)
    expected = []
    po = qo = 0
    radii = []
    for s in range(len(plan)):
        fs = workloads.forest_set(plan, s)
        n, m, d = len(fs.points), len(fs.queries), fs.dim
        pts_d[po:po + n * d].copy_(torch.from_numpy(fs.points.reshape(-1)))
        qs_d[qo:qo + m * d].copy_(torch.from_numpy(fs.queries.reshape(-1)))
        po += n * d
        qo += m * d
        radii.append(fs.radius)
        sel = np.sort(rng.choice(m, min(4, m), replace=False))
        expected.append((sel, oracle.radius(fs.points, fs.queries[sel], fs.radius, threads=1),
                         oracle.knn(fs.points, fs.queries[sel], fs.k, threads=1)))
    forest = arbx.Forest(packed=pts_d, dims=dims, counts=ns)
    batch = arbx.ForestBatch(forest, ms, radii)
    off, idx, d2 = batch.radius(qs_d)
    kidx, kd2 = batch.knn(qs_d, 8)
    gbase = np.concatenate([[0], np.cumsum(ms)])
    rows = np.concatenate([gbase[s] + e[0] for s, e in enumerate(expected)])
    rows_t = torch.from_numpy(rows).cuda()
    lo, hi = off[rows_t], off[rows_t + 1]
    lens = (hi - lo).cpu().numpy()
    pos = torch.repeat_interleave(lo, hi - lo) + (torch.arange(int(lens.sum()), device="cuda") -
                                                 torch.repeat_interleave(torch.cumsum(hi - lo, 0) - (hi - lo), hi - lo))
    g_idx, g_d2 = idx[pos].cpu().numpy(), d2[pos].cpu().numpy()
    g_kidx, g_kd2 = kidx[rows_t].cpu().numpy(), kd2[rows_t].cpu().numpy()
    a = 0
    r = 0
    for s, (sel, rad, kn) in enumerate(expected):
        nq = len(sel)
        l = lens[r:r + nq]
        sub_off = np.concatenate([[0], np.cumsum(l)])
        assert_crs_equal((sub_off, g_idx[a:a + l.sum()], g_d2[a:a + l.sum()]), rad, what=f"forest set {s}")
        assert np.array_equal(g_kidx[r:r + nq], kn[0]), s
        assert np.array_equal(g_kd2[r:r + nq].view(np.uint32), kn[1].view(np.uint32)), s
        a += int(l.sum())
        r += nq
