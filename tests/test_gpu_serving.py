"""Serving runtime: every request's result is the same alone and in the mix.

A server with resident trees runs a stream of mixed requests (radius CRS,
kNN with k in {1, 8, 32}, count callbacks; sizes from 1 to 20k queries).  Each
request is first served alone (one at a time), then all are submitted at once
to a server with several slots, where they are admitted as slots and memory
free up and overlap on the device.  Results must be byte-identical (the
stated tolerance is exact), and a few are checked against the oracle.  A
tight memory budget must still complete every request with the same bytes,
and a host-side wait limit must report a timeout without stopping the work.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

KINDS = ("radius", "knn1", "knn8", "knn32", "count")


@pytest.fixture(scope="module")
def arbx():
    import paper_2507_23700_b300 as m
    return m


def make_requests(nreq=60, seed=3):
    rng = np.random.default_rng(seed)
    model = workloads.mixture_model(77)
    reqs = []
    for i in range(nreq):
        size = int(np.exp(rng.uniform(0, np.log(20000))))
        kind = KINDS[i % len(KINDS)]
        tree = int(rng.integers(0, 2))
        q = workloads.mixture_points(model, size, 9000 + i)
        reqs.append((tree, kind, q))
    return reqs


@pytest.fixture(scope="module")
def trees_host():
    model = workloads.mixture_model(77)
    return [workloads.mixture_points(model, 200_000, 78), workloads.mixture_points(model, 500_000, 79)]


def radius_for(n):
    return float(np.float32(workloads.LARGE_RADIUS * (1e7 / n) ** (1.0 / 3.0)))


def new_server(arbx, trees_host, slots, budget):
    sv = arbx.Server(slots=slots, hbm_budget_bytes=budget)
    for pts in trees_host:
        sv.add_tree(arbx.Tree(torch.from_numpy(pts).cuda()))
    return sv


def submit(arbx, sv, trees_host, tree, kind, q):
    qd = torch.from_numpy(q).cuda()
    r = radius_for(len(trees_host[tree]))
    if kind == "radius":
        return sv.submit(tree, arbx.SPHERE, qd, radius=r)
    if kind == "count":
        return sv.submit(tree, arbx.SPHERE, qd, radius=r, callback=arbx.CB_COUNT)
    return sv.submit(tree, arbx.NEAREST, qd, k=int(kind[3:]))


def to_host(res):
    out = {}
    for name in ("offsets", "indices", "d2", "counts"):
        t = getattr(res, name)
        out[name] = None if t is None else t.cpu().numpy().copy()
    return out


def same(a, b):
    for name in ("offsets", "indices", "d2", "counts"):
        x, y = a[name], b[name]
        if (x is None) != (y is None):
            return False
        if x is not None and not np.array_equal(x.view(np.uint8), y.view(np.uint8)):
            return False
    return True


def test_alone_equals_mix(arbx, trees_host):
    reqs = make_requests()
    alone_sv = new_server(arbx, trees_host, slots=1, budget=64 << 30)
    alone = []
    for tree, kind, q in reqs:
        t = submit(arbx, alone_sv, trees_host, tree, kind, q)
        alone.append(to_host(alone_sv.wait(t)))
    alone_sv.close()
    for slots, budget in ((4, 64 << 30), (8, 1 << 20)):
        sv = new_server(arbx, trees_host, slots=slots, budget=budget)
        tickets = [submit(arbx, sv, trees_host, tree, kind, q) for tree, kind, q in reqs]
        mixed = [to_host(sv.wait(t)) for t in tickets]
        st = sv.stats()
        assert st["completed"] == len(reqs) and st["p99_s"] >= st["p50_s"] > 0
        sv.close()
        for i, (a, b) in enumerate(zip(alone, mixed)):
            assert same(a, b), (i, reqs[i][1], slots, budget)
    # spot checks against the oracle
    for i, (tree, kind, q) in enumerate(reqs[:15]):
        pts = trees_host[tree]
        q = q[:300]
        n = len(q)
        if kind == "radius":
            r_off, r_idx, r_d2 = oracle.radius(pts, q, radius_for(len(pts)))
            off = alone[i]["offsets"][:n + 1]
            assert np.array_equal(off, r_off), i
            for j in range(n):
                seg = sorted(zip(alone[i]["indices"][off[j]:off[j + 1]].tolist(),
                                 alone[i]["d2"][off[j]:off[j + 1]].view(np.uint32).tolist()))
                exp = sorted(zip(r_idx[r_off[j]:r_off[j + 1]].tolist(),
                                 r_d2[r_off[j]:r_off[j + 1]].view(np.uint32).tolist()))
                assert seg == exp, (i, j)
        elif kind == "count":
            assert np.array_equal(alone[i]["counts"][:n], oracle.radius_count(pts, q, radius_for(len(pts)))), i
        else:
            k = int(kind[3:])
            ridx, rd2 = oracle.knn(pts, q, k)
            assert np.array_equal(alone[i]["indices"][:n * k], ridx.reshape(-1)), i
            assert np.array_equal(alone[i]["d2"][:n * k].view(np.uint32), rd2.reshape(-1).view(np.uint32)), i


def check_sample_vs_oracle(pts, q, r, kind, res, sample):
    """Rows `sample` of a served result against the oracle run on those queries."""
    qs = q[sample]
    if kind == "count":
        assert np.array_equal(res["counts"][sample], oracle.radius_count(pts, qs, r))
        return
    if kind == "radius":
        off = res["offsets"]
        r_off, r_idx, r_d2 = oracle.radius(pts, qs, r)
        for j, i in enumerate(sample):
            seg = sorted(zip(res["indices"][off[i]:off[i + 1]].tolist(),
                             res["d2"][off[i]:off[i + 1]].view(np.uint32).tolist()))
            exp = sorted(zip(r_idx[r_off[j]:r_off[j + 1]].tolist(), r_d2[r_off[j]:r_off[j + 1]].view(np.uint32).tolist()))
            assert seg == exp, (kind, int(i))
        return
    k = int(kind[3:])
    ridx, rd2 = oracle.knn(pts, qs, k)
    gi = res["indices"].reshape(-1, k)[sample]
    gd = res["d2"].reshape(-1, k)[sample]
    assert np.array_equal(gi, ridx), kind
    assert np.array_equal(gd.view(np.uint32), rd2.view(np.uint32)), kind


def test_config_size_requests(arbx):
    """Requests of the serving workload's largest size (1M queries) of every
    kind on a resident 20M-point mixture tree, mixed with small requests on a
    second tree: served together they give the bytes they give alone, and a
    seeded 300-row sample of each large request equals the oracle (kNN indices
    and d2 bits)."""
    model = workloads.mixture_model(5001 * 100)
    big = workloads.mixture_points(model, 20_000_000, 5001 * 100 + 1)
    small = workloads.mixture_points(workloads.mixture_model(77), 1_000_000, 80)
    trees = [big, small]
    reqs = [(0, kind, workloads.mixture_points(model, 1_000_000, 7700 + i)) for i, kind in enumerate(KINDS)]
    rng = np.random.default_rng(11)
    for i in range(20):
        size = int(np.exp(rng.uniform(0, np.log(50000))))
        reqs.append((1, KINDS[i % len(KINDS)], workloads.mixture_points(workloads.mixture_model(77), size, 8800 + i)))
    alone_sv = new_server(arbx, trees, slots=1, budget=64 << 30)
    alone = [to_host(alone_sv.wait(submit(arbx, alone_sv, trees, t, kind, q))) for t, kind, q in reqs]
    alone_sv.close()
    sv = new_server(arbx, trees, slots=4, budget=64 << 30)
    tickets = [submit(arbx, sv, trees, t, kind, q) for t, kind, q in reqs]
    mixed = [to_host(sv.wait(tk)) for tk in tickets]
    assert sv.stats()["completed"] == len(reqs)
    sv.close()
    for i, (a, b) in enumerate(zip(alone, mixed)):
        assert same(a, b), (i, reqs[i][1])
    sample = np.sort(np.random.default_rng(12).choice(1_000_000, 300, replace=False))
    for i, (t, kind, q) in enumerate(reqs[:len(KINDS)]):
        check_sample_vs_oracle(big, q, radius_for(len(big)), kind, alone[i], sample)


def test_over_budget_branch_fails_cleanly(arbx, trees_host):
    """A budget too small for any radius output sends the requests through the
    "oldest proceeds over budget" branch; with one device allocation failing
    there, each request ends with ARBX_ERR_OOM or its bytes, and afterwards the
    server serves every request again."""
    reqs = [r for r in make_requests(nreq=25, seed=8) if r[1] == "radius"]
    assert len(reqs) >= 4
    alone_sv = new_server(arbx, trees_host, slots=1, budget=64 << 30)
    ref = [to_host(alone_sv.wait(submit(arbx, alone_sv, trees_host, t, kind, q))) for t, kind, q in reqs]
    alone_sv.close()
    sv = new_server(arbx, trees_host, slots=3, budget=1 << 16)
    failed = 0
    for after in range(0, 12, 3):
        arbx.debug_fail_allocs(after, 1)
        try:
            tickets = [submit(arbx, sv, trees_host, t, kind, q) for t, kind, q in reqs]
            for i, tk in enumerate(tickets):
                try:
                    assert same(to_host(sv.wait(tk)), ref[i]), i
                except arbx.ArbxError as e:
                    assert e.status == arbx.ERR_OOM
                    failed += 1
        finally:
            arbx.debug_fail_allocs(0, 0)
    assert failed > 0
    tickets = [submit(arbx, sv, trees_host, t, kind, q) for t, kind, q in reqs]
    for i, tk in enumerate(tickets):
        assert same(to_host(sv.wait(tk)), ref[i]), i
    sv.close()


def test_wait_timeout_is_host_side(arbx, trees_host):
    sv = new_server(arbx, trees_host, slots=1, budget=64 << 30)
    big = workloads.mixture_points(workloads.mixture_model(77), 2_000_000, 555)
    t = submit(arbx, sv, trees_host, 1, "knn32", big)
    with pytest.raises(arbx.ArbxError) as e:
        sv.wait(t, timeout_s=0.0)
    assert e.value.status == arbx.ERR_TIMEOUT
    res = sv.wait(t)  # the request itself completes normally
    assert res.indices.numel() == 2_000_000 * 32
    sv.close()
