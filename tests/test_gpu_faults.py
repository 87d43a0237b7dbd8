"""Failure handling without a GPU fault: device allocations made to fail on
the host (arbx_debug_fail_allocs) at every point of a call.  Each call
either fails with ARBX_ERR_OOM or (where the library has a fallback, the
single-pass storage query) returns the normal result; afterwards the same
calls return the oracle's bytes, the device error word is clean and a served
request that failed leaves the server working."""
from __future__ import annotations

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
    yield m
    m.debug_fail_allocs(0, 0)


def cu(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def each_failure_point(arbx, call, max_points=60):
    """Run call() with the (k+1)-th allocation failing, k = 0, 1, ...; stop
    once a call needs fewer allocations than k.  Returns the outcomes."""
    outcomes = []
    for k in range(max_points):
        arbx.debug_fail_allocs(k, 1)
        try:
            out = call()
            outcomes.append(("ok", out))
        except arbx.ArbxError as e:
            assert e.status == arbx.ERR_OOM, (k, e.status)
            outcomes.append(("oom", None))
        finally:
            arbx.debug_fail_allocs(0, 0)
        torch.cuda.synchronize()
        arbx.stream_check()
        if outcomes[-1][0] == "ok" and k > 0 and all(o[0] == "ok" for o in outcomes[-3:]):
            break
    return outcomes


def test_build_and_storage_queries_fail_cleanly(arbx):
    wl = workloads.tiny_uniform()
    pts, qs, r = wl["points"], wl["queries"], wl["radius"]
    ref = oracle.radius(pts, qs, r)
    rk = oracle.knn(pts, qs, 8)
    outs = each_failure_point(arbx, lambda: arbx.Tree(cu(pts)))
    assert any(o[0] == "oom" for o in outs)
    t = arbx.Tree(cu(pts))
    q = cu(qs)
    for tu in (dict(single_pass=0), dict(single_pass=1)):
        outs = each_failure_point(arbx, lambda: t.radius(q, r, tuning=tu))
        assert any(o[0] == "oom" for o in outs)
        for kind, out in outs:
            if kind == "ok":
                assert_crs_equal(out, ref, what=f"radius under injected failures {tu}")
    outs = each_failure_point(arbx, lambda: t.knn(q, 8))
    for kind, out in outs:
        if kind == "ok":
            assert np.array_equal(to_np(out[0]), rk[0])
    assert_crs_equal(t.radius(q, r), ref, what="radius after injected failures")
    idx, d2 = t.knn(q, 8)
    assert np.array_equal(to_np(idx), rk[0]) and np.array_equal(to_np(d2).view(np.uint32), rk[1].view(np.uint32))


def test_ray_dbscan_forest_fail_cleanly(arbx):
    tris = workloads.heightfield_triangles(33, 17, seed=9)
    rays = workloads.heightfield_rays(500, seed=10, extent_x=32 * workloads.HF_SPACING,
                                      extent_y=16 * workloads.HF_SPACING)
    t = arbx.Tree(cu(tris), kind="triangle", quantized=True)
    roff, ridx, rt = oracle.ray_all(tris, rays)
    outs = each_failure_point(arbx, lambda: t.ray_intersect(cu(rays), ordered=True))
    assert any(o[0] == "oom" for o in outs)
    off, idx, tt = t.ray_intersect(cu(rays), ordered=True)
    assert np.array_equal(to_np(off), roff) and np.array_equal(to_np(idx), ridx)
    pts = np.random.default_rng(3).random((3000, 3)).astype(np.float32)
    outs = each_failure_point(arbx, lambda: arbx.dbscan(cu(pts), 0.05, 4))
    assert any(o[0] == "oom" for o in outs)
    labels, nc = arbx.dbscan(cu(pts), 0.05, 4)
    rl, rn = oracle.dbscan(pts, 0.05, 4)
    assert np.array_equal(to_np(labels), rl) and nc == rn
    sets = [np.random.default_rng(s).random((200 + 50 * s, 3)).astype(np.float32) for s in range(5)]
    outs = each_failure_point(arbx, lambda: arbx.Forest([cu(x) for x in sets]))
    assert any(o[0] == "oom" for o in outs)


def test_served_request_failure_leaves_server_working(arbx):
    rng = np.random.default_rng(6)
    pts = rng.random((20000, 3)).astype(np.float32)
    qs = rng.random((3000, 3)).astype(np.float32)
    sv = arbx.Server(slots=2, hbm_budget_bytes=1 << 30)
    tid = sv.add_tree(arbx.Tree(cu(pts)))
    q = cu(qs)
    failed = 0
    for k in range(8):
        arbx.debug_fail_allocs(k, 1)
        try:
            res = sv.wait(sv.submit(tid, arbx.SPHERE, q, radius=0.03))
            res_ok = True
        except arbx.ArbxError as e:
            assert e.status == arbx.ERR_OOM
            res_ok = False
            failed += 1
        finally:
            arbx.debug_fail_allocs(0, 0)
        if res_ok:
            del res
    assert failed > 0
    res = sv.wait(sv.submit(tid, arbx.SPHERE, q, radius=0.03))
    ref = oracle.radius(pts, qs, 0.03)
    assert_crs_equal((res.offsets, res.indices, res.d2), ref, what="served after failures")
    sv.close()
