"""Storage queries whose results go to host memory in query ranges that fit
the device (arbx_query_crs_host), for result sets larger than device memory.

The bytes must equal the device CRS of arbx_query_crs (offsets, and indices /
d2 in the same per-query order) for every chunk budget, including budgets
smaller than one query's results (that query is filled alone); a too-small
capacity reports ARBX_ERR_CAPACITY after writing the offsets; failing device
allocations end the call with ARBX_ERR_OOM and leave the tree usable.
"""
from __future__ import annotations

import ctypes

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


def device_crs(tree, kind, q, radius=None):
    crs = tree.query_crs(kind, q, radius)
    return to_np(crs.offsets), to_np(crs.indices), None if crs.d2 is None else to_np(crs.d2)


def same(a, b):
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    if a[2] is None or b[2] is None:
        assert a[2] is None and b[2] is None
    else:
        assert np.array_equal(a[2].view(np.uint32), b[2].view(np.uint32))


@pytest.mark.parametrize("dim", [2, 3, 6])
def test_chunks_equal_device_crs(arbx, dim):
    rng = np.random.default_rng(60 + dim)
    pts = rng.random((30011, dim), dtype=np.float32)
    pts[500:900] = pts[3]  # one query sees 400+ duplicates
    qs = rng.random((4099, dim), dtype=np.float32)
    qs[17] = pts[3]
    r = float((30.0 / (workloads.unit_ball_volume(dim) * len(pts))) ** (1.0 / dim))
    t = arbx.Tree(torch.from_numpy(pts).cuda())
    q = torch.from_numpy(qs).cuda()
    ref = device_crs(t, arbx.SPHERE, q, r)
    assert_crs_equal(ref, oracle.radius(pts, qs, r), what=f"radius d={dim}")
    for chunk in (0, 8, 4096, 1 << 16, 1 << 30):
        same(t.query_crs_host(arbx.SPHERE, q, r, chunk_bytes=chunk), ref)
    # without distances, and box predicates
    off, idx, d2 = t.query_crs_host(arbx.SPHERE, q, r, want_d2=False, chunk_bytes=1000)
    assert d2 is None and np.array_equal(off, ref[0]) and np.array_equal(idx, ref[1])
    h = np.float32(r)
    boxes = torch.from_numpy(np.concatenate([qs - h, qs + h], 1).astype(np.float32)).cuda()
    bref = device_crs(t, arbx.BOX_PRED, boxes)
    same(t.query_crs_host(arbx.BOX_PRED, boxes, chunk_bytes=2048), (bref[0], bref[1], None))


def test_chunks_rays_ordered(arbx):
    tris = workloads.heightfield_triangles(129, 65, seed=31)
    rays = workloads.heightfield_rays(3000, seed=32, extent_x=128 * workloads.HF_SPACING,
                                      extent_y=64 * workloads.HF_SPACING)
    t = arbx.Tree(torch.from_numpy(tris).cuda(), kind="triangle")
    rd = torch.from_numpy(rays).cuda()
    for kind in (arbx.RAY_INTERSECT, arbx.RAY_ORDERED):
        ref = device_crs(t, kind, rd)
        for chunk in (16, 1 << 12, 0):
            same(t.query_crs_host(kind, rd, chunk_bytes=chunk), ref)
    roff, ridx, rt = oracle.ray_all(tris, rays)
    off, idx, tt = t.query_crs_host(arbx.RAY_ORDERED, rd, chunk_bytes=512)
    assert np.array_equal(off, roff) and np.array_equal(idx, ridx)
    assert np.array_equal(tt.view(np.uint32), rt.view(np.uint32))


def test_capacity_and_failures(arbx):
    rng = np.random.default_rng(9)
    pts = rng.random((20000, 3), dtype=np.float32)
    qs = rng.random((3000, 3), dtype=np.float32)
    t = arbx.Tree(torch.from_numpy(pts).cuda())
    q = torch.from_numpy(qs).cuda()
    ref = device_crs(t, arbx.SPHERE, q, 0.03)
    nnz = int(ref[0][-1])
    p, keep = t._pred(arbx.SPHERE, q, 0.03)
    off = np.empty(len(qs) + 1, np.int64)
    idx = np.empty(nnz, np.int32)
    d2 = np.empty(nnz, np.float32)
    got = ctypes.c_int64(0)
    st = arbx._lib.arbx_query_crs_host(t._h, ctypes.byref(p), 1, None, off.ctypes.data, idx.ctypes.data,
                                        d2.ctypes.data, nnz - 1, 4096, ctypes.byref(got), arbx._stream())
    assert st == arbx.ERR_CAPACITY and got.value == nnz and np.array_equal(off, ref[0])
    failed = 0
    for after in range(10):
        arbx.debug_fail_allocs(after, 1)
        try:
            st = arbx._lib.arbx_query_crs_host(t._h, ctypes.byref(p), 1, None, off.ctypes.data, idx.ctypes.data,
                                                d2.ctypes.data, nnz, 4096, None, arbx._stream())
        finally:
            arbx.debug_fail_allocs(0, 0)
        if st == arbx.OK:
            same((off, idx, d2), ref)
        else:
            assert st == arbx.ERR_OOM
            failed += 1
    assert failed > 0
    same(t.query_crs_host(arbx.SPHERE, q, 0.03, chunk_bytes=4096), ref)
    arbx.stream_check()
