"""The allocation-free offsets entry point against the regular one.

arbx_query_offsets_noalloc serves callers that cannot allocate device memory
while they run (device memory owned by another allocator or budget,
latency-critical paths where an allocation could synchronise the device, work
captured into a CUDA graph in a mode that forbids allocation).  It keeps its
temporaries in a fixed device array inside the library, shared by all calls.
These tests call it through the C ABI twice in a row, with different inputs,
and require exactly the offsets that arbx_query_offsets (which allocates its
temporaries) produces -- the second call must not see anything left behind by
the first.  The file is named to be collected last so that a run stopping at
its first failure has run every other test before it.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arbx():
    import paper_2507_23700_b300 as m
    return m


def _pred(arbx, kind, data, dim, radius=0.0):
    return arbx.arbx_predicates(kind, dim, data.shape[0], data.data_ptr() if data.shape[0] else None, None,
                                float(radius), 0)


def _regular_offsets(arbx, tree, pred):
    off = torch.empty(pred.m + 1, dtype=torch.int64, device="cuda")
    st = arbx._stream()
    assert arbx._lib.arbx_query_offsets(tree._h, ctypes.byref(pred), None, off.data_ptr(), st) == arbx.OK
    return off


def _noalloc_offsets(arbx, tree, pred):
    off = torch.full((pred.m + 1,), -7, dtype=torch.int64, device="cuda")
    err = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    st = arbx._stream()
    # every device allocation the library attempts from here on fails: a call
    # that allocated anything would return ARBX_ERR_OOM instead of OK
    arbx.debug_fail_allocs(0, 1 << 30)
    try:
        status = arbx._lib.arbx_query_offsets_noalloc(tree._h, ctypes.byref(pred), off.data_ptr(), err.data_ptr(),
                                                      st)
    finally:
        arbx.debug_fail_allocs(0, 0)
    assert status == arbx.OK, status
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return off


def test_noalloc_offsets_match_regular_twice(arbx):
    wl = workloads.tiny_uniform()
    pts = torch.from_numpy(wl["points"]).cuda()
    tree = arbx.Tree(pts)
    qa = torch.from_numpy(wl["queries"]).cuda()
    qb = torch.from_numpy(np.random.default_rng(77).random((5001, 3), dtype=np.float32)).cuda()
    pa = _pred(arbx, arbx.SPHERE, qa, 3, wl["radius"])
    pb = _pred(arbx, arbx.SPHERE, qb, 3, 1.5 * wl["radius"])
    ref_a = _regular_offsets(arbx, tree, pa)
    ref_b = _regular_offsets(arbx, tree, pb)
    got_a = _noalloc_offsets(arbx, tree, pa)   # first call (sets up the scratch address on first use)
    got_b = _noalloc_offsets(arbx, tree, pb)   # second call, different size and radius
    assert torch.equal(got_a, ref_a)
    assert torch.equal(got_b, ref_b)
    assert int(got_a[-1]) > 0 and int(got_b[-1]) > 0


def test_noalloc_box_predicate_and_limits(arbx):
    rng = np.random.default_rng(3)
    pts = torch.from_numpy(rng.random((20000, 2), dtype=np.float32)).cuda()
    tree = arbx.Tree(pts)
    c = rng.random((3000, 2), dtype=np.float32)
    h = np.float32(0.01)
    boxes = torch.from_numpy(np.concatenate([c - h, c + h], 1)).cuda()
    p = _pred(arbx, arbx.BOX_PRED, boxes, 2)
    ref = _regular_offsets(arbx, tree, p)
    assert torch.equal(_noalloc_offsets(arbx, tree, p), ref)
    assert torch.equal(_noalloc_offsets(arbx, tree, p), ref)
    # more queries than the fixed array holds: refused before any device work
    big = arbx.arbx_predicates(arbx.BOX_PRED, 2, (1 << 20) + 1, boxes.data_ptr(), None, 0.0, 0)
    off = torch.empty(2, dtype=torch.int64, device="cuda")
    st = arbx._stream()
    assert arbx._lib.arbx_query_offsets_noalloc(tree._h, ctypes.byref(big), off.data_ptr(), None, st) == \
        arbx.ERR_CAPACITY


@pytest.mark.parametrize("quantized", [True, "parent"])
def test_noalloc_quantized_tree(arbx, quantized):
    """Box predicates on a tree of 16-bit nodes (either form) give the regular
    offsets; a sphere predicate there is refused before any device work."""
    tris = workloads.heightfield_triangles(65, 33, seed=21)
    tree = arbx.Tree(torch.from_numpy(tris).cuda(), kind="triangle", quantized=quantized)
    rng = np.random.default_rng(5)
    c = np.concatenate([rng.random((4000, 2), dtype=np.float32) * np.float32(64 * workloads.HF_SPACING),
                        rng.random((4000, 1), dtype=np.float32) * np.float32(0.2)], 1).astype(np.float32)
    h = np.float32(2 * workloads.HF_SPACING)
    boxes = torch.from_numpy(np.concatenate([c - h, c + h], 1)).cuda()
    p = _pred(arbx, arbx.BOX_PRED, boxes, 3)
    ref = _regular_offsets(arbx, tree, p)
    assert torch.equal(_noalloc_offsets(arbx, tree, p), ref)
    assert torch.equal(_noalloc_offsets(arbx, tree, p), ref)
    assert int(ref[-1]) > 0
    sph = _pred(arbx, arbx.SPHERE, c_t := torch.from_numpy(c).cuda(), 3, 0.01)
    off = torch.empty(c_t.shape[0] + 1, dtype=torch.int64, device="cuda")
    assert arbx._lib.arbx_query_offsets_noalloc(tree._h, ctypes.byref(sph), off.data_ptr(), None,
                                                arbx._stream()) == arbx.ERR_UNSUPPORTED
