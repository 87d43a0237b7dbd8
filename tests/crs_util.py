"""Comparison helpers for CRS results (used by the GPU parity tests)."""
from __future__ import annotations

import numpy as np


def to_np(x):
    if x is None:
        return None
    try:
        return x.detach().cpu().numpy()
    except AttributeError:
        return np.asarray(x)


def canonical(offsets, indices, d2=None):
    """Sort each query's segment by primitive index; return (offsets, idx, d2)."""
    off = to_np(offsets).astype(np.int64)
    idx = to_np(indices).astype(np.int64)
    seg = np.repeat(np.arange(len(off) - 1), np.diff(off))
    order = np.lexsort((idx, seg))
    d = None if d2 is None else to_np(d2)[order]
    return off, idx[order], d


def assert_crs_equal(gpu, ref, check_d2=True, what=""):
    """GPU CRS equals the oracle CRS as sets per query, with bit-identical d2."""
    goff, gidx, gd2 = canonical(*gpu)
    roff, ridx, rd2 = canonical(*ref)
    assert len(goff) == len(roff), what
    if not np.array_equal(goff, roff):
        bad = np.nonzero(np.diff(goff) != np.diff(roff))[0]
        raise AssertionError(f"{what}: counts differ for {len(bad)} queries, first {bad[:5].tolist()}: "
                             f"gpu {np.diff(goff)[bad[:5]].tolist()} oracle {np.diff(roff)[bad[:5]].tolist()}")
    assert np.array_equal(gidx, ridx), f"{what}: neighbour sets differ"
    if check_d2 and rd2 is not None:
        assert gd2 is not None, what
        assert np.array_equal(gd2.view(np.uint32), rd2.view(np.uint32)), f"{what}: d2 bits differ"


def assert_leaf_order_valid(offsets, indices):
    """Every segment holds distinct indices."""
    off = to_np(offsets)
    idx = to_np(indices)
    for i in range(0, len(off) - 1, max(1, (len(off) - 1) // 200)):
        seg = idx[off[i]:off[i + 1]]
        assert len(np.unique(seg)) == len(seg)
