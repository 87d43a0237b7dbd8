"""CPU oracle for the linear-BVH search path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` import this package.  The product package never does, and
it has no CPU fallback.

The arithmetic lives in ``brute.cpp`` (plain all-pairs brute force, built with
``-ffp-contract=off`` and no fast-math, so every float operation is one IEEE
binary32 round-to-nearest operation).  This module only builds and loads it and
marshals numpy arrays.  Results:

* ``radius(points, queries, r)`` -> (offsets int64[m+1], indices int32[nnz], d2 float32[nnz]),
  indices ascending within each query (ArborX 2.0, section 2.1, the CRS form).
* ``knn(points, queries, k)`` -> (indices int32[m, min(k,n)], d2 float32[m, min(k,n)]),
  ascending by (d2, index) (section 2.1, nearest predicates).
* ``box_query(prims, kind, boxes)`` -> (offsets, indices) (section 2.1, intersects(Box)).
* ``ray_nearest(tris, rays)`` -> (hit int32[m], t float32[m]) (section 2.5, nearest k=1).
* ``radius_count_up_to`` (section 2.2, the count-up-to-N callback).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_DIR = Path(__file__).resolve().parent
_SRC = _DIR / "brute.cpp"
_LIB = _DIR / "_liboracle.so"
_lib = None

POINT, TRIANGLE = 0, 2

CXXFLAGS = ["-O3", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-pthread"]


def build(force: bool = False) -> Path:
    """Compile ``brute.cpp`` into ``_liboracle.so`` (skipped when up to date)."""
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
        subprocess.run(["g++", *CXXFLAGS, str(_SRC), "-o", str(tmp)], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(str(_LIB))
        P, I64, I32, F, INT = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                               ctypes.c_float, ctypes.c_int)
        sig = {
            "oracle_abi_version": ([], INT),
            "oracle_sq_dist": ([P, P, INT], F),
            "oracle_moller_trumbore": ([P, P, P], INT),
            "oracle_radius_count": ([P, I64, P, I64, INT, P, F, P, INT], None),
            "oracle_radius_fill": ([P, I64, P, I64, INT, P, F, P, P, P, INT], None),
            "oracle_radius_count_up_to": ([P, I64, P, I64, INT, P, F, I32, P, INT], None),
            "oracle_knn": ([P, I64, P, I64, INT, INT, P, P, INT], None),
            "oracle_box_count": ([P, I64, INT, P, I64, INT, P, INT], None),
            "oracle_box_fill": ([P, I64, INT, P, I64, INT, P, P, INT], None),
            "oracle_ray_nearest": ([P, I64, P, I64, P, P, INT], None),
            "oracle_ray_all_count": ([P, I64, P, I64, P, INT], None),
            "oracle_ray_all_fill": ([P, I64, P, I64, P, P, P, INT], None),
            "oracle_dbscan": ([P, I64, INT, F, I32, P, INT], I64),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


def _f32(a, cols=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if cols is not None:
        a = a.reshape(-1, cols)
    return a


def _p(a):
    return None if a is None else a.ctypes.data


def _radii(radius, m):
    if np.ndim(radius) == 0:
        return None, float(radius)
    r = np.ascontiguousarray(radius, dtype=np.float32)
    assert r.shape == (m,)
    return r, 0.0


def sq_dist(q, p) -> np.float32:
    q, p = _f32(q), _f32(p)
    return np.float32(_load().oracle_sq_dist(_p(q), _p(p), q.size))


def radius_count(points, queries, radius, threads: int = 0) -> np.ndarray:
    dim = np.shape(queries)[-1]
    pts, qs = _f32(points, dim), _f32(queries, dim)
    radii, r = _radii(radius, len(qs))
    out = np.empty(len(qs), np.int32)
    _load().oracle_radius_count(_p(pts), len(pts), _p(qs), len(qs), dim, _p(radii), r, _p(out), threads)
    return out


def radius(points, queries, radius, threads: int = 0):
    """CRS of the inclusive-radius predicate: (offsets, indices, d2)."""
    dim = np.shape(queries)[-1]
    pts, qs = _f32(points, dim), _f32(queries, dim)
    radii, r = _radii(radius, len(qs))
    counts = radius_count(pts, qs, radius if radii is None else radii, threads)
    offsets = np.zeros(len(qs) + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    nnz = int(offsets[-1])
    idx = np.empty(nnz, np.int32)
    d2 = np.empty(nnz, np.float32)
    _load().oracle_radius_fill(_p(pts), len(pts), _p(qs), len(qs), dim, _p(radii), r,
                               _p(offsets), _p(idx), _p(d2), threads)
    return offsets, idx, d2


def radius_count_up_to(points, queries, radius, limit: int, threads: int = 0) -> np.ndarray:
    dim = np.shape(queries)[-1]
    pts, qs = _f32(points, dim), _f32(queries, dim)
    radii, r = _radii(radius, len(qs))
    out = np.empty(len(qs), np.int32)
    _load().oracle_radius_count_up_to(_p(pts), len(pts), _p(qs), len(qs), dim, _p(radii), r,
                                      int(limit), _p(out), threads)
    return out


def knn(points, queries, k: int, threads: int = 0):
    """(indices, d2), shape (m, min(k, n)), ascending by (d2, index)."""
    dim = np.shape(queries)[-1]
    pts, qs = _f32(points, dim), _f32(queries, dim)
    kk = min(int(k), len(pts))
    idx = np.empty((len(qs), kk), np.int32)
    d2 = np.empty((len(qs), kk), np.float32)
    if kk > 0:
        _load().oracle_knn(_p(pts), len(pts), _p(qs), len(qs), dim, int(k), _p(idx), _p(d2), threads)
    return idx, d2


def box_query(prims, kind: int, boxes, threads: int = 0):
    """CRS (offsets, indices) of the closed box-overlap predicate."""
    if kind == TRIANGLE:
        pr, dim = _f32(prims, 9), 3
    else:
        dim = np.shape(boxes)[-1] // 2
        pr = _f32(prims, dim)
    bx = _f32(boxes, 2 * dim)
    counts = np.empty(len(bx), np.int32)
    lib = _load()
    lib.oracle_box_count(_p(pr), len(pr), kind, _p(bx), len(bx), dim, _p(counts), threads)
    offsets = np.zeros(len(bx) + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    idx = np.empty(int(offsets[-1]), np.int32)
    lib.oracle_box_fill(_p(pr), len(pr), kind, _p(bx), len(bx), dim, _p(offsets), _p(idx), threads)
    return offsets, idx


def ray_nearest(tris, rays, threads: int = 0):
    tr, ry = _f32(tris, 9), _f32(rays, 6)
    hit = np.empty(len(ry), np.int32)
    t = np.empty(len(ry), np.float32)
    _load().oracle_ray_nearest(_p(tr), len(tr), _p(ry), len(ry), _p(hit), _p(t), threads)
    return hit, t


def dbscan(points, eps: float, min_pts: int, threads: int = 0):
    """DBSCAN labels (int32[n]: smallest core index of the cluster, -1 for
    noise; border points take their smallest adjacent cluster) and the number
    of clusters."""
    dim = np.shape(points)[-1]
    pts = _f32(points, dim)
    labels = np.empty(len(pts), np.int32)
    nc = _load().oracle_dbscan(_p(pts), len(pts), dim, float(eps), int(min_pts), _p(labels), threads)
    return labels, int(nc)


def ray_all(tris, rays, threads: int = 0):
    """Every hit of each ray, CRS ascending by (t, index)."""
    tr, ry = _f32(tris, 9), _f32(rays, 6)
    counts = np.empty(len(ry), np.int32)
    lib = _load()
    lib.oracle_ray_all_count(_p(tr), len(tr), _p(ry), len(ry), _p(counts), threads)
    offsets = np.zeros(len(ry) + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    idx = np.empty(int(offsets[-1]), np.int32)
    t = np.empty(int(offsets[-1]), np.float32)
    lib.oracle_ray_all_fill(_p(tr), len(tr), _p(ry), len(ry), _p(offsets), _p(idx), _p(t), threads)
    return offsets, idx, t


def moller_trumbore(ray6, tri9):
    r, t9 = _f32(ray6), _f32(tri9)
    t = ctypes.c_float(0.0)
    hit = _load().oracle_moller_trumbore(_p(r), _p(t9), ctypes.addressof(t))
    return bool(hit), np.float32(t.value)


def threads_used(threads: int = 0) -> int:
    return threads if threads > 0 else (os.cpu_count() or 1)
