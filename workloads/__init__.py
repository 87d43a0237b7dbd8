"""Seeded synthetic inputs for the five workloads of the linear-BVH search path.

This module only draws random inputs (points, query centres, radii, triangles,
rays, boxes, request streams).  It holds none of the search arithmetic: no
distances, no Morton codes, no tree.  Both the CPU oracle (through the tests)
and the CUDA path (through the tests and the benchmark) take their inputs from
here, so the two sides see identical bytes.

Every generator uses numpy's PCG64 ``default_rng`` with fixed seeds, computes in
float64 where a formula is involved and stores float32 row-major arrays, the
layout the C ABI takes (``float[n][dim]``, triangles ``float[n][3][3]``, rays
``float[m][6]`` = origin then direction, boxes ``float[m][2*dim]`` = lo then hi).

Workloads (the paper measures one cosmology dataset of about 37M points with a
radius query, Table 1 of section 2.6; that dataset is not available, and the
clustered mixture of ``large_mixture`` stands in for its shape):

* ``tiny_uniform``      16384 uniform points in [0,1)^3, 16384 queries, radius
                        for ~16 expected neighbours, kNN k=8.
* ``large_mixture``     10M points of a 64-component isotropic Gaussian mixture
                        (sigma log-uniform in [1e-3, 1e-1]), 10M queries from the
                        same mixture, radius for a mean of 32 neighbours, k=16.
* ``forest_sets``       4096 independent uniform sets in dims {2,3,6}, sizes
                        log-uniform, 0.5-2x as many queries, per-set radius for
                        ~16 neighbours, k=8.
* ``heightfield``       2048x1024-vertex fBm heightfield (4,188,162 triangles),
                        4M downward cosine-weighted rays, 4M boxes.
* ``serving_stream``    resident mixture trees of 1M-50M points and a Poisson
                        stream of mixed-size, mixed-kind requests.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "uniform_points", "MixtureModel", "mixture_model", "mixture_points",
    "tiny_uniform", "large_mixture", "subset_indices", "forest_sets",
    "ForestSet", "heightfield_triangles", "heightfield_rays", "heightfield_boxes",
    "serving_stream", "unit_ball_volume", "TINY_RADIUS", "LARGE_RADIUS",
]


def _rng(*seed: int) -> np.random.Generator:
    return np.random.default_rng(list(seed) if len(seed) > 1 else seed[0])


def uniform_points(n: int, dim: int, seed: int) -> np.ndarray:
    """``n`` points uniform in [0,1)^dim, float32, drawn directly in float32."""
    return _rng(seed).random((n, dim), dtype=np.float32)


# ---------------------------------------------------------------- mixtures

@dataclass(frozen=True)
class MixtureModel:
    means: np.ndarray   # (C, 3) float64, uniform in [0,1)^3
    sigmas: np.ndarray  # (C,) float64, log-uniform


def mixture_model(seed: int, components: int = 64,
                  sigma_lo: float = 1e-3, sigma_hi: float = 1e-1) -> MixtureModel:
    r = _rng(seed)
    means = r.random((components, 3))
    sigmas = np.exp(r.uniform(math.log(sigma_lo), math.log(sigma_hi), components))
    return MixtureModel(means, sigmas)


def mixture_points(model: MixtureModel, n: int, seed: int,
                   chunk: int = 1 << 22) -> np.ndarray:
    """``n`` float32 3D points of ``model``: equal weights, multinomial labels,
    isotropic normals, no clipping.  Generated in chunks so that 10M points do
    not need several GB of float64 temporaries."""
    r = _rng(seed)
    out = np.empty((n, 3), dtype=np.float32)
    c = len(model.sigmas)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab = r.integers(0, c, e - s)
        z = r.standard_normal((e - s, 3))
        out[s:e] = model.means[lab] + model.sigmas[lab, None] * z
    return out


# ---------------------------------------------------------------- workloads

def unit_ball_volume(d: int) -> float:
    """Volume of the unit d-ball, pi^(d/2) / Gamma(d/2 + 1)."""
    return math.pi ** (d / 2) / math.gamma(d / 2 + 1)


# Radius of the tiny uniform workload: the ball holding 16 expected points of a
# unit-density-16384 cloud, r = cbrt(3*16 / (4*pi*16384)).
TINY_RADIUS = float(np.float32((3.0 * 16.0 / (4.0 * math.pi * 16384.0)) ** (1.0 / 3.0)))

# Radius of the large mixture workload, calibrated once by
# ``oracle/calibrate_radius.py``: the smallest float32 r at which the exact mean
# neighbour count of 1000 seeded mixture queries (against all 10M points) reaches
# 32.  Stored as float32 bits so that both sides use the same value.
LARGE_RADIUS_BITS = 0x39c3d276  # r = 0.00037350104
LARGE_RADIUS = float(np.array([LARGE_RADIUS_BITS], dtype=np.uint32).view(np.float32)[0])

SEED_TINY_POINTS, SEED_TINY_QUERIES = 1001, 1002
SEED_MIX_MODEL, SEED_MIX_POINTS, SEED_MIX_QUERIES = 2001, 2002, 2003
SEED_MIX_CALIB, SEED_MIX_SUBSET = 2004, 2005


def tiny_uniform() -> dict:
    """The tiny plain workload: N = M = 16384 uniform 3D points, r for ~16
    expected neighbours, kNN k=8."""
    return dict(points=uniform_points(16384, 3, SEED_TINY_POINTS),
                queries=uniform_points(16384, 3, SEED_TINY_QUERIES),
                radius=TINY_RADIUS, k=8, dim=3)


def large_mixture(n: int = 10_000_000, m: int = 10_000_000) -> dict:
    """The large plain workload: N = M = 10M points of the 64-component
    mixture, radius for a mean of 32 neighbours, kNN k=16.  Smaller ``n``/``m``
    give prefixes of the same streams (useful for quick runs)."""
    model = mixture_model(SEED_MIX_MODEL)
    return dict(points=mixture_points(model, n, SEED_MIX_POINTS),
                queries=mixture_points(model, m, SEED_MIX_QUERIES),
                radius=LARGE_RADIUS, k=16, dim=3)


def large_mixture_calibration_queries(count: int = 1000) -> np.ndarray:
    return mixture_points(mixture_model(SEED_MIX_MODEL), count, SEED_MIX_CALIB)


def subset_indices(m: int, count: int = 10_000, seed: int = SEED_MIX_SUBSET) -> np.ndarray:
    """The seeded query subset the oracle checks at full size (sorted)."""
    count = min(count, m)
    return np.sort(_rng(seed).choice(m, count, replace=False)).astype(np.int64)


# ---------------------------------------------------------------- forest

@dataclass
class ForestSet:
    dim: int
    points: np.ndarray
    queries: np.ndarray
    radius: float
    k: int = 8


SEED_FOREST = 3001


def forest_plan(nsets: int = 4096, size_lo: float = 1e3, size_hi: float = 1e6,
                seed: int = SEED_FOREST) -> list[tuple[int, int, int]]:
    """Per set (dim, n_s, m_s): dim uniform over {2,3,6}, n_s = floor(exp(U(ln lo,
    ln hi))), m_s = floor(n_s * exp(U(ln 0.5, ln 2)))."""
    r = _rng(seed)
    dims = r.choice(np.array([2, 3, 6]), nsets)
    ns = np.floor(np.exp(r.uniform(math.log(size_lo), math.log(size_hi), nsets))).astype(np.int64)
    ms = np.floor(ns * np.exp(r.uniform(math.log(0.5), math.log(2.0), nsets))).astype(np.int64)
    return [(int(d), int(n), int(mm)) for d, n, mm in zip(dims, ns, ms)]


def forest_set(plan: list[tuple[int, int, int]], s: int, seed: int = SEED_FOREST) -> ForestSet:
    """Set ``s`` of a forest plan; its points and queries come from their own
    seeded streams, so any set can be generated without the others."""
    d, n, m = plan[s]
    pts = _rng(seed, s, 1).random((n, d), dtype=np.float32)
    qs = _rng(seed, s, 2).random((m, d), dtype=np.float32)
    # V_d r^d n = 16 expected neighbours in the unit cube (fewer near the edges)
    r = float(np.float32((16.0 / (unit_ball_volume(d) * n)) ** (1.0 / d)))
    return ForestSet(d, pts, qs, r)


def forest_sets(nsets: int = 4096, size_lo: float = 1e3, size_hi: float = 1e6,
                seed: int = SEED_FOREST) -> list[ForestSet]:
    plan = forest_plan(nsets, size_lo, size_hi, seed)
    return [forest_set(plan, s, seed) for s in range(nsets)]


# ---------------------------------------------------------------- heightfield

SEED_HF_NOISE, SEED_HF_RAYS, SEED_HF_BOXES = 4001, 4002, 4003
HF_NX, HF_NY = 2048, 1024
HF_SPACING = 1.0 / 1023.0


def _hash2(ix: np.ndarray, iy: np.ndarray, octave: int, seed: int) -> np.ndarray:
    """32-bit integer hash of a lattice point -> uniform [0,1) (float64)."""
    m = np.uint64(0xFFFFFFFF)
    h = (ix.astype(np.uint64) * np.uint64(0x9E3779B1)) & m
    h ^= (iy.astype(np.uint64) * np.uint64(0x85EBCA77)) & m
    h ^= np.uint64((octave * 0xC2B2AE3D + seed * 0x27D4EB2F) & 0xFFFFFFFF)
    h ^= h >> np.uint64(15)
    h = (h * np.uint64(0x2C1B3C6D)) & m
    h ^= h >> np.uint64(12)
    h = (h * np.uint64(0x297A2D39)) & m
    h ^= h >> np.uint64(15)
    return h.astype(np.float64) / 4294967296.0


def _value_noise(x: np.ndarray, y: np.ndarray, octave: int, seed: int) -> np.ndarray:
    x0 = np.floor(x)
    y0 = np.floor(y)
    fx, fy = x - x0, y - y0
    sx, sy = fx * fx * (3 - 2 * fx), fy * fy * (3 - 2 * fy)
    ix, iy = x0.astype(np.int64) & 0xFFFFFFFF, y0.astype(np.int64) & 0xFFFFFFFF
    v00 = _hash2(ix, iy, octave, seed)
    v10 = _hash2(ix + 1, iy, octave, seed)
    v01 = _hash2(ix, iy + 1, octave, seed)
    v11 = _hash2(ix + 1, iy + 1, octave, seed)
    a = v00 + sx * (v10 - v00)
    b = v01 + sx * (v11 - v01)
    return a + sy * (b - a)


def heightfield_vertices(nx: int = HF_NX, ny: int = HF_NY, seed: int = SEED_HF_NOISE,
                         octaves: int = 8, base_freq: float = 4.0) -> np.ndarray:
    """(ny, nx, 3) float32 grid vertices; heights = fBm of hashed value noise
    (lacunarity 2, gain 0.5), computed in float64 and scaled to z in [0, 0.2]."""
    xs = np.arange(nx, dtype=np.float64) * HF_SPACING
    ys = np.arange(ny, dtype=np.float64) * HF_SPACING
    X, Y = np.meshgrid(xs, ys)
    z = np.zeros_like(X)
    amp, freq = 1.0, base_freq
    for o in range(octaves):
        z += amp * _value_noise(X * freq, Y * freq, o, seed)
        amp *= 0.5
        freq *= 2.0
    z = (z - z.min()) / (z.max() - z.min()) * 0.2
    return np.stack([X, Y, z], axis=-1).astype(np.float32)


def heightfield_triangles(nx: int = HF_NX, ny: int = HF_NY, seed: int = SEED_HF_NOISE) -> np.ndarray:
    """(2*(nx-1)*(ny-1), 3, 3) float32 triangles; cell (i, j) gives
    (v[j,i], v[j,i+1], v[j+1,i+1]) then (v[j,i], v[j+1,i+1], v[j+1,i])."""
    V = heightfield_vertices(nx, ny, seed)
    a = V[:-1, :-1].reshape(-1, 3)
    b = V[:-1, 1:].reshape(-1, 3)
    c = V[1:, 1:].reshape(-1, 3)
    d = V[1:, :-1].reshape(-1, 3)
    t = np.empty((a.shape[0], 2, 3, 3), dtype=np.float32)
    t[:, 0, 0], t[:, 0, 1], t[:, 0, 2] = a, b, c
    t[:, 1, 0], t[:, 1, 1], t[:, 1, 2] = a, c, d
    return t.reshape(-1, 3, 3)


def heightfield_rays(m: int = 4_000_000, seed: int = SEED_HF_RAYS,
                     extent_x: float = (HF_NX - 1) * HF_SPACING,
                     extent_y: float = (HF_NY - 1) * HF_SPACING) -> np.ndarray:
    """(m, 6) float32 rays: origin (U[0,X], U[0,Y], 0.25); cosine-weighted
    downward direction by Malley's method,
    d = (sqrt(u1) cos 2 pi u2, sqrt(u1) sin 2 pi u2, -sqrt(1 - u1))."""
    r = _rng(seed)
    o = np.stack([r.uniform(0, extent_x, m), r.uniform(0, extent_y, m), np.full(m, 0.25)], 1)
    u1, u2 = r.random(m), r.random(m)
    s = np.sqrt(u1)
    d = np.stack([s * np.cos(2 * np.pi * u2), s * np.sin(2 * np.pi * u2), -np.sqrt(1 - u1)], 1)
    return np.concatenate([o, d], 1).astype(np.float32)


def heightfield_boxes(m: int = 4_000_000, seed: int = SEED_HF_BOXES,
                      extent_x: float = (HF_NX - 1) * HF_SPACING,
                      extent_y: float = (HF_NY - 1) * HF_SPACING) -> np.ndarray:
    """(m, 6) float32 query boxes (lo xyz, hi xyz): centre uniform over the
    domain x [0, 0.2], half-extent per axis exp(U(ln 0.5, ln 8)) / 1023."""
    r = _rng(seed)
    c = np.stack([r.uniform(0, extent_x, m), r.uniform(0, extent_y, m), r.uniform(0, 0.2, m)], 1)
    h = np.exp(r.uniform(math.log(0.5), math.log(8.0), (m, 3))) * HF_SPACING
    return np.concatenate([c - h, c + h], 1).astype(np.float32)


# ---------------------------------------------------------------- layered scene

SEED_LAYERS = 4101


def layered_triangles(layers: int = 64, duplicate_layer: int = 7) -> np.ndarray:
    """(2 * (layers + 1), 3, 3) float32 triangles: layer i is the unit square
    at z = i / layers split along its diagonal into (0,0)-(1,0)-(1,1)
    (index 2i, covering y <= x) and (0,0)-(1,1)-(0,1) (index 2i + 1, y >= x);
    the last two triangles repeat layer `duplicate_layer` (exact duplicates)."""
    tris = []
    for i in list(range(layers)) + [duplicate_layer]:
        z = i / layers
        tris.append([[0, 0, z], [1, 0, z], [1, 1, z]])
        tris.append([[0, 0, z], [1, 1, z], [0, 1, z]])
    return np.asarray(tris, np.float32)


def layered_rays(m: int, seed: int = SEED_LAYERS, z0: float = 1.5, tilt: float = 0.0) -> np.ndarray:
    """(m, 6) float32 rays from (U[0,1), U[0,1), z0) heading down: direction
    (tilt * N(0,1), tilt * N(0,1), -1)."""
    r = _rng(seed)
    o = np.stack([r.random(m), r.random(m), np.full(m, z0)], 1)
    d = np.concatenate([tilt * r.standard_normal((m, 2)), -np.ones((m, 1))], 1)
    return np.concatenate([o, d], 1).astype(np.float32)


# ---------------------------------------------------------------- serving

SEED_RAY_STRESS = 4201


def ray_stress_scene(ntris: int = 6000, seed: int = SEED_RAY_STRESS) -> tuple[np.ndarray, np.ndarray]:
    """Triangles and rays where a float32 ray-triangle hit is closest to its
    triangle's edge of validity: (tris (ntris, 3, 3), rays (m, 6)) float32.

    Triangles, a third each: ordinary ones of size 1e-2..1 near coordinates
    ~1e3 (few float32 bits below the unit); slivers (the third vertex within
    1e-6..1e-3 of the midpoint of a 0.1..1 edge); tiny ones (size 1e-4..1e-3)
    near 1e3.  Per triangle, rays towards its three vertices, its three edge
    midpoints and its centroid, from 0.5..20 away, coming in at grazing angles
    (1e-4..1e-1 rad above the triangle's plane) or head on, plus rays lying in
    the plane through an edge midpoint (parallel)."""
    r = _rng(seed)
    third = ntris // 3
    base = 1000.0 + r.uniform(-5.0, 5.0, (ntris, 1, 3))
    v = np.empty((ntris, 3, 3))
    v[:third] = base[:third] + r.uniform(-1.0, 1.0, (third, 3, 3)) * np.exp(r.uniform(np.log(1e-2), 0.0, (third, 1, 1)))
    ns = ntris - 2 * third
    a = base[third:2 * third, 0]
    e = r.normal(size=(third, 3))
    e *= (r.uniform(0.1, 1.0, (third, 1)) / np.linalg.norm(e, axis=1, keepdims=True))
    off = r.normal(size=(third, 3))
    off -= (off * e).sum(1, keepdims=True) * e / (e * e).sum(1, keepdims=True)
    off *= np.exp(r.uniform(np.log(1e-6), np.log(1e-3), (third, 1))) / np.linalg.norm(off, axis=1, keepdims=True)
    v[third:2 * third, 0] = a
    v[third:2 * third, 1] = a + e
    v[third:2 * third, 2] = a + 0.5 * e + off
    v[2 * third:] = base[2 * third:] + r.uniform(-1.0, 1.0, (ns, 3, 3)) * np.exp(
        r.uniform(np.log(1e-4), np.log(1e-3), (ns, 1, 1)))
    tris = v.astype(np.float32)
    t64 = tris.astype(np.float64)
    targets = np.concatenate([t64, 0.5 * (t64 + np.roll(t64, -1, axis=1)), t64.mean(1, keepdims=True)], axis=1)
    nrm = np.cross(t64[:, 1] - t64[:, 0], t64[:, 2] - t64[:, 0])
    nrm /= np.maximum(np.linalg.norm(nrm, axis=1, keepdims=True), 1e-300)
    rays = []
    for j in range(targets.shape[1]):
        p = targets[:, j]
        inplane = r.normal(size=(ntris, 3))
        inplane -= (inplane * nrm).sum(1, keepdims=True) * nrm
        inplane /= np.maximum(np.linalg.norm(inplane, axis=1, keepdims=True), 1e-300)
        ang = np.where(r.random((ntris, 1)) < 0.7, np.exp(r.uniform(np.log(1e-4), np.log(1e-1), (ntris, 1))),
                       r.uniform(0.3, 1.5, (ntris, 1)))
        side = np.where(r.random((ntris, 1)) < 0.5, 1.0, -1.0)
        d = np.cos(ang) * inplane - side * np.sin(ang) * nrm      # towards the plane
        o = p - d * r.uniform(0.5, 20.0, (ntris, 1))
        rays.append(np.concatenate([o, d], 1))
    # parallel rays in the plane, through an edge midpoint
    p = targets[:, 3]
    inplane = np.cross(nrm, r.normal(size=(ntris, 3)))
    inplane /= np.maximum(np.linalg.norm(inplane, axis=1, keepdims=True), 1e-300)
    rays.append(np.concatenate([p - 3.0 * inplane, inplane], 1))
    return tris, np.concatenate(rays).astype(np.float32)


SEED_SERVE = 5001
SERVE_KINDS = ("radius", "knn1", "knn8", "knn32", "count")


@dataclass
class ServingStream:
    tree_sizes: list[int]
    tree_seeds: list[int]
    sizes: np.ndarray          # queries per request
    kinds: np.ndarray          # index into SERVE_KINDS
    trees: np.ndarray          # target tree per request
    interarrival: np.ndarray   # unit-rate exponential gaps (scale by 1/lambda)
    extra: dict = field(default_factory=dict)


def serving_stream(ntrees: int = 8, nreq: int = 20_000, tree_lo: float = 1e6,
                   tree_hi: float = 5e7, req_lo: float = 1.0, req_hi: float = 1e6,
                   seed: int = SEED_SERVE) -> ServingStream:
    r = _rng(seed)
    sizes_t = np.floor(np.exp(r.uniform(math.log(tree_lo), math.log(tree_hi), ntrees))).astype(np.int64)
    seeds_t = [int(seed * 100 + t) for t in range(ntrees)]
    sizes = np.floor(np.exp(r.uniform(math.log(req_lo), math.log(req_hi), nreq))).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    kinds = r.integers(0, len(SERVE_KINDS), nreq)
    trees = r.integers(0, ntrees, nreq)
    gaps = r.exponential(1.0, nreq)
    return ServingStream([int(x) for x in sizes_t], seeds_t, sizes, kinds, trees, gaps)


def serving_tree_points(stream: ServingStream, t: int) -> np.ndarray:
    model = mixture_model(stream.tree_seeds[t])
    return mixture_points(model, stream.tree_sizes[t], stream.tree_seeds[t] + 1)


def serving_request_queries(stream: ServingStream, req: int) -> np.ndarray:
    t = int(stream.trees[req])
    model = mixture_model(stream.tree_seeds[t])
    return mixture_points(model, int(stream.sizes[req]), SEED_SERVE * 1000 + req)
