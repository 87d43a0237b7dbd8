"""Ray culling where it is closest to wrong: the traversal culls against
padded boxes (a float32 Moller-Trumbore hit can lie a little outside the exact
triangle), so every hit the oracle finds must survive the culling.

The scene (workloads.ray_stress_scene) puts triangles near coordinates 1e3 --
ordinary ones, slivers whose third vertex lies 1e-6..1e-3 off an edge, and
tiny ones -- and aims rays at their vertices, edge midpoints and centroids
from grazing angles (1e-4..1e-1 rad above the plane) or head on, plus rays
lying in a triangle's plane.  With float32 and 16-bit nodes, all hits in
(t, index) order, the nearest hit and the first four hits equal the oracle's
bit for bit, translated by +-512 too.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import workloads
from crs_util import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arbx():
    import paper_2507_23700_b300 as m
    return m


@pytest.fixture(scope="module")
def scene():
    return workloads.ray_stress_scene()


@pytest.mark.parametrize("quantized", [False, True, "parent"])
@pytest.mark.parametrize("shift", [0.0, 512.0, -512.0])
def test_stress_rays_equal_oracle(arbx, scene, quantized, shift):
    tris, rays = scene
    tris = (tris + np.float32(shift)).astype(np.float32)
    rays = rays.copy()
    rays[:, :3] = (rays[:, :3] + np.float32(shift)).astype(np.float32)
    t = arbx.Tree(torch.from_numpy(tris).cuda(), kind="triangle", quantized=quantized)
    rd = torch.from_numpy(rays).cuda()
    roff, ridx, rt = oracle.ray_all(tris, rays)
    assert roff[-1] > 10000  # the scene does hit
    off, idx, tt = t.ray_intersect(rd, ordered=True)
    assert np.array_equal(to_np(off), roff)
    assert np.array_equal(to_np(idx), ridx)
    assert np.array_equal(to_np(tt).view(np.uint32), rt.view(np.uint32))
    hit, th = t.ray_nearest(rd)
    nh, nt = oracle.ray_nearest(tris, rays)
    assert np.array_equal(to_np(hit), nh)
    assert np.array_equal(to_np(th).view(np.uint32), nt.view(np.uint32))
    hk, tk = t.ray_nearest(rd, k=4)
    hk, tk = to_np(hk), to_np(tk)
    for i in np.flatnonzero(np.diff(roff) > 0)[:2000]:
        n = min(4, int(roff[i + 1] - roff[i]))
        assert np.array_equal(hk[i, :n], ridx[roff[i]:roff[i] + n]), i
        assert np.array_equal(tk[i, :n].view(np.uint32), rt[roff[i]:roff[i] + n].view(np.uint32)), i
