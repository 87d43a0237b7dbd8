"""DBSCAN (section 2.4) on the GPU against the oracle's labels: every label
equal on small inputs in dims 2, 3 and 6 (clustered data with noise, minPts
from 1 to 16, duplicates, eps = 0, one point, none); on the 10M-point mixture,
a seeded sample of points checked against the oracle's neighbourhoods."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def arbx():
    import paper_2507_23700_b300 as m
    return m


def clustered(n, dim, seed, noise=0.1):
    rng = np.random.default_rng(seed)
    nc = max(2, n // 400)
    centres = rng.random((nc, dim))
    k = int(n * (1 - noise))
    pts = centres[rng.integers(0, nc, k)] + 0.02 * rng.standard_normal((k, dim))
    pts = np.concatenate([pts, rng.random((n - k, dim))]).astype(np.float32)
    return pts[rng.permutation(n)]


@pytest.mark.parametrize("dim", [2, 3, 6])
@pytest.mark.parametrize("n,eps,min_pts", [(3000, 0.02, 5), (6000, 0.03, 16), (2000, 0.01, 1), (4000, 0.015, 2)])
def test_dbscan_vs_oracle(arbx, dim, n, eps, min_pts):
    pts = clustered(n, dim, seed=n + dim)
    if dim == 6:
        eps *= 3.0
    labels, nc = arbx.dbscan(torch.from_numpy(pts).cuda(), eps, min_pts)
    r_labels, r_nc = oracle.dbscan(pts, eps, min_pts)
    assert np.array_equal(labels.cpu().numpy(), r_labels), (dim, n, eps, min_pts)
    assert nc == r_nc
    arbx.stream_check()


def test_dbscan_edge_cases(arbx):
    rng = np.random.default_rng(3)
    pts = rng.random((800, 3)).astype(np.float32)
    pts[100:140] = pts[5]
    pts[200:203] = pts[7]
    for eps, mp in ((0.0, 3), (0.0, 41), (0.0, 1), (0.05, 4)):
        labels, nc = arbx.dbscan(torch.from_numpy(pts).cuda(), eps, mp)
        r, rnc = oracle.dbscan(pts, eps, mp)
        assert np.array_equal(labels.cpu().numpy(), r) and nc == rnc, (eps, mp)
    one, nc1 = arbx.dbscan(torch.zeros((1, 2), device="cuda"), 0.1, 1)
    assert one.tolist() == [0] and nc1 == 1
    one, nc1 = arbx.dbscan(torch.zeros((1, 2), device="cuda"), 0.1, 2)
    assert one.tolist() == [-1] and nc1 == 0
    none, nc0 = arbx.dbscan(torch.zeros((0, 3), device="cuda"), 0.1, 2)
    assert none.numel() == 0 and nc0 == 0
    with pytest.raises(arbx.ArbxError):
        arbx.dbscan(torch.zeros((5, 3), device="cuda"), float("nan"), 2)


def test_dbscan_large_mixture_sample(arbx):
    """10M mixture, eps = the radius of the workload (mean 32 neighbours),
    minPts = 16: for 60 seeded points the oracle's neighbourhoods decide which
    are core; a core point shares its label with every core neighbour and its
    label is a core point labelled by itself with no larger index than its
    own; a non-core point carries the smallest label of its core neighbours,
    or -1."""
    wl = workloads.large_mixture()
    pts, eps, min_pts = wl["points"], wl["radius"], 16
    labels, nc = arbx.dbscan(torch.from_numpy(pts).cuda(), eps, min_pts)
    labels = labels.cpu().numpy()
    assert nc > 0 and (labels == -1).any()
    sample = workloads.subset_indices(len(pts), 60)
    off, idx, _ = oracle.radius(pts, pts[sample], eps)
    nbrs = np.unique(np.concatenate([idx, sample]))
    core_of = dict(zip(nbrs.tolist(), (oracle.radius_count_up_to(pts, pts[nbrs], eps, min_pts) >= min_pts).tolist()))
    for s, i in enumerate(sample):
        js = idx[off[s]:off[s + 1]]
        core_js = [j for j in js.tolist() if core_of[j]]
        if core_of[int(i)]:
            lab = labels[i]
            assert lab >= 0 and lab <= i and labels[lab] == lab
            assert all(labels[j] == lab for j in core_js)
        else:
            want = min((labels[j] for j in core_js), default=-1)
            assert labels[i] == want
