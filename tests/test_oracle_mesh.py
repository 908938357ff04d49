"""Pins of the oracle's connectivity and orderings (Sec. 2.1) by invariants
and brute force."""
import os

import numpy as np
import pytest

from oracle import mesh as OM
from oracle.assemble import sigma
from paper_2401_17806_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_sigma_golden():
    for line in open(os.path.join(GOLD, "sigma.txt")):
        if line.strip() and not line.startswith("#"):
            i, l, r, s = [int(v) for v in line.split()]
            assert sigma(i, l, r) == s


@pytest.mark.parametrize("N,seed", [(3, 0), (4, 1), (7, 2), (16, 3)])
def test_connectivity_invariants(N, seed):
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    c = OM.connectivity(xy, tri, per)
    assert c.n_tri == 2 * N * N and c.n_edge == 3 * N * N
    # Euler characteristic of the torus: V - E + F = 0
    assert N * N - c.n_edge + c.n_tri == 0
    # every triangle has three distinct edges; each edge is on exactly 2
    assert np.all(np.sort(c.tri_edge, 1)[:, 1:] != np.sort(c.tri_edge, 1)[:, :-1])
    counts = np.bincount(c.tri_edge.ravel(), minlength=c.n_edge)
    assert np.all(counts == 2)
    # brute force: edge j's vertex pair appears in l at loc_l and reversed in r
    for j in range(0, c.n_edge, max(1, c.n_edge // 50)):
        l, r = c.lr[j]
        kl, kr = c.loc[j]
        assert (tri[l, kl], tri[l, (kl + 1) % 3]) == tuple(c.edge_vtx[j])
        assert (tri[r, (kr + 1) % 3], tri[r, kr]) == tuple(c.edge_vtx[j])
        assert l < r                      # first encounter is the lower id
    # normal points from l towards r: centroid of r (moved to l's frame) is on +n
    X1 = c.tri_xy[c.lr[:, 0], c.loc[:, 0].astype(int)]
    X2 = c.tri_xy[c.lr[:, 0], (c.loc[:, 0].astype(int) + 1) % 3]
    d = X2 - X1
    n = np.stack([d[:, 1], -d[:, 0]], 1)
    br = c.tri_xy[c.lr[:, 1]].mean(1) + c.shift * per
    bl = c.tri_xy[c.lr[:, 0]].mean(1)
    assert np.all(((br - X1) * n).sum(1) > 0)
    assert np.all(((bl - X1) * n).sum(1) < 0)


def test_too_coarse_periodic_mesh_rejected():
    xy, tri, per = synth.jittered_periodic_mesh(2, 0)
    with pytest.raises(OM.MeshError):
        OM.connectivity(xy, tri, per)


def test_inverted_triangle_rejected():
    xy, tri, per = synth.jittered_periodic_mesh(4, 0)
    tri = tri.copy()
    tri[5] = tri[5][::-1]
    with pytest.raises(OM.MeshError):
        OM.connectivity(xy, tri, per)


@pytest.mark.parametrize("N,seed", [(3, 0), (8, 5), (16, 3)])
def test_rcm_and_colouring_valid(N, seed):
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    c = OM.connectivity(xy, tri, per)
    perm = OM.rcm_order(c)
    assert sorted(perm.tolist()) == list(range(c.n_tri))
    colour, eperm, offs = OM.colouring(c, perm)
    assert sorted(eperm.tolist()) == list(range(c.n_edge))
    assert colour.max() + 1 <= 5
    # no two edges of one triangle share a colour
    assert np.all(np.sort(colour[c.tri_edge], 1)[:, 1:] != np.sort(colour[c.tri_edge], 1)[:, :-1])
    assert offs[-1] == c.n_edge
    assert np.all(colour[eperm] == np.repeat(np.arange(len(offs) - 1), np.diff(offs)))


def test_rcm_reduces_bandwidth():
    xy, tri, per = synth.jittered_periodic_mesh(16, 3)
    c = OM.connectivity(xy, tri, per)
    perm = OM.rcm_order(c)
    rank = np.empty_like(perm)
    rank[perm] = np.arange(len(perm))
    bw_nat = np.abs(c.lr[:, 0] - c.lr[:, 1]).max()
    bw_rcm = np.abs(rank[c.lr[:, 0]] - rank[c.lr[:, 1]]).max()
    assert bw_rcm <= bw_nat
