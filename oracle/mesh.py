"""Oracle: staggered mesh connectivity and orderings (Sec. 2.1).

Reading of Sec. 2.1 (left/right triangles "randomly assigned"): made
deterministic.  Local edge k of triangle t joins vertices (v_k, v_{k+1 mod 3});
edges are numbered by first encounter, scanning triangles by id and k = 0,1,2;
l(j) is the first triangle that meets edge j, r(j) the second.  The edge
nodes (X1, X2) follow l's counter-clockwise order, so the unit normal n_j,
the outward normal of l, points from l to r.

Orderings (not in the paper; needed for the GPU layout): reverse
Cuthill-McKee on the triangle adjacency graph starting at triangle 0,
neighbours queued in increasing (degree, id); greedy edge colouring over
edges sorted by (min(rcm(l), rcm(r)), max(...), id), each edge taking the
smallest colour unused by edges that share l or r; final edge order sorted by
(colour, same key).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

from collections import deque
from dataclasses import dataclass

import numpy as np


class MeshError(ValueError):
    pass


@dataclass
class Connectivity:
    n_tri: int
    n_edge: int
    edge_vtx: np.ndarray   # i32[Nd, 2]  (X1, X2) in l's CCW order
    lr: np.ndarray         # i32[Nd, 2]  (l, r)
    loc: np.ndarray        # u8[Nd, 2]   local edge index in l and in r
    shift: np.ndarray      # i8[Nd, 2]   periods to add to r's frame to reach l's
    tri_edge: np.ndarray   # i32[Ne, 3]  edge id of local edge k
    tri_xy: np.ndarray     # f64[Ne, 3, 2] unwrapped vertex coordinates


def min_image(d, period):
    return d - period * np.round(d / period)


def unwrap_triangles(xy, tri, period):
    """Vertex coordinates of each triangle in its own frame: v0 as stored,
    v1 and v2 moved to their minimum image relative to v0."""
    p0 = xy[tri[:, 0]]
    p1 = p0 + min_image(xy[tri[:, 1]] - p0, period)
    p2 = p0 + min_image(xy[tri[:, 2]] - p0, period)
    return np.stack([p0, p1, p2], axis=1)


def connectivity(xy, tri, period) -> Connectivity:
    xy = np.asarray(xy, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    period = np.asarray(period, dtype=np.float64)
    ne = tri.shape[0]
    if tri.ndim != 2 or tri.shape[1] != 3 or ne == 0:
        raise MeshError("triangle list must be [Ne, 3] and non-empty")
    if tri.min() < 0 or tri.max() >= xy.shape[0]:
        raise MeshError("vertex index out of range")
    txy = unwrap_triangles(xy, tri, period)
    e1 = txy[:, 1] - txy[:, 0]
    e2 = txy[:, 2] - txy[:, 0]
    area2 = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    if np.any(area2 <= 0):
        raise MeshError("triangle with non-positive area (not CCW or degenerate)")

    key_to_edge = {}
    edge_vtx, lr, loc = [], [], []
    tri_edge = np.full((ne, 3), -1, dtype=np.int32)
    for t in range(ne):
        for k in range(3):
            a = int(tri[t, k])
            b = int(tri[t, (k + 1) % 3])
            if a == b:
                raise MeshError("degenerate edge")
            key = (a, b) if a < b else (b, a)
            j = key_to_edge.get(key)
            if j is None:
                j = len(edge_vtx)
                key_to_edge[key] = j
                edge_vtx.append((a, b))
                lr.append([t, -1])
                loc.append([k, -1])
            else:
                if lr[j][1] != -1:
                    raise MeshError("edge shared by more than two triangles")
                if edge_vtx[j] != (b, a):
                    raise MeshError("inconsistent orientation across an edge")
                if lr[j][0] == t:
                    raise MeshError("triangle meets the same edge twice")
                lr[j][1] = t
                loc[j][1] = k
            tri_edge[t, k] = j
    lr = np.asarray(lr, dtype=np.int32)
    if np.any(lr[:, 1] < 0):
        raise MeshError("boundary edge: only periodic (closed) meshes are supported")
    loc = np.asarray(loc, dtype=np.uint8)
    edge_vtx = np.asarray(edge_vtx, dtype=np.int32)
    # periodic shift of r into l's frame, measured on X1
    l, r = lr[:, 0], lr[:, 1]
    x1_in_l = txy[l, loc[:, 0].astype(np.int64)]
    x1_in_r = txy[r, (loc[:, 1].astype(np.int64) + 1) % 3]
    shift = np.round((x1_in_l - x1_in_r) / period).astype(np.int8)
    # the other edge node must agree with the same shift
    x2_in_l = txy[l, (loc[:, 0].astype(np.int64) + 1) % 3]
    x2_in_r = txy[r, loc[:, 1].astype(np.int64)]
    if np.any(np.abs(x2_in_l - (x2_in_r + shift * period)) > 1e-9):
        raise MeshError("edge endpoints disagree across the periodic boundary")
    # a periodic mesh this small makes triangles share two edges
    nb = np.sort(np.stack([np.where(lr[tri_edge[:, k], 0] == np.arange(ne),
                                    lr[tri_edge[:, k], 1], lr[tri_edge[:, k], 0])
                           for k in range(3)], 1), axis=1)
    if np.any(nb[:, 0] == nb[:, 1]) or np.any(nb[:, 1] == nb[:, 2]):
        raise MeshError("two triangles share more than one edge (mesh too coarse)")
    return Connectivity(ne, len(edge_vtx), edge_vtx, lr, loc, shift, tri_edge, txy)


def neighbours(conn: Connectivity):
    """Neighbour triangle across each local edge, i32[Ne, 3]."""
    lr = conn.lr
    te = conn.tri_edge
    t = np.arange(conn.n_tri)[:, None]
    return np.where(lr[te, 0] == t, lr[te, 1], lr[te, 0]).astype(np.int32)


def rcm_order(conn: Connectivity) -> np.ndarray:
    """perm[new] = old triangle id (reverse Cuthill-McKee from triangle 0)."""
    nb = neighbours(conn)
    ne = conn.n_tri
    deg = np.array([len(set(nb[t].tolist())) for t in range(ne)])
    seen = np.zeros(ne, dtype=bool)
    order = []
    for start in range(ne):
        if seen[start]:
            continue
        seen[start] = True
        q = deque([start])
        while q:
            t = q.popleft()
            order.append(t)
            cand = sorted(set(int(u) for u in nb[t] if not seen[u]),
                          key=lambda u: (deg[u], u))
            for u in cand:
                seen[u] = True
                q.append(u)
    return np.asarray(order[::-1], dtype=np.int32)


def colouring(conn: Connectivity, perm: np.ndarray):
    """Greedy edge colouring; returns (colour u8[Nd], edge_perm i32[Nd],
    colour_offsets i32[c+1])."""
    rank = np.empty(conn.n_tri, dtype=np.int64)
    rank[perm] = np.arange(conn.n_tri)
    rl = rank[conn.lr[:, 0]]
    rr = rank[conn.lr[:, 1]]
    lo = np.minimum(rl, rr)
    hi = np.maximum(rl, rr)
    ids = np.arange(conn.n_edge)
    visit = sorted(range(conn.n_edge), key=lambda j: (lo[j], hi[j], j))
    colour = np.full(conn.n_edge, -1, dtype=np.int64)
    for j in visit:
        used = set()
        for t in conn.lr[j]:
            for e in conn.tri_edge[t]:
                if e != j and colour[e] >= 0:
                    used.add(int(colour[e]))
        c = 0
        while c in used:
            c += 1
        colour[j] = c
    edge_perm = np.asarray(sorted(ids.tolist(), key=lambda j: (colour[j], lo[j], hi[j], j)),
                           dtype=np.int32)
    nc = int(colour.max()) + 1
    offs = np.zeros(nc + 1, dtype=np.int32)
    for c in range(nc):
        offs[c + 1] = offs[c] + int((colour == c).sum())
    return colour.astype(np.uint8), edge_perm, offs
