"""Oracle: load vectors, L2 errors and nodal positions (Sec. 2.2-2.3).

  load_vector:  b_{i,k} = int_{T_i} phi_k f             (main grid)
  dual_load:    b_{j,k} = int_{R_j} psi_k f             (dual grid)
  l2_error:     sqrt(sum_i int_{T_i} (p_h - p_ex)^2)
  main_nodes:   physical position of nodal DOF (i, k): image of node k of
                T_ref under eq. linmap for triangle i (its own frame)
  dual_nodes:   physical position of dual DOF (j, k): left half nodes are
                images under (b_l, X1, X2), right-only nodes under
                (b_r, X2, X1) moved into l's frame by the periodic shift.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import basis as B
from .assemble import _sub_triangles


def _tri_rule(conn, p, nq=None):
    nq = nq or p + 3
    rpts, rw = B.duffy_rule(nq)
    P = conn.tri_xy
    e1 = P[:, 1] - P[:, 0]
    e2 = P[:, 2] - P[:, 0]
    area2 = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    xq = B.triangle_points(P, rpts)
    return P, xq, rw[None, :] * area2[:, None]


def load_vector(conn, p, f, nq=None):
    """f: callable f(x, y) -> values.  Quadrature with p+3 points/direction
    by default (the integrand is not a polynomial)."""
    P, xq, w = _tri_rule(conn, p, nq or p + 4)
    phi = B.eval_phi(p, B.pull_back(P, xq))
    fv = f(xq[..., 0], xq[..., 1])
    return np.einsum("eq,eqk,eq->ek", w, phi, fv).ravel()


def l2_error(conn, p, x, fexact, nq=None):
    P, xq, w = _tri_rule(conn, p, nq or p + 4)
    phi = B.eval_phi(p, B.pull_back(P, xq))
    ph = np.einsum("eqk,ek->eq", phi, x.reshape(conn.n_tri, -1))
    ex = fexact(xq[..., 0], xq[..., 1])
    return np.sqrt(np.sum(w * (ph - ex) ** 2))


def integral(conn, p, x):
    """int_Omega p_h for a main-grid coefficient vector."""
    P, xq, w = _tri_rule(conn, p)
    phi = B.eval_phi(p, B.pull_back(P, xq))
    return float(np.einsum("eq,eqk,ek->", w, phi, x.reshape(conn.n_tri, -1)))


def main_nodes(conn, p):
    return B.triangle_points(conn.tri_xy, B.nodes(p))       # [Ne, Nphi, 2]


def dual_nodes(conn, p, period=(1.0, 1.0)):
    L, R = B.dual_maps(p)
    nd = conn.n_edge
    idx = np.arange(nd)
    _, _, _, _, Tl, Tr, _, _ = _sub_triangles(conn, idx)
    ref = B.nodes(p)
    out = np.zeros((nd, B.n_psi(p), 2))
    out[:, L] = B.triangle_points(Tl, ref)
    right = B.triangle_points(Tr, ref) + (conn.shift.astype(np.float64)
                                          * np.asarray(period))[:, None, :]
    own = R >= B.n_phi(p)
    out[:, R[own]] = right[:, own]
    return out


def dual_load(conn, p, f, nq=None):
    """int_{R_j} psi_k f, f(x, y) evaluated in l's frame."""
    L, R = B.dual_maps(p)
    nq = nq or p + 4
    rpts, rw = B.duffy_rule(nq)
    idx = np.arange(conn.n_edge)
    _, _, _, _, Tl, Tr, _, _ = _sub_triangles(conn, idx)
    out = np.zeros((conn.n_edge, B.n_psi(p)))
    for Tsub, perm in ((Tl, L), (Tr, R)):
        s1 = Tsub[:, 1] - Tsub[:, 0]
        s2 = Tsub[:, 2] - Tsub[:, 0]
        a = s1[:, 0] * s2[:, 1] - s1[:, 1] * s2[:, 0]
        xs = B.triangle_points(Tsub, rpts)
        ps = B.eval_phi(p, B.pull_back(Tsub, xs))
        fv = f(xs[..., 0], xs[..., 1])
        out[:, perm] += np.einsum("eq,eqk,eq->ek", rw[None, :] * a[:, None], ps, fv)
    return out
