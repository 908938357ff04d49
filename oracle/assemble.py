"""Oracle: mass, divergence, gradient and coupling blocks by quadrature in
physical coordinates (Sec. 2.3-2.4).

Every block is an integral over the physical sub-triangle T_{i,j} =
(b_i, X1, X2) or the physical edge Gamma_j, evaluated with the rules of
``oracle.basis`` at physical points; basis values come from pulling each
point back through the affine maps (eq. linmap for T_i, eq. mapDual for the
two halves of the dual quad).  The reference-operator decomposition of
Sec. 2.4 (12 reference operators) is deliberately NOT used here, so that it
remains an independent check.

Definitions followed:
  Mbar_i[k,l]       = int_{T_i} phi_k phi_l                         (eq. Mi)
  Mhat_j[k,l]       = int_{R_j} psi_k psi_l                         (eq. Mj)
  D_ij[k,l,:]       = int_{G_j} phi_k psi_l sigma_ij n_j
                      - int_{T_ij} grad(phi_k) psi_l                (eq. D)
  Q_ij[k,l,:]       = int_{T_ij} psi_k grad(phi_l)
                      - int_{G_j} psi_k phi_l sigma_ij n_j          (eq. ad5.2)
  U_ij[k,l]         = int_{T_ij} psi_k phi_l                        (eq. u)
  sigma_ij          = (r - 2 i + l) / (r - l)                       (eq. sigma)
Right half of the dual quad: the sub-triangle (b_r, X2, X1) is the image of
T_ref, i.e. the point reflection xi -> 1 - xi of the square maps X1 to (1,0)
and X2 to (0,1) on both halves (reading of eq. mapDual).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import basis as B
from .mesh import Connectivity, connectivity


def sigma(i, l, r):
    """Sign function of eq. sigma (exact in integers)."""
    return (r - 2 * i + l) / (r - l)


@dataclass
class Blocks:
    p: int
    conn: Connectivity
    area2: np.ndarray    # A_i = 2|T_i|
    Mbar: np.ndarray     # [Ne, Nphi, Nphi]
    Mhat: np.ndarray     # [Nd, Npsi, Npsi]
    D: np.ndarray        # [Nd, 2(side l,r), Nphi, Npsi, 2]
    Q: np.ndarray        # [Nd, 2(side), Npsi, Nphi, 2]
    U: np.ndarray        # [Nd, 2(side), Npsi, Nphi]
    normal: np.ndarray   # [Nd, 2]
    length: np.ndarray   # [Nd]


def _sub_triangles(conn: Connectivity, idx, local=False):
    """Vertex coordinates of T_{l,j} = (b_l, X1, X2) and T_{r,j} = (b_r, X2, X1),
    each in its own triangle's frame, plus the edge endpoints in each frame.
    local=True moves each triangle's frame so that its first vertex is the
    origin (the block integrals depend only on vertex differences)."""
    l = conn.lr[idx, 0]
    r = conn.lr[idx, 1]
    al = conn.loc[idx, 0].astype(np.int64)
    ar = conn.loc[idx, 1].astype(np.int64)
    Pl = conn.tri_xy[l]
    Pr = conn.tri_xy[r]
    if local:
        Pl = Pl - Pl[:, :1, :]
        Pr = Pr - Pr[:, :1, :]
    e = np.arange(len(idx))
    X1l = Pl[e, al]
    X2l = Pl[e, (al + 1) % 3]
    X1r = Pr[e, (ar + 1) % 3]
    X2r = Pr[e, ar]
    bl = Pl.mean(axis=1)
    br = Pr.mean(axis=1)
    Tl = np.stack([bl, X1l, X2l], axis=1)
    Tr = np.stack([br, X2r, X1r], axis=1)
    return l, r, Pl, Pr, Tl, Tr, (X1l, X2l), (X1r, X2r)


def edge_blocks(conn: Connectivity, p, idx):
    """Mhat, D, Q, U, normal, length for the edges idx (physical quadrature)."""
    nphi, npsi = B.n_phi(p), B.n_psi(p)
    L, R = B.dual_maps(p)
    nq = p + 2
    rpts, rw = B.duffy_rule(nq)           # on T_ref, sum w = 1/2
    tau, wt = B.gauss_legendre(nq)        # on [0, 1]
    ne_ = len(idx)
    Mhat = np.zeros((ne_, npsi, npsi))
    D = np.zeros((ne_, 2, nphi, npsi, 2))
    Q = np.zeros((ne_, 2, npsi, nphi, 2))
    U = np.zeros((ne_, 2, npsi, nphi))
    # every integral below is invariant under translating an element, so each
    # element is evaluated relative to its first vertex: points near the
    # element then carry no absolute-coordinate cancellation in the pull-back
    l, r, Pl, Pr, Tl, Tr, (X1l, X2l), (X1r, X2r) = _sub_triangles(conn, idx, local=True)
    d = X2l - X1l
    glen = np.hypot(d[:, 0], d[:, 1])
    n = np.stack([d[:, 1], -d[:, 0]], 1) / glen[:, None]
    for side, (Pi, Tsub, Xa, Xb, tri_id, perm) in enumerate(
            [(Pl, Tl, X1l, X2l, l, L), (Pr, Tr, X1r, X2r, r, R)]):
        sg = sigma(tri_id, l, r)                                # +1 / -1
        # volume part on the physical sub-triangle
        s1 = Tsub[:, 1] - Tsub[:, 0]
        s2 = Tsub[:, 2] - Tsub[:, 0]
        a_sub = s1[:, 0] * s2[:, 1] - s1[:, 1] * s2[:, 0]        # A_ij
        xs = B.triangle_points(Tsub, rpts)                      # [E, q, 2]
        ws = rw[None, :] * a_sub[:, None]
        psi_loc = B.eval_phi(p, B.pull_back(Tsub, xs))          # [E, q, Nphi]
        psi = np.zeros(psi_loc.shape[:2] + (npsi,))
        psi[..., perm] = psi_loc
        xi = B.pull_back(Pi, xs)
        ph = B.eval_phi(p, xi)                                  # [E, q, Nphi]
        gref = B.eval_grad_phi(p, xi)                           # [E, q, Nphi, 2]
        J = np.stack([Pi[:, 1] - Pi[:, 0], Pi[:, 2] - Pi[:, 0]], axis=-1)  # dx/dxi
        # grad_x phi = J^{-T} grad_xi phi
        JT = np.swapaxes(J, -1, -2)
        gx = np.linalg.solve(JT[:, None, None, :, :], gref[..., None])[..., 0]
        # edge part on the physical segment, parametrised X1 -> X2
        xe = Xa[:, None, :] + tau[None, :, None] * (Xb - Xa)[:, None, :]
        we = wt[None, :] * glen[:, None]
        pe_loc = B.eval_phi(p, B.pull_back(Tsub, xe))
        pe = np.zeros(pe_loc.shape[:2] + (npsi,))
        pe[..., perm] = pe_loc
        phe = B.eval_phi(p, B.pull_back(Pi, xe))
        sn = sg[:, None] * n                                    # sigma_ij n_j
        Mhat += np.einsum("eq,eqk,eql->ekl", ws, psi, psi)
        line = np.einsum("eq,eqk,eql->ekl", we, phe, pe)        # phi_k psi_l
        vol = np.einsum("eq,eqkc,eql->eklc", ws, gx, psi)       # grad phi_k psi_l
        D[:, side] = line[..., None] * sn[:, None, None, :] - vol
        lineq = np.einsum("eq,eqk,eql->ekl", we, pe, phe)       # psi_k phi_l
        volq = np.einsum("eq,eqk,eqlc->eklc", ws, psi, gx)      # psi_k grad phi_l
        Q[:, side] = volq - lineq[..., None] * sn[:, None, None, :]
        U[:, side] = np.einsum("eq,eqk,eql->ekl", ws, psi, ph)
    return Mhat, D, Q, U, n, glen


def main_mass(conn: Connectivity, p):
    """Mbar_i (eq. Mi) by physical quadrature on T_i, and A_i = 2|T_i|."""
    rpts, rw = B.duffy_rule(p + 2)
    P = conn.tri_xy - conn.tri_xy[:, :1, :]      # element-local frame (translation invariant)
    e1 = P[:, 1] - P[:, 0]
    e2 = P[:, 2] - P[:, 0]
    area2 = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    xq = B.triangle_points(P, rpts)                     # [Ne, q, 2]
    phi = B.eval_phi(p, B.pull_back(P, xq))             # [Ne, q, Nphi]
    wq = rw[None, :] * area2[:, None]                   # physical weights
    return np.einsum("eq,eqk,eql->ekl", wq, phi, phi), area2


def assemble(xy, tri, period, p, chunk=1024, conn=None) -> Blocks:
    conn = conn if conn is not None else connectivity(xy, tri, period)
    nphi, npsi = B.n_phi(p), B.n_psi(p)
    Mbar, area2 = main_mass(conn, p)
    nd = conn.n_edge
    Mhat = np.zeros((nd, npsi, npsi))
    D = np.zeros((nd, 2, nphi, npsi, 2))
    Q = np.zeros((nd, 2, npsi, nphi, 2))
    U = np.zeros((nd, 2, npsi, nphi))
    normal = np.zeros((nd, 2))
    length = np.zeros(nd)
    for s0 in range(0, nd, chunk):
        idx = np.arange(s0, min(nd, s0 + chunk))
        Mhat[idx], D[idx], Q[idx], U[idx], normal[idx], length[idx] = edge_blocks(conn, p, idx)
    return Blocks(p, conn, area2, Mbar, Mhat, D, Q, U, normal, length)
