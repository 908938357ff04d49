"""Oracle: a two-level multigrid preconditioner for the CG solves of
eq. pressure_final and eq. ad5 (an extension, as the block-Jacobi PCG is: the
paper runs CG unpreconditioned, and its iteration counts grow like 1/h).

Method (textbook algebraic multigrid; Saad, Iterative Methods for Sparse
Linear Systems, 2nd ed., Ch. 13; smoothed aggregation after Vanek, Mandel and
Brezina, Computing 56 (1996)):

  Fine level: the DG pressure space of degree p, smoothed by damped block
  Jacobi, x += omega_f D^-1 (r - A x), D = blockdiag of the N_phi x N_phi
  diagonal blocks of A, omega_f = 0.7.  A is a sum over edges of PSD
  two-block terms, each bounded by twice its block diagonal, so
  lambda_max(D^-1 A) <= 2 and omega_f lambda_max < 2 (the smoother
  contracts and the preconditioner is symmetric positive definite).

  Coarse space: continuous piecewise-linear functions on the mesh vertices.
  Vertex numbering: first appearance, scanning the triangles in reverse
  Cuthill-McKee order and their vertices v0, v1, v2.  Prolongation Pc
  (n x n_v): row (triangle t, node k) holds the barycentric coordinates
  lambda_m(xi_k) of node k at the columns of t's vertices (nodal
  interpolation of a linear function, exact; constants reproduced).
  A_0 = Pc^T A Pc (Galerkin), on the combinatorial pattern {(u, w): u a vertex
  of triangle t, w a vertex of t or of a triangle sharing an edge with t}.

  A_0 is solved approximately by one V(1,1)-cycle of smoothed aggregation:
   - aggregation on a graph only (no values): pass 1 visits the DOFs in
     order and makes every DOF whose closed neighbourhood is still free the
     root of a new aggregate (the root and its neighbours); pass 2 visits the
     DOFs again and puts each free DOF into the aggregate of its first
     (lowest-numbered) aggregated neighbour, or into a new aggregate of its
     own if it has none.  The graph of the vertex level joins the vertices of
     every triangle (the mesh edges); the graph of the next level joins two
     aggregates that hold adjacent DOFs (the pattern of T^T G T).  (The
     operator's own pattern also reaches the vertices of neighbouring
     triangles, and aggregates built on it coarsen too fast for one
     Jacobi-smoothed prolongation: the V-cycle then degrades with the mesh.)
   - tentative prolongation T (n x n_agg): T[i, agg(i)] = 1;
   - smoothed prolongation P = T - omega_P D^-1 A T, D = diag(A),
     omega_P = (4/3) / lambda_G with the Gershgorin bound
     lambda_G = max_i sum_j |a_ij| / a_ii >= lambda_max(D^-1 A);
   - next level A' = P^T A P, its pattern the boolean product of the patterns
     of P^T, A and P (entries that cancel are kept as explicit zeros);
   - until at most 256 DOFs remain (or an aggregation step removes fewer than
     20% of them), then a dense solve: the pseudo-inverse for the pressure
     operator (nullspace span{1}, removed explicitly from the
     eigendecomposition; every coarse right-hand side has zero sum because
     each prolongation reproduces constants), the inverse otherwise;
   - damped Jacobi smoothing with weights omega_J / a_ii,
     omega_J = (4/3) / lambda_G.

  One application z = M r:
    x1 = omega_f D^-1 r
    x2 = x1 + Pc V(Pc^T (r - A x1))
    z  = x2 + omega_f D^-1 (r - A x2)
  (symmetric: the same smoother before and after the coarse correction).

Vectors in the natural triangle numbering (triangle i, local DOF k at
i * N_phi + k); A is the oracle's sparse Schur or Helmholtz matrix.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import basis as B
from . import mesh as OM
from .operators import apply_blocks, block_jacobi_blocks

OMEGA_F = 0.7
COARSEST = 256


def vertex_numbering(conn: OM.Connectivity, tri):
    """cvid[t] (natural triangle t): coarse DOF of each of its 3 vertices,
    numbered by first appearance over the triangles in RCM order."""
    perm = OM.rcm_order(conn)
    tri = np.asarray(tri)
    cvid = np.full(tri.shape, -1, dtype=np.int64)
    ids = {}
    for t in perm:
        for m in range(3):
            v = int(tri[t, m])
            if v not in ids:
                ids[v] = len(ids)
            cvid[t, m] = ids[v]
    return cvid, len(ids)


def p1_prolongation(cvid, nv, p):
    """Pc (n x nv): nodal interpolation of the vertex values of a continuous
    piecewise-linear function at the N_phi nodes of every triangle."""
    X = B.nodes(p)
    lam = np.stack([1.0 - X[:, 0] - X[:, 1], X[:, 0], X[:, 1]], axis=1)   # [nphi, 3]
    ne, nphi = cvid.shape[0], X.shape[0]
    rows = np.repeat(np.arange(ne * nphi), 3)
    cols = np.repeat(cvid[:, None, :], nphi, axis=1).ravel()
    vals = np.tile(lam[None], (ne, 1, 1)).ravel()
    return sp.csr_matrix((vals, (rows, cols)), shape=(ne * nphi, nv))


def vertex_graph(cvid, nv):
    """Boolean graph of the vertex level: the vertices of each triangle are
    pairwise adjacent (the mesh edges), with the diagonal."""
    r = np.repeat(cvid, 3, axis=1).ravel()
    c = np.tile(cvid, (1, 3)).ravel()
    G = sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(nv, nv))
    G.data[:] = 1.0
    G.sort_indices()
    return G


def coarse_pattern(conn: OM.Connectivity, cvid, nv):
    """Boolean pattern of A_0: vertices of t against vertices of t and of
    its three edge neighbours."""
    nb = OM.neighbours(conn)
    rows, cols = [], []
    for t in range(conn.n_tri):
        for u in (t, *nb[t]):
            for m in range(3):
                rows.extend([cvid[t, m]] * 3)
                cols.extend(cvid[u])
    S = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(nv, nv))
    S.data[:] = 1.0
    S.sort_indices()
    return S


def on_pattern(M, pattern):
    """The values of M at the entries of `pattern` (explicit zeros where M has
    none), as a CSR matrix with pattern's structure."""
    pat = sp.csr_matrix(pattern)
    pat.sort_indices()
    Mc = sp.coo_matrix(M)
    ncol = pat.shape[1]
    keys_m = Mc.row.astype(np.int64) * ncol + Mc.col
    order = np.argsort(keys_m)
    keys_m, vals_m = keys_m[order], Mc.data[order]
    rows = np.repeat(np.arange(pat.shape[0], dtype=np.int64), np.diff(pat.indptr))
    keys_p = rows * ncol + pat.indices
    pos = np.searchsorted(keys_m, keys_p)
    pos_c = np.minimum(pos, max(len(keys_m) - 1, 0))
    hit = (pos < len(keys_m)) & (keys_m[pos_c] == keys_p) if len(keys_m) else np.zeros(len(keys_p), bool)
    data = np.where(hit, vals_m[pos_c] if len(keys_m) else 0.0, 0.0)
    if not np.all(np.isin(keys_m, keys_p)):
        raise ValueError("M has entries outside the pattern")
    return sp.csr_matrix((data, pat.indices.copy(), pat.indptr.copy()), shape=pat.shape)


def aggregate(pattern):
    """Greedy two-pass aggregation on a boolean CSR pattern (sorted rows)."""
    S = sp.csr_matrix(pattern)
    S.sort_indices()
    n = S.shape[0]
    agg = -np.ones(n, dtype=np.int64)
    na = 0
    for i in range(n):
        nbr = S.indices[S.indptr[i]:S.indptr[i + 1]]
        if agg[i] < 0 and np.all(agg[nbr] < 0):
            agg[nbr] = na
            agg[i] = na
            na += 1
    for i in range(n):
        if agg[i] >= 0:
            continue
        nbr = S.indices[S.indptr[i]:S.indptr[i + 1]]
        got = [a for a in agg[nbr] if a >= 0]
        if got:
            agg[i] = got[0]
        else:
            agg[i] = na
            na += 1
    return agg, na


def gershgorin(A):
    A = sp.csr_matrix(A)
    return float(np.max(abs(A) @ np.ones(A.shape[0]) / A.diagonal()))


class Level:
    def __init__(self, A, pattern):
        self.A = sp.csr_matrix(A)
        self.pattern = pattern
        self.lam = gershgorin(self.A)
        self.wd = (4.0 / 3.0) / self.lam / self.A.diagonal()
        self.agg = None
        self.P = None


def boolean(M):
    B = (sp.csr_matrix(M) != 0).astype(np.float64)
    B.sort_indices()
    return B


def sa_hierarchy(A0, pattern0, graph0, singular):
    """Smoothed-aggregation levels from the coarse operator A0 (CSR on its
    pattern), aggregated on graph0 and the graphs derived from it, down to a
    dense coarsest solve."""
    levels = [Level(A0, pattern0)]
    G = graph0
    while levels[-1].A.shape[0] > COARSEST:
        L = levels[-1]
        n = L.A.shape[0]
        agg, na = aggregate(G)
        if na > 0.8 * n:
            break
        T = sp.csr_matrix((np.ones(n), (np.arange(n), agg)), shape=(n, na))
        omega = (4.0 / 3.0) / L.lam
        Ppat = boolean(T + L.pattern @ T)
        P = on_pattern(T - omega * sp.diags(1.0 / L.A.diagonal()) @ (L.A @ T), Ppat)
        L.agg, L.P = agg, P
        pat = boolean(Ppat.T @ L.pattern @ Ppat)
        levels.append(Level(on_pattern(P.T @ L.A @ P, pat), pat))
        G = boolean(T.T @ G @ T)
    Ac = levels[-1].A.toarray()
    if singular:
        # pseudo-inverse with the known one-dimensional kernel removed
        # explicitly: the kernel's eigenvalue is zero only to rounding, and a
        # relative cut-off could invert it
        w, Q = np.linalg.eigh(0.5 * (Ac + Ac.T))
        k = int(np.argmin(np.abs(w)))
        keep = np.arange(len(w)) != k
        levels[-1].C = (Q[:, keep] / w[keep]) @ Q[:, keep].T
    else:
        levels[-1].C = np.linalg.inv(Ac)
    return levels


def vcycle(levels, b, l=0):
    L = levels[l]
    if L.P is None:
        return L.C @ b
    x = L.wd * b
    x = x + L.P @ vcycle(levels, L.P.T @ (b - L.A @ x), l + 1)
    return x + L.wd * (b - L.A @ x)


class TwoLevel:
    """The preconditioner M of the module docstring for the sparse matrix A
    (natural numbering) of a mesh and degree."""

    def __init__(self, A, conn, tri, p, singular):
        from . import basis
        self.A = sp.csr_matrix(A)
        self.nphi = basis.n_phi(p)
        self.singular = singular
        self.cvid, self.nv = vertex_numbering(conn, tri)
        self.Pc = p1_prolongation(self.cvid, self.nv, p)
        pat = coarse_pattern(conn, self.cvid, self.nv)
        A0 = on_pattern(self.Pc.T @ self.A @ self.Pc, pat)
        self.levels = sa_hierarchy(A0, pat, vertex_graph(self.cvid, self.nv), singular)
        self.Dinv = block_jacobi_blocks(self.A, self.nphi)

    def __call__(self, r):
        A, w = self.A, OMEGA_F
        x1 = w * apply_blocks(self.Dinv, r)
        x2 = x1 + self.Pc @ vcycle(self.levels, self.Pc.T @ (r - A @ x1))
        return x2 + w * apply_blocks(self.Dinv, r - A @ x2)
