"""Oracle: global operators and solves (eqs. ad5, pressure_final, d2m, m2d).

With G the global gradient (rows (c, j, k): component c of dual DOF k of
edge j; columns (i, l): DOF l of triangle i) built from the blocks Q_ij of
eq. ad5.2, and Mhat^{-1} block diagonal (dense Cholesky per edge, both
components), the left-hand side of eq. pressure_final is
    sum_j D_ij Mhat_j^{-1} (Q_lj p_l + Q_rj p_r) = -(G^T Mhat^{-1} G p)_i
because D = -Q^T.  Reading (sign): the oracle and the library expose the
symmetric positive semidefinite form
    S = dt^2 * G^T Mhat^{-1} G,
so a caller holding the paper's right-hand side negates it; and the implicit
diffusion system of eq. ad5 (lambda = nu) becomes
    H = Mbar + nu*dt * G^T Mhat^{-1} G   (SPD).
Mean-zero reading: the Schur solution is the x with sum(x) = 0 (coefficient
space), b is projected the same way.

Solves: sparse direct LU (SuperLU) of S with DOF 0 grounded, shifted to
mean zero (equal to the bordered-system solution), LU of H; a plain CG (x0 = 0, stop at ||r||/||b|| <= tol) for sizes
where a factorisation does not fit.

Preconditioned CG (an extension; the paper's CG is unpreconditioned): the
textbook PCG recurrence (Hestenes-Stiefel form with z = P r, as in Saad,
Iterative Methods for Sparse Linear Systems, 2nd ed., Algorithm 9.1) with the
block-Jacobi P = blockdiag(D_i)^-1, D_i the N_phi x N_phi diagonal block of A
on triangle i, sliced from the oracle's own sparse matrix and inverted densely.

Vectors are in the natural numbering: triangle i, local DOF k at i*Nphi + k.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .assemble import Blocks


def gradient_matrix(bl: Blocks) -> sp.csr_matrix:
    """Global G (2*Nd*Npsi x Ne*Nphi) from the blocks Q_ij of eq. ad5.2."""
    nd = bl.conn.n_edge
    npsi, nphi = bl.Q.shape[2], bl.Q.shape[3]
    rows, cols, vals = [], [], []
    kk, ll = np.meshgrid(np.arange(npsi), np.arange(nphi), indexing="ij")
    for side in range(2):
        tri_id = bl.conn.lr[:, side]
        for c in range(2):
            r = c * nd * npsi + np.arange(nd)[:, None, None] * npsi + kk[None]
            col = tri_id[:, None, None] * nphi + ll[None]
            rows.append(np.broadcast_to(r, (nd, npsi, nphi)).ravel())
            cols.append(np.broadcast_to(col, (nd, npsi, nphi)).ravel())
            vals.append(bl.Q[:, side, :, :, c].ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    keep = vals != 0.0
    G = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])),
                      shape=(2 * nd * npsi, bl.conn.n_tri * nphi))
    return G.tocsr()


def divergence_matrix(bl: Blocks) -> sp.csr_matrix:
    """Global D (Ne*Nphi x 2*Nd*Npsi) from the blocks D_ij of eq. D."""
    nd = bl.conn.n_edge
    nphi, npsi = bl.D.shape[2], bl.D.shape[3]
    rows, cols, vals = [], [], []
    kk, ll = np.meshgrid(np.arange(nphi), np.arange(npsi), indexing="ij")
    for side in range(2):
        tri_id = bl.conn.lr[:, side]
        for c in range(2):
            r = tri_id[:, None, None] * nphi + kk[None]
            col = c * nd * npsi + np.arange(nd)[:, None, None] * npsi + ll[None]
            rows.append(np.broadcast_to(r, (nd, nphi, npsi)).ravel())
            cols.append(np.broadcast_to(col, (nd, nphi, npsi)).ravel())
            vals.append(bl.D[:, side, :, :, c].ravel())
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    keep = vals != 0.0
    D = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])),
                      shape=(bl.conn.n_tri * nphi, 2 * nd * npsi))
    return D.tocsr()


def dual_mass_inverse(bl: Blocks) -> np.ndarray:
    """Mhat_j^{-1} per edge by dense Cholesky: f64[Nd, Npsi, Npsi]."""
    Lc = np.linalg.cholesky(bl.Mhat)
    eye = np.broadcast_to(np.eye(bl.Mhat.shape[1]), bl.Mhat.shape)
    Linv = np.linalg.solve(Lc, eye)
    return np.swapaxes(Linv, -1, -2) @ Linv


def block_diag_csr(blocks, repeat=1) -> sp.csr_matrix:
    mats = [sp.csr_matrix(b) for b in blocks] * repeat
    return sp.block_diag(mats, format="csr")


class Operators:
    """Global sparse operators of one mesh and degree."""

    def __init__(self, bl: Blocks):
        self.bl = bl
        self.p = bl.p
        self.nphi = bl.Mbar.shape[1]
        self.npsi = bl.Mhat.shape[1]
        self.n = bl.conn.n_tri * self.nphi
        self.nd = bl.conn.n_edge
        self.G = gradient_matrix(bl)
        self.Dm = divergence_matrix(bl)
        self.Minv = dual_mass_inverse(bl)
        self._K = None

    # -- factored applies -------------------------------------------------
    def apply_Mhat_inv(self, v):
        """v laid out [2, Nd, Npsi] (flattened)."""
        v = v.reshape(2, self.nd, self.npsi)
        return np.einsum("jkl,cjl->cjk", self.Minv, v).ravel()

    def apply_K(self, x):
        """K_h x = G^T Mhat^{-1} G x."""
        return self.G.T @ self.apply_Mhat_inv(self.G @ x)

    def apply_schur(self, x, dt):
        return dt * dt * self.apply_K(x)

    def apply_Mbar(self, x):
        x = x.reshape(-1, self.nphi)
        return np.einsum("ekl,el->ek", self.bl.Mbar, x).ravel()

    def apply_helmholtz(self, x, nu_dt):
        return self.apply_Mbar(x) + nu_dt * self.apply_K(x)

    # -- assembled matrices ----------------------------------------------
    def K(self):
        if self._K is None:
            Minv = block_diag_csr(self.Minv, repeat=2)
            self._K = (self.G.T @ (Minv @ self.G)).tocsr()
        return self._K

    def schur_matrix(self, dt):
        return (dt * dt) * self.K()

    def helmholtz_matrix(self, nu_dt):
        return (block_diag_csr(self.bl.Mbar) + nu_dt * self.K()).tocsr()

    # -- projections of eqs. d2m / m2d ------------------------------------
    def d2m_rhs(self, vhat):
        """b_i = sum_{j in S_i} U_ij^T vhat_j (the M-weighted form of eq. d2m)
        for one scalar dual field vhat [Nd, Npsi]."""
        vhat = vhat.reshape(self.nd, self.npsi)
        out = np.zeros((self.bl.conn.n_tri, self.nphi))
        for side in range(2):
            contrib = np.einsum("jkl,jk->jl", self.bl.U[:, side], vhat)
            np.add.at(out, self.bl.conn.lr[:, side], contrib)
        return out.ravel()

    def d2m(self, vhat):
        """Eq. d2m: vbar_i = Mbar_i^{-1} sum_j U_ij^T vhat_j."""
        b = self.d2m_rhs(vhat).reshape(-1, self.nphi)
        return np.linalg.solve(self.bl.Mbar, b[..., None])[..., 0].ravel()

    def m2d(self, vbar):
        """Eq. m2d: vhat_j = Mhat_j^{-1} (U_lj vbar_l + U_rj vbar_r)."""
        vbar = vbar.reshape(-1, self.nphi)
        lr = self.bl.conn.lr
        t = (np.einsum("jkl,jl->jk", self.bl.U[:, 0], vbar[lr[:, 0]])
             + np.einsum("jkl,jl->jk", self.bl.U[:, 1], vbar[lr[:, 1]]))
        return np.einsum("jkl,jl->jk", self.Minv, t).ravel()

    # -- velocity update of eq. nc.2 ---------------------------------------
    def velocity_update(self, F, p, coef):
        """Eq. nc.2 without its source terms, solved for the new dual velocity:
        vhat_j = F_j - coef Mhat_j^{-1} (Q_lj p_l + Q_rj p_r), F a vector dual
        field [2, Nd, Npsi] (flattened), p a main field.  coef is dt for the
        paper's pressure; dt^2 for the p of S p = G^T F (S = dt^2 G^T Mhat^-1 G)."""
        return np.asarray(F, dtype=float).ravel() - coef * self.apply_Mhat_inv(self.G @ p)


def project_mean(v):
    return v - v.mean()


def schur_direct_solver(S):
    """Factorises S once and returns b -> the mean-zero solution of
    S x = Pi b.  The nullspace of S is span{1}, so grounding DOF 0 (deleting
    its row and column) leaves a nonsingular SPD system; its sparse LU
    solution (x_0 = 0) is then shifted to mean zero.  This equals the
    solution of the bordered system [[S, 1], [1^T, 0]] without the fill-in of
    the dense border."""
    S = sp.csr_matrix(S)
    n = S.shape[0]
    lu = spla.splu(S[1:, 1:].tocsc())

    def solve(b):
        rhs = project_mean(b)
        x = np.zeros(n)
        x[1:] = lu.solve(rhs[1:])
        return project_mean(x)
    return solve


def schur_solve_direct(S, b):
    """Mean-zero solution of S x = Pi b (see schur_direct_solver)."""
    return schur_direct_solver(S)(b)


def direct_solve(A, b):
    return spla.splu(sp.csc_matrix(A)).solve(b)


def cg(apply, b, tol=1e-12, maxit=100000, mean_zero=False):
    """Plain conjugate gradients, x0 = 0, stop at ||r||_2 <= tol ||b||_2.
    Returns (x, iterations, recursive relative residual)."""
    if mean_zero:
        b = project_mean(b)
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    bn = np.sqrt(b @ b)
    if bn == 0.0:
        return x, 0, 0.0
    it = 0
    while np.sqrt(rr) > tol * bn and it < maxit:
        q = apply(p)
        if mean_zero:
            q = project_mean(q)
        alpha = rr / (p @ q)
        x += alpha * p
        r -= alpha * q
        rr_new = r @ r
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, np.sqrt(rr) / bn


def cg_lanczos_extremes(apply, b, iters, mean_zero=False):
    """Extreme eigenvalues of A estimated from plain CG's own coefficients
    (the Lanczos connection of CG; Saad, Iterative Methods for Sparse Linear
    Systems, 2nd ed., Sec. 6.7.3): after k steps with step lengths alpha_j and
    direction updates beta_j, the symmetric tridiagonal T_k with
        T[j, j]   = 1/alpha_j + beta_{j-1}/alpha_{j-1}   (beta_{-1} = 0)
        T[j, j+1] = sqrt(beta_j) / alpha_j
    is the Lanczos matrix of A started from b, so its extreme eigenvalues
    approach A's from inside: lambda_max from below, the smallest eigenvalue
    on the Krylov space (the smallest nonzero one for the mean-zero Schur
    operator) from above.  The recurrence stops once ||r|| <= 1e-13 ||b||:
    beyond that its coefficients are rounding noise.  Returns (lambda_min,
    lambda_max, k)."""
    if mean_zero:
        b = project_mean(b)
    r = b.copy()
    p = r.copy()
    rr = r @ r
    stop = (1e-13 ** 2) * rr
    alphas, betas = [], []
    for _ in range(iters):
        q = apply(p)
        if mean_zero:
            q = project_mean(q)
        pq = p @ q
        if not pq > 0.0:
            break
        alpha = rr / pq
        r = r - alpha * q
        rr_new = r @ r
        beta = rr_new / rr
        alphas.append(alpha)
        betas.append(beta)
        rr = rr_new
        if rr <= stop:
            break
        p = r + beta * p
    k = len(alphas)
    diag = np.empty(k)
    off = np.empty(max(0, k - 1))
    for j in range(k):
        diag[j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            off[j] = np.sqrt(betas[j]) / alphas[j]
    T = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    ev = np.linalg.eigvalsh(T)
    return float(ev[0]), float(ev[-1]), k


def block_jacobi_blocks(A, nphi):
    """Inverse diagonal blocks of A: [n/nphi, nphi, nphi], block i =
    (A[i*nphi:(i+1)*nphi, i*nphi:(i+1)*nphi])^-1 (symmetrised before inversion)."""
    A = sp.csr_matrix(A)
    ne = A.shape[0] // nphi
    out = np.empty((ne, nphi, nphi))
    for i in range(ne):
        sl = slice(i * nphi, (i + 1) * nphi)
        D = A[sl, sl].toarray()
        out[i] = np.linalg.inv(0.5 * (D + D.T))
    return out


def apply_blocks(blocks, v):
    """y_i = blocks[i] v_i for every triangle i (v in the natural numbering)."""
    ne, nphi, _ = blocks.shape
    return np.einsum("ekl,el->ek", blocks, np.asarray(v).reshape(ne, nphi)).ravel()


def pcg(apply, b, precond, tol=1e-12, maxit=100000, mean_zero=False):
    """Preconditioned CG (textbook form): x0 = 0, r = b, z = P r, p = z;
    alpha = (r, z) / (p, A p); x += alpha p; r -= alpha A p; z = P r;
    beta = (r, z)_new / (r, z)_old; p = z + beta p; stop at ||r||_2 <= tol ||b||_2.
    precond(v) applies P.  mean_zero: b projected to mean zero, A p projected
    likewise (the pressure operator's nullspace is span{1}), x returned
    mean-free.  Returns (x, iterations, recursive relative residual)."""
    if mean_zero:
        b = project_mean(b)
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.sqrt(b @ b)
    if bn == 0.0:
        return x, 0, 0.0
    z = precond(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while np.sqrt(r @ r) > tol * bn and it < maxit:
        q = apply(p)
        if mean_zero:
            q = project_mean(q)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
        it += 1
    if mean_zero:
        x = project_mean(x)
    return x, it, np.sqrt(r @ r) / bn


def sampled_rows(conn, p, x, tri_ids, coefK, coefM=0.0):
    """Rows of (coefM Mbar + coefK G^T Mhat^{-1} G) x for the triangles tri_ids
    only (natural numbering), assembling just the edges they touch.  Used to
    check full-size results one output block at a time."""
    from .assemble import edge_blocks, main_mass
    from . import basis as B
    nphi = B.n_phi(p)
    tri_ids = np.asarray(tri_ids)
    edges = np.unique(conn.tri_edge[tri_ids].ravel())
    Mhat, D, Q, U, n, glen = edge_blocks(conn, p, edges)
    Lc = np.linalg.cholesky(Mhat)
    X = x.reshape(-1, nphi)
    lr = conn.lr[edges]
    t = np.stack([np.einsum("eklc,el->cek", Q[:, s], X[lr[:, s]]) for s in range(2)]).sum(0)
    g = np.stack([np.linalg.solve(np.swapaxes(Lc, -1, -2),
                                  np.linalg.solve(Lc, t[c][..., None]))[..., 0] for c in range(2)])
    pos = {int(e): k for k, e in enumerate(edges)}
    out = np.zeros((len(tri_ids), nphi))
    for a, i in enumerate(tri_ids):
        for e in conn.tri_edge[i]:
            k = pos[int(e)]
            s = 0 if conn.lr[e, 0] == i else 1
            out[a] += coefK * np.einsum("klc,ck->l", Q[k, s], g[:, k])
    if coefM != 0.0:
        sub = type(conn)(len(tri_ids), 0, None, None, None, None, None, conn.tri_xy[tri_ids])
        Mb, _ = main_mass(sub, p)
        out += coefM * np.einsum("akl,al->ak", Mb, X[tri_ids])
    return out
