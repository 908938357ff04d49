"""Oracle: nodal bases and quadrature (Sec. 2.2).

Main basis: Lagrange polynomials of degree p on T_ref = {xi, eta >= 0,
xi + eta <= 1}.  Reading of "a simple nodal approach": equispaced nodes
(a/p, b/p), a + b <= p, ordered b-major then a, so that for p = 1 the nodes
are (0,0), (1,0), (0,1) as in the paper's example.  The coefficients come
from inverting the monomial Vandermonde matrix in FP64.

Dual basis (Sec. 2.2, unnumbered equation for psi): on the split unit square
the left half is T_ref and carries phi_m, the right half is 1 - T_ref and
carries phi_m(1 - xi); nodes on the diagonal xi + eta = 1 are identified.
Reading: the permutations L, R are fixed by node coincidence (the printed
p = 1 example swaps psi_2 and psi_3 on the right half, which would make them
discontinuous).  Dual index order: the N_phi left nodes in phi order, then the
right nodes off the diagonal in phi order.  N_psi = (p+1)^2.

Quadrature: Gauss-Legendre nodes by Newton iteration on the three-term
recurrence; triangles by the collapsed (Duffy) product rule, exact to
degree 2n-2 in each direction with n points (n = p+2 is used, so every
integrand of degree <= 2p+1 is integrated exactly).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def n_phi(p):
    return (p + 1) * (p + 2) // 2


def n_psi(p):
    return (p + 1) ** 2


def nodes(p):
    """Equispaced nodes on T_ref, b-major: f64[N_phi, 2]."""
    out = [(a / p, b / p) for b in range(p + 1) for a in range(p + 1 - b)]
    return np.asarray(out, dtype=np.float64)


def node_ab(p):
    return [(a, b) for b in range(p + 1) for a in range(p + 1 - b)]


def monomials(p):
    return [(i, j) for i in range(p + 1) for j in range(p + 1 - i)]


def vandermonde_coeffs(p):
    """C such that phi_k(x) = sum_m C[m, k] * mono_m(x)."""
    X = nodes(p)
    mono = monomials(p)
    V = np.array([[x ** i * y ** j for (i, j) in mono] for (x, y) in X])
    return np.linalg.inv(V)


def eval_phi(p, pts):
    """phi_k at pts (f64[..., 2]) -> f64[..., N_phi]."""
    C = vandermonde_coeffs(p)
    x = pts[..., 0]
    y = pts[..., 1]
    M = np.stack([x ** i * y ** j for (i, j) in monomials(p)], axis=-1)
    return M @ C


def eval_grad_phi(p, pts):
    """d phi_k / d(xi, eta) at pts -> f64[..., N_phi, 2]."""
    C = vandermonde_coeffs(p)
    x = pts[..., 0]
    y = pts[..., 1]
    dx, dy = [], []
    for (i, j) in monomials(p):
        dx.append(i * x ** max(i - 1, 0) * y ** j if i > 0 else np.zeros_like(x))
        dy.append(j * x ** i * y ** max(j - 1, 0) if j > 0 else np.zeros_like(x))
    Mx = np.stack(dx, axis=-1) @ C
    My = np.stack(dy, axis=-1) @ C
    return np.stack([Mx, My], axis=-1)


def dual_maps(p):
    """(L i64[N_phi], R i64[N_phi]): dual index of left / right local node m."""
    ab = node_ab(p)
    index = {v: k for k, v in enumerate(ab)}
    nphi = len(ab)
    L = np.arange(nphi)
    R = np.empty(nphi, dtype=np.int64)
    nxt = nphi
    for m, (a, b) in enumerate(ab):
        if a + b < p:
            R[m] = nxt
            nxt += 1
        else:
            # right local node (a/p, b/p) sits at 1 - (a/p, b/p) = (b/p, a/p)
            R[m] = L[index[(b, a)]]
    assert nxt == n_psi(p)
    return L, R


def gauss_legendre(n, tol=1e-15):
    """n-point Gauss-Legendre rule on [0, 1] (own Newton iteration)."""
    x = np.cos(np.pi * (np.arange(1, n + 1) - 0.25) / (n + 0.5))
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        if n == 1:
            p0, p1 = np.ones_like(x), x.copy()
        dp = n * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < tol:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for k in range(2, n + 1):
        p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
    if n == 1:
        p0, p1 = np.ones_like(x), x.copy()
    dp = n * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    order = np.argsort(x)
    return 0.5 * (x[order] + 1.0), 0.5 * w[order]


def duffy_rule(n):
    """Collapsed rule on T_ref: (pts f64[n*n, 2], w f64[n*n]), sum w = 1/2."""
    u, wu = gauss_legendre(n)
    v, wv = gauss_legendre(n)
    U, V = np.meshgrid(u, v, indexing="ij")
    WU, WV = np.meshgrid(wu, wv, indexing="ij")
    xi = U
    eta = V * (1.0 - U)
    w = WU * WV * (1.0 - U)
    return np.stack([xi.ravel(), eta.ravel()], 1), w.ravel()


def triangle_points(P, ref_pts):
    """Physical points of the affine image of T_ref with vertices P[..., 3, 2]."""
    P0 = P[..., 0, :][..., None, :]
    e1 = (P[..., 1, :] - P[..., 0, :])[..., None, :]
    e2 = (P[..., 2, :] - P[..., 0, :])[..., None, :]
    return P0 + ref_pts[:, 0:1] * e1 + ref_pts[:, 1:2] * e2


def pull_back(P, x):
    """Reference coordinates of physical points x[..., q, 2] in the affine
    triangle P[..., 3, 2] (solves the 2x2 system of eq. linmap)."""
    P0 = P[..., 0, :]
    J = np.stack([P[..., 1, :] - P0, P[..., 2, :] - P0], axis=-1)  # [..., 2(x,y), 2(xi,eta)]
    d = x - P0[..., None, :]
    return np.linalg.solve(J[..., None, :, :], d[..., None])[..., 0]
