"""Oracle: semi-Lagrangian trajectories and transport (Sec. 2.5, eq. lagrtrj;
the Gauss-point projection of eq. intstage).

Reading of Sec. 2.5 (the paper describes the method in words):
 - The trajectory equation dx/dt = v is integrated backward in time over dt
   with straight pieces (Euler).  A trajectory starts at a quadrature point
   x_g of main triangle i.  From a point x in triangle T, with the velocity
   v = vbar_T(x) of T's DG velocity polynomial at x, the backward ray
   x - s v (0 <= s <= tau, tau the time left) either stays in T up to
   s = tau, giving the foot x - tau v, or leaves T through an edge at
   s = s_e < tau.  The walk then moves to that exit point, sets
   tau <- tau - s_e, and continues in the neighbour across the edge with the
   neighbour's velocity polynomial.  Each piece crosses at most one cell, so
   no global search is needed, and periodic neighbours are reached by a frame
   translation.
 - Local edge k joins vertices (v_k, v_{k+1}); the ray leaves through it when
   the barycentric coordinate of the opposite vertex v_{k+2} reaches 0.  Among
   the edges whose opposite barycentric decreases along the ray, the exit is
   the one with the smallest s (a slightly negative barycentric counts as 0);
   equal s goes to the lowest k.  A zero velocity ends the walk in place.
 - dt < 0 (forward characteristics): the same walk along x + s v, i.e. with
   -v over the time |dt|.
 - Held trajectories (the paper is silent here): the DG velocity jumps
   across edges, and where the backward rays of two neighbours both point at
   their shared edge (the forward flow leaves the edge on both sides) the walk
   would cross back and forth with pieces of zero length and never end.  A
   walk that leaves a cell through the edge it entered by (a bounce: the
   velocity at the arrival point sends the ray straight back) is normal once,
   since the cell it returns to may carry it on along its own velocity; when
   the cell it bounced back into sends it across that same edge again, the
   trajectory is held: the foot is the current point (on that edge) in the
   current cell, and the time left is dropped.
 - Each triangle has its own frame: its vertices unwrapped around v_0
   (Connectivity.tri_xy).  Crossing local edge k adds the whole number of
   periods that maps T's frame to the neighbour's; the foot is reported in
   the frame of the triangle that contains it.
 - The quadrature is the collapsed Gauss-Legendre rule with (p+1)^2 points
   (exact to degree 2p+1), and the transported field is the projection of
   eq. intstage:
       c*_i = Mbar_i^{-1} sum_g phi(xi_g) c(x_F(x_g)) w_g |J_i|,
   with |J_i| = A_i = 2|T_i| and c(x_F) the field's polynomial in the
   triangle that contains the foot.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import basis as B
from .assemble import main_mass
from .mesh import Connectivity, neighbours


class WalkError(RuntimeError):
    pass


def quadrature(p):
    """Gauss points (pts f64[(p+1)^2, 2] on T_ref) and weights (sum 1/2)."""
    return B.duffy_rule(p + 1)


def frames(conn: Connectivity, period):
    """Neighbour across each local edge, i32[Ne, 3]; the translation
    f64[Ne, 3, 2] that maps a point of a triangle's frame into that
    neighbour's frame (conn.shift: periods to add to r's frame to reach l's);
    and back i32[Ne, 3], the local index of the same edge in the neighbour."""
    period = np.asarray(period, dtype=np.float64)
    nbr = neighbours(conn)
    trans = np.zeros((conn.n_tri, 3, 2))
    back = np.zeros((conn.n_tri, 3), dtype=np.int32)
    for t in range(conn.n_tri):
        for k in range(3):
            j = conn.tri_edge[t, k]
            l, r = conn.lr[j]
            s = conn.shift[j].astype(np.float64) * period
            trans[t, k] = -s if t == l else s
            back[t, k] = conn.loc[j, 1] if t == l else conn.loc[j, 0]
    return nbr, trans, back


def barycentric(P, x):
    """Barycentric coordinates (lambda_0, lambda_1, lambda_2) of x in the
    triangle with vertices P[3, 2], and its reference coordinates (xi, eta)
    (the inverse of the affine map, by Cramer's rule)."""
    e1 = P[1] - P[0]
    e2 = P[2] - P[0]
    d = x - P[0]
    det = e1[0] * e2[1] - e1[1] * e2[0]
    xi = (d[0] * e2[1] - d[1] * e2[0]) / det
    eta = (e1[0] * d[1] - e1[1] * d[0]) / det
    return np.array([1.0 - xi - eta, xi, eta]), xi, eta


def barycentric_rates(P, v):
    """d lambda / d s along the backward ray x - s v."""
    e1 = P[1] - P[0]
    e2 = P[2] - P[0]
    det = e1[0] * e2[1] - e1[1] * e2[0]
    dxi = (v[0] * e2[1] - v[1] * e2[0]) / det
    deta = (e1[0] * v[1] - e1[1] * v[0]) / det
    return -np.array([-dxi - deta, dxi, deta])


def dg_value(p, coeffs, xi, eta):
    """Value at (xi, eta) of the polynomial with nodal coefficients coeffs[Nphi]."""
    phi = B.eval_phi(p, np.array([[xi, eta]]))[0]
    return float(phi @ coeffs)


def walk(tri_xy, nbr, trans, back, velocity, x, cell, dt, max_steps=4096):
    """Backward trajectory from x (in triangle `cell`'s frame) over dt.
    velocity(cell, xi, eta) -> v[2].  Returns (foot, cell, pieces crossed)."""
    x = np.array(x, dtype=np.float64)
    sign = -1.0 if dt < 0 else 1.0
    tau = abs(float(dt))
    steps = 0
    k_in = -1  # local edge of `cell` through which the walk entered it
    bounced = False  # the walk entered `cell` by leaving the last cell through its entry edge
    while True:
        P = tri_xy[cell]
        lam, xi, eta = barycentric(P, x)
        v = sign * np.asarray(velocity(cell, xi, eta), dtype=np.float64)
        if v[0] == 0.0 and v[1] == 0.0:
            return x, cell, steps
        rate = barycentric_rates(P, v)
        s_exit, k_exit = np.inf, -1
        for k in range(3):
            o = (k + 2) % 3
            if rate[o] < 0.0:
                s = max(lam[o], 0.0) / -rate[o]
                if s < s_exit:
                    s_exit, k_exit = s, k
        if k_exit < 0 or s_exit >= tau:
            return x - tau * v, cell, steps
        if k_exit == k_in and bounced:  # a second bounce on the same edge: held
            return x, cell, steps
        x = x - s_exit * v + trans[cell, k_exit]
        tau -= s_exit
        bounced = k_exit == k_in
        k_in = int(back[cell, k_exit])
        cell = int(nbr[cell, k_exit])
        steps += 1
        if steps > max_steps:
            raise WalkError("trajectory crossed more than max_steps cells")


def transport(conn: Connectivity, period, p, vbar, c, dt, max_steps=4096):
    """Feet of every Gauss-point trajectory and the transported fields.

    vbar: f64[2, Ne, Nphi] main-grid velocity (nodal coefficients, natural
    order); c: f64[nf, Ne, Nphi] fields.  Returns (foot f64[Ne, Ng, 2] in the
    frame of the containing triangle, cell i32[Ne, Ng], steps i32[Ne, Ng],
    cstar f64[nf, Ne, Nphi])."""
    vbar = np.asarray(vbar, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    ne = conn.n_tri
    pts, w = quadrature(p)
    ng = len(w)
    nphi = B.n_phi(p)
    nbr, trans, back = frames(conn, period)
    X = B.triangle_points(conn.tri_xy, pts)  # [Ne, Ng, 2]

    def velocity(cell, xi, eta):
        phi = B.eval_phi(p, np.array([[xi, eta]]))[0]
        return vbar[:, cell, :] @ phi

    foot = np.zeros((ne, ng, 2))
    cell = np.zeros((ne, ng), dtype=np.int32)
    steps = np.zeros((ne, ng), dtype=np.int32)
    vals = np.zeros((c.shape[0], ne, ng))
    for i in range(ne):
        for g in range(ng):
            xf, cf, st = walk(conn.tri_xy, nbr, trans, back, velocity, X[i, g], i, dt, max_steps)
            foot[i, g], cell[i, g], steps[i, g] = xf, cf, st
            _, xi, eta = barycentric(conn.tri_xy[cf], xf)
            phi = B.eval_phi(p, np.array([[xi, eta]]))[0]
            vals[:, i, g] = c[:, cf, :] @ phi
    # eq. intstage
    phi_g = B.eval_phi(p, pts)  # [Ng, Nphi]
    Mbar, _ = main_mass(conn, p)  # [Ne, Nphi, Nphi]
    e1 = conn.tri_xy[:, 1] - conn.tri_xy[:, 0]
    e2 = conn.tri_xy[:, 2] - conn.tri_xy[:, 0]
    absJ = np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    cstar = np.zeros((c.shape[0], ne, nphi))
    for f in range(c.shape[0]):
        rhs = np.einsum("gl,g,ig->il", phi_g, w, vals[f]) * absJ[:, None]
        cstar[f] = np.linalg.solve(Mbar, rhs[..., None])[..., 0]
    return foot, cell, steps, cstar


def locate(tri_xy, period, x):
    """Brute force: the triangles whose closure contains the point x (any
    periodic image), with the point in each one's frame."""
    period = np.asarray(period, dtype=np.float64)
    out = []
    for t in range(tri_xy.shape[0]):
        P = tri_xy[t]
        d = x - P[0]
        y = P[0] + d - period * np.round(d / period)
        lam, _, _ = barycentric(P, y)
        if lam.min() >= -1e-12:
            out.append((t, y))
    return out
