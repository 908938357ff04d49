"""Oracle: the semi-implicit IMEX Runge-Kutta tableaux of App. A (eq. IMEX1,
IMEX2, IMEX3), the semi-Lagrangian stage trajectories of Sec. 3 (after
eq. butcher) that use the explicit tableau, and the SL-IMEX step of the
advection-diffusion model (Sec. 3, its advection-diffusion subsection): a
main-grid scalar C carried by a steady main-grid velocity and diffused
implicitly.

Readings (the paper gives the scheme as an overview):
 - Tableaux: the numbers of App. A as printed (six digits for R = 2, whose
   weights then sum to 0.999999); gamma = 1 - 1/sqrt(2) and
   beta = 1/(2 gamma) exactly for R = 1.
 - Stage trajectories: the characteristic equation integrated backward over
   dt by the explicit Runge-Kutta scheme (A~, b) from the Gauss point x:
       x^E_s = x - dt sum_{j<s} a~_{s,j} V_j,   V_j = vbar(x^E_j),
       x_F   = x - dt sum_j b_j V_j.
   The printed updates combine H^L = -vbar with a minus sign, which would
   move the points forward; both are read as one backward step.
 - Each stage point is located by walking the straight segment from x to it
   element by element (the walk of Sec. 2.5 with a constant velocity), so no
   global search is made; vbar is evaluated with the polynomial of the cell
   reached.
 - Without diffusion the stage fluxes H^P vanish, the shifted fluxes and the
   stage solves drop out, and the new field is the old one at the final foot,
   projected as eq. intstage.

Readings of the advection-diffusion step (the paper gives the stage
formulas as an overview; stages s = 1..Ns, implicit tableau (A, b, c)):
 - V_j(x) = vbar(x^E_j(x)) are the stage velocities of the trajectory from
   the Gauss point x (above); the implicit trajectory of stage s is
   x^I_s = x - dt sum_{j<=s} a_{s,j} V_j.
 - The stage-j flux enters stage s at the point where the characteristic
   through x at stage s was at stage j: x - (c_s - c_j) dt V_j.  The printed
   shift weight w_j = sum_{r<=j} a_{j,r} - sum_{r<=j} a_{s,r} is read with
   the second sum over the whole row s (c_j - c_s) and with the backward
   sign of the trajectories.  As printed, the sum leaves out a_{s,s} (and
   any entries between j and s), so even a constant velocity misplaces the
   fluxes by O(dt) and the scheme falls to first order.
 - The stage value is C^I_s = proj[C^n(x^I_s) + sum_{j<s} dt a_{s,j}
   H_j(x - (c_s - c_j) dt V_j)], projected by eq. intstage from the Gauss
   points (the printed "U^n(x)" is read as C^n at the implicit foot, where
   the text says the solution is interpolated).
 - The diffusion sub-system (Mbar + a_{s,s} dt alpha K) C*_s = Mbar C^I_s,
   the discrete form of eq. ad5 with lambda = alpha, gives the stage flux
   H_s = (C*_s - C^I_s) / (a_{s,s} dt) = -alpha Mbar^-1 K C*_s.
 - The tableaux of App. A are stiffly accurate (a_{Ns,j} = b_j), so the final
   update C^n(x_F) + sum_j dt b_j H_j(x - (1 - c_j) dt V_j) equals the last
   stage: C^{n+1} = C*_{Ns}.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from . import basis as B
from . import sl as SL
from .assemble import main_mass
from .mesh import Connectivity


def tableau(R):
    """(At, bt, ct, A, b, c) of App. A for R = 0, 1, 2 (explicit At strictly
    lower triangular; implicit A with its diagonal)."""
    if R == 0:
        At = np.array([[0.0]])
        bt = np.array([1.0])
        A = np.array([[1.0]])
        b = np.array([1.0])
    elif R == 1:
        g = 1.0 - 1.0 / math.sqrt(2.0)
        be = 1.0 / (2.0 * g)
        At = np.array([[0.0, 0.0], [be, 0.0]])
        bt = np.array([1.0 - g, g])
        A = np.array([[g, 0.0], [1.0 - g, g]])
        b = bt.copy()
    elif R == 2:
        g = 0.435866
        At = np.array([[0.0, 0.0, 0.0, 0.0],
                       [g, 0.0, 0.0, 0.0],
                       [1.437745, -0.719812, 0.0, 0.0],
                       [0.916993, 0.5, -0.416993, 0.0]])
        bt = np.array([0.0, 1.208496, -0.644363, g])
        A = np.array([[g, 0.0, 0.0, 0.0],
                      [0.0, g, 0.0, 0.0],
                      [0.0, 0.282066, g, 0.0],
                      [0.0, 1.208496, -0.644363, g]])
        b = bt.copy()
    else:
        raise ValueError("R must be 0, 1 or 2")
    return At, bt, At.sum(axis=1), A, b, A.sum(axis=1)


def rk_foot(velocity_at, x, dt, R):
    """x_F for one point: velocity_at(stage point) -> v[2] (any callable)."""
    At, bt, _, _, _, _ = tableau(R)
    x = np.asarray(x, dtype=np.float64)
    V = []
    for s in range(len(bt)):
        xs = x - dt * sum(At[s, j] * V[j] for j in range(s)) if s else x.copy()
        V.append(np.asarray(velocity_at(xs), dtype=np.float64))
    return x - dt * sum(bt[j] * V[j] for j in range(len(bt)))


def locate_from(tri_xy, nbr, trans, back, x, cell, d, max_steps=4096):
    """The point x + d reached from x (in `cell`'s frame) along the straight
    segment, element by element: (point in the frame of its cell, cell,
    cells crossed)."""
    d = np.asarray(d, dtype=np.float64)
    if d[0] == 0.0 and d[1] == 0.0:
        return np.array(x, dtype=np.float64), cell, 0
    # the walk follows x - s v over the time 1: v = -d
    return SL.walk(tri_xy, nbr, trans, back, lambda c, xi, eta: -d, x, cell, 1.0, max_steps)


def rk_transport(conn: Connectivity, period, p, vbar, c, dt, R, max_steps=4096):
    """Feet of the stage-trajectory scheme for every Gauss point and the
    fields at the feet projected (eq. intstage).

    vbar: f64[2, Ne, Nphi] steady main-grid velocity; c: f64[nf, Ne, Nphi].
    Returns (foot f64[Ne, Ng, 2] in the containing cell's frame, cell
    i32[Ne, Ng], steps i32[Ne, Ng] = cells crossed by all the stage walks and
    the final one, cstar f64[nf, Ne, Nphi])."""
    vbar = np.asarray(vbar, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    At, bt, _, _, _, _ = tableau(R)
    ne = conn.n_tri
    pts, w = SL.quadrature(p)
    ng = len(w)
    nphi = B.n_phi(p)
    nbr, trans, back = SL.frames(conn, period)
    X = B.triangle_points(conn.tri_xy, pts)

    def vel(cell, y):
        _, xi, eta = SL.barycentric(conn.tri_xy[cell], y)
        return vbar[:, cell, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]

    foot = np.zeros((ne, ng, 2))
    cell = np.zeros((ne, ng), dtype=np.int32)
    steps = np.zeros((ne, ng), dtype=np.int32)
    vals = np.zeros((c.shape[0], ne, ng))
    for i in range(ne):
        for g in range(ng):
            x = X[i, g]
            V = []
            nst = 0
            for s in range(len(bt)):
                d = -dt * sum(At[s, j] * V[j] for j in range(s)) if s else np.zeros(2)
                y, cy, st = locate_from(conn.tri_xy, nbr, trans, back, x, i, d, max_steps)
                nst += st
                V.append(vel(cy, y))
            d = -dt * sum(bt[j] * V[j] for j in range(len(bt)))
            xf, cf, st = locate_from(conn.tri_xy, nbr, trans, back, x, i, d, max_steps)
            foot[i, g], cell[i, g], steps[i, g] = xf, cf, nst + st
            _, xi, eta = SL.barycentric(conn.tri_xy[cf], xf)
            vals[:, i, g] = c[:, cf, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]
    phi_g = B.eval_phi(p, pts)
    Mbar, _ = main_mass(conn, p)
    e1 = conn.tri_xy[:, 1] - conn.tri_xy[:, 0]
    e2 = conn.tri_xy[:, 2] - conn.tri_xy[:, 0]
    absJ = np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    cstar = np.zeros((c.shape[0], ne, nphi))
    for f in range(c.shape[0]):
        rhs = np.einsum("gl,g,ig->il", phi_g, w, vals[f]) * absJ[:, None]
        cstar[f] = np.linalg.solve(Mbar, rhs[..., None])[..., 0]
    return foot, cell, steps, cstar


def advdiff_step(ops, conn: Connectivity, period, p, vbar, C, dt, alpha, R, max_steps=4096):
    """One SL-IMEX step of the advection-diffusion model: vbar f64[2, Ne,
    Nphi] steady main-grid velocity, C f64[Ne * Nphi] (natural order), ops an
    oracle.operators.Operators of the same mesh and degree.  Returns C^{n+1}."""
    from . import operators as OPS
    vbar = np.asarray(vbar, dtype=np.float64)
    Cn = np.asarray(C, dtype=np.float64).reshape(conn.n_tri, -1)
    At, bt, _, A, b, c = tableau(R)
    ns = len(b)
    ne = conn.n_tri
    pts, w = SL.quadrature(p)
    ng = len(w)
    nphi = B.n_phi(p)
    nbr, trans, back = SL.frames(conn, period)
    X = B.triangle_points(conn.tri_xy, pts)

    def value(field, cell, y):
        _, xi, eta = SL.barycentric(conn.tri_xy[cell], y)
        return field[..., cell, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]

    def at(field, i, x, d):
        y, cy, _ = locate_from(conn.tri_xy, nbr, trans, back, x, i, d, max_steps)
        return value(field, cy, y)

    # stage velocities of every Gauss-point trajectory: V[j, i, g]
    V = np.zeros((ns, ne, ng, 2))
    for i in range(ne):
        for g in range(ng):
            for s in range(ns):
                d = -dt * sum(At[s, j] * V[j, i, g] for j in range(s)) if s else np.zeros(2)
                V[s, i, g] = at(vbar, i, X[i, g], d)
    # projection of Gauss-point values (eq. intstage)
    phi_g = B.eval_phi(p, pts)
    Mbar, _ = main_mass(conn, p)
    e1 = conn.tri_xy[:, 1] - conn.tri_xy[:, 0]
    e2 = conn.tri_xy[:, 2] - conn.tri_xy[:, 0]
    absJ = np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])

    def project(vals):
        rhs = np.einsum("gl,g,ig->il", phi_g, w, vals) * absJ[:, None]
        return np.linalg.solve(Mbar, rhs[..., None])[..., 0]

    H = []
    Cs = None
    for s in range(ns):
        vals = np.zeros((ne, ng))
        for i in range(ne):
            for g in range(ng):
                x = X[i, g]
                d = -dt * sum(A[s, j] * V[j, i, g] for j in range(s + 1))
                v = at(Cn, i, x, d)
                for j in range(s):
                    if A[s, j] != 0.0:
                        v += dt * A[s, j] * at(H[j], i, x, -(c[s] - c[j]) * dt * V[j, i, g])
                vals[i, g] = v
        CI = project(vals).ravel()
        Hm = ops.helmholtz_matrix(A[s, s] * dt * alpha)
        Cs = OPS.direct_solve(Hm, ops.apply_Mbar(CI))
        H.append(((Cs - CI) / (A[s, s] * dt)).reshape(ne, nphi))
    return Cs


def ns_imex_step(ops, conn: Connectivity, period, p, vhat, dt, nu, R, max_steps=4096):
    """One SL-IMEX step of the incompressible Navier-Stokes equations (no
    temperature or gravity) with the tableaux of App. A: vhat f64[2 * Nd *
    Npsi] (component-major, natural order) -> (vhat^{n+1}, pressure of the
    last stage).

    Readings, extending those of advdiff_step to a velocity that changes
    within the step (stages s = 1..Ns, explicit (A~, c~), implicit (A, c)):
     - the main-grid velocity vbar^n = L_dm(vhat^n) (eq. d2m) is transported;
     - the explicit stage velocity field is
         vbar^E_s = proj[vbar^n(x - dt sum_{j<s} a~_{s,j} V_j)
                         + sum_{j<s} dt a~_{s,j} Hbar_j(x - (c~_s - c_j) dt V_j)],
       the same projection as the implicit stage value with the explicit
       row, and the stage velocity of the trajectory from x is
       V_s = vbar^E_s(x^E_s) (V_1 = vbar^n(x));
     - the implicit stage value vbar^I_s is formed as in advdiff_step, each
       component solves (Mbar + a_ss dt nu K) vbar* = Mbar vbar^I_s (eq. ad5),
       vhat* = L_md(vbar*) (eq. m2d), the pressure solves S pi = G^T vhat* with
       S = (a_ss dt)^2 G^T Mhat^-1 G (eq. pressure_final for the stage) and
       vhat_s = vhat* - (a_ss dt)^2 Mhat^-1 G pi (eq. nc.2);
     - the stage flux Hhat_s = (vhat_s - L_md(vbar^I_s)) / (a_ss dt) lives on
       the dual grid, where the velocity is defined; its main-grid copy
       Hbar_s = L_dm(Hhat_s) is the field that is shifted;
     - stiffly accurate tableaux: vhat^{n+1} = vhat_Ns."""
    from . import operators as OPS
    nd, npsi, ne, nphi = ops.nd, ops.npsi, conn.n_tri, ops.nphi
    At, bt, ct, A, b, c = tableau(R)
    ns = len(b)
    pts, w = SL.quadrature(p)
    ng = len(w)
    nbr, trans, back = SL.frames(conn, period)
    X = B.triangle_points(conn.tri_xy, pts)
    phi_g = B.eval_phi(p, pts)
    Mbar, _ = main_mass(conn, p)
    e1 = conn.tri_xy[:, 1] - conn.tri_xy[:, 0]
    e2 = conn.tri_xy[:, 2] - conn.tri_xy[:, 0]
    absJ = np.abs(e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])

    def project(vals):  # [2, Ne, Ng] -> [2, Ne, Nphi]
        rhs = np.einsum("gl,g,kig->kil", phi_g, w, vals) * absJ[None, :, None]
        return np.stack([np.linalg.solve(Mbar, rhs[k][..., None])[..., 0] for k in range(2)])

    def at(field, i, x, d):  # field [2, Ne, Nphi] at x + d
        y, cy, _ = locate_from(conn.tri_xy, nbr, trans, back, x, i, d, max_steps)
        _, xi, eta = SL.barycentric(conn.tri_xy[cy], y)
        return field[:, cy, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]

    vh = np.asarray(vhat, dtype=np.float64).reshape(2, nd * npsi)
    vn = np.stack([ops.d2m(vh[k]) for k in range(2)]).reshape(2, ne, nphi)
    V = np.zeros((ns, ne, ng, 2))
    Hbar = []

    def stage_field(row, cs, s, with_diag):
        """proj[vbar^n(x - dt sum_j row_j V_j) + sum_{j<s} dt row_j Hbar_j(x - (cs - c_j) dt V_j)]."""
        vals = np.zeros((2, ne, ng))
        for i in range(ne):
            for g in range(ng):
                x = X[i, g]
                jmax = s + 1 if with_diag else s
                d = -dt * sum(row[j] * V[j, i, g] for j in range(jmax)) if jmax else np.zeros(2)
                v = at(vn, i, x, d)
                for j in range(s):
                    if row[j] != 0.0:
                        v = v + dt * row[j] * at(Hbar[j], i, x, -(cs - c[j]) * dt * V[j, i, g])
                vals[:, i, g] = v
        return project(vals)

    pr = None
    vs = None
    for s in range(ns):
        # stage velocity of every trajectory
        if s == 0:
            for i in range(ne):
                for g in range(ng):
                    V[0, i, g] = at(vn, i, X[i, g], np.zeros(2))
        else:
            vE = stage_field(At[s], ct[s], s, False)
            for i in range(ne):
                for g in range(ng):
                    d = -dt * sum(At[s, j] * V[j, i, g] for j in range(s))
                    V[s, i, g] = at(vE, i, X[i, g], d)
        vI = stage_field(A[s], c[s], s, True).reshape(2, -1)
        h = A[s, s] * dt
        Hm = ops.helmholtz_matrix(nu * h)
        vst = np.stack([OPS.direct_solve(Hm, ops.apply_Mbar(vI[k])) for k in range(2)])
        vhs = np.stack([ops.m2d(vst[k]) for k in range(2)]).ravel()
        pr = OPS.schur_solve_direct(ops.schur_matrix(h), ops.G.T @ vhs)
        vs = ops.velocity_update(vhs, pr, h * h).reshape(2, -1)
        vIh = np.stack([ops.m2d(vI[k]) for k in range(2)])
        Hh = (vs - vIh) / h
        Hbar.append(np.stack([ops.d2m(Hh[k]) for k in range(2)]).reshape(2, ne, nphi))
    return vs.ravel(), pr
