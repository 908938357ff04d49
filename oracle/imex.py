"""Oracle: the semi-implicit IMEX Runge-Kutta tableaux of App. A (eq. IMEX1,
IMEX2, IMEX3) and the semi-Lagrangian stage trajectories of Sec. 3 (after
eq. butcher) that use the explicit tableau, for a passive field carried by
a steady main-grid velocity without diffusion (the setting of the paper's
non-linear transport test, Table ct1).

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
