"""Oracle: one first-order semi-Lagrangian semi-implicit step of the
incompressible Navier-Stokes equations on the staggered grids (the R = 0,
one-stage Euler tableau of App. A applied to the splitting of Sec. 3:
convection by the semi-Lagrangian transport of Sec. 2.5, the viscous
sub-system of eq. ad5, then the pressure of eq. pressure_final and the
velocity update of eq. nc.2), without temperature or gravity.

Readings (the paper gives the multi-stage scheme; this is its one-stage case):
 - the main-grid velocity vbar^n = L_dm(vhat^n) (eq. d2m) is the transport
   velocity and is itself transported (the projection of the dual velocity
   is transported instead of the dual velocity: the transport of Sec. 2.5
   lives on the main grid);
 - the trajectory is the element-by-element walk of Sec. 2.5 (oracle.sl);
 - viscous step: (Mbar + nu dt K) vbar* = Mbar c, c the transported velocity
   (eq. ad5 with lambda = nu, per component);
 - vhat* = L_md(vbar*) (eq. m2d); the pressure solves S p = G^T vhat* with
   S = dt^2 G^T Mhat^-1 G; vhat^{n+1} = vhat* - dt^2 Mhat^-1 G p (eq. nc.2),
   so that G^T vhat^{n+1} = 0 (eq. nc.1).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import operators as OP
from . import sl as SL


def ns_step(op: OP.Operators, conn, period, p, vhat, dt, nu):
    """vhat f64[2 * Nd * Npsi] (component-major) -> (vhat^{n+1}, p^{n+1})."""
    nd, npsi, ne, nphi = op.nd, op.npsi, conn.n_tri, op.nphi
    vh = np.asarray(vhat, dtype=np.float64).reshape(2, nd, npsi)
    vbar = np.stack([op.d2m(vh[c]) for c in (0, 1)])
    vb = vbar.reshape(2, ne, nphi)
    _, _, _, cs = SL.transport(conn, period, p, vb, vb, dt)
    H = op.helmholtz_matrix(nu * dt)
    vstar = np.stack([OP.direct_solve(H, op.apply_Mbar(cs[k].ravel())) for k in (0, 1)])
    vhs = np.stack([op.m2d(vstar[k]) for k in (0, 1)]).ravel()
    b = op.G.T @ vhs
    pr = OP.schur_solve_direct(op.schur_matrix(dt), b)
    return op.velocity_update(vhs, pr, dt * dt), pr
