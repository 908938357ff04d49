"""Pins of the oracle's first-order semi-Lagrangian Navier-Stokes step
(oracle.ns): every step leaves a discretely divergence-free dual velocity
(eq. nc.1); a uniform velocity is an exact steady solution; and the decaying
Taylor-Green vortex (exact: the initial field times exp(-8 pi^2 nu t) on the
unit torus, its convection being a pure gradient) is approached at first
order in dt."""
import numpy as np

from oracle import assemble as OA
from oracle import fields as OF
from oracle import mesh as OM
from oracle import ns as NS
from oracle import operators as OP
from paper_2401_17806_gb300 import synth


def _setup(N, p, seed=3):
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    conn = OM.connectivity(xy, tri, per)
    return conn, per, OP.Operators(OA.assemble(xy, tri, per, p, conn=conn))


def _tg(x, y):
    tp = 2.0 * np.pi
    return np.sin(tp * x) * np.cos(tp * y), -np.cos(tp * x) * np.sin(tp * y)


def test_uniform_velocity_is_steady_and_steps_are_divergence_free():
    conn, per, op = _setup(6, 2)
    v = np.concatenate([np.full(op.nd * op.npsi, 0.3), np.full(op.nd * op.npsi, -0.2)])
    v1, pr = NS.ns_step(op, conn, per, 2, v, 0.4, 0.01)
    np.testing.assert_allclose(v1, v, rtol=0, atol=1e-12)
    Xd = OF.dual_nodes(conn, 2, per)
    u0, w0 = _tg(Xd[..., 0], Xd[..., 1])
    v1, _ = NS.ns_step(op, conn, per, 2, np.stack([u0, w0]).ravel() + 0.05 * synth.standard_normal(
        2 * op.nd * op.npsi, 4), 0.05, 0.01)
    assert np.linalg.norm(op.G.T @ v1) <= 1e-12 * np.linalg.norm(v1)


def test_taylor_green_first_order_in_time():
    conn, per, op = _setup(12, 2)
    nu, T = 0.01, 0.1
    Xd = OF.dual_nodes(conn, 2, per)
    u0, w0 = _tg(Xd[..., 0], Xd[..., 1])
    v0 = np.stack([u0, w0]).ravel()
    ref = np.exp(-8.0 * np.pi ** 2 * nu * T) * v0
    errs = []
    for n in (2, 4, 8):
        v = v0.copy()
        for _ in range(n):
            v, _ = NS.ns_step(op, conn, per, 2, v, T / n, nu)
        errs.append(np.linalg.norm(v - ref) / np.linalg.norm(ref))
    assert errs[0] < 0.1
    assert errs[0] / errs[1] >= 1.8 and errs[1] / errs[2] >= 1.8, errs
