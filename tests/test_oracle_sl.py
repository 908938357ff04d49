"""Pins of the oracle's semi-Lagrangian walk and transport (Sec. 2.5, eq.
lagrtrj, eq. intstage): the frame translations carry each shared edge onto
its neighbour's copy; under a uniform velocity (exact in every DG space) the
foot is x - dt v to rounding, in the cell a brute-force point location finds;
a zero velocity gives back the fields and a constant field stays constant
(the quadrature is exact to degree 2p + 1); and for the Taylor-Green velocity
the feet converge at first order to the exact characteristics (integrated by
SciPy to 1e-12) as the mesh is refined at fixed dt."""
import numpy as np
import pytest

from oracle import basis as B
from oracle import fields as OF
from oracle import mesh as OM
from oracle import sl as SL
from paper_2401_17806_gb300 import synth


def _conn(N, seed=3):
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    return OM.connectivity(xy, tri, per), per


def _tg(x, y):
    tp = 2.0 * np.pi
    return np.sin(tp * x) * np.cos(tp * y), -np.cos(tp * x) * np.sin(tp * y)


def test_frame_translations_match_shared_edges():
    conn, per = _conn(5)
    nbr, trans = SL.frames(conn, per)
    for t in range(conn.n_tri):
        for k in range(3):
            n = nbr[t, k]
            a, b = conn.tri_xy[t, k], conn.tri_xy[t, (k + 1) % 3]
            # the neighbour holds the same two vertices (opposite orientation)
            P = conn.tri_xy[n]
            for q in (a, b):
                d = np.abs(P - (q + trans[t, k])).max(axis=1)
                assert d.min() < 1e-12


@pytest.mark.parametrize("p", [1, 2])
def test_uniform_velocity_foot_and_cell(p):
    conn, per = _conn(6)
    nphi = B.n_phi(p)
    V = np.array([0.37, -0.21])
    vbar = np.zeros((2, conn.n_tri, nphi))
    vbar[0], vbar[1] = V[0], V[1]
    dt = 0.5  # about 2.5 cells per trajectory
    foot, cell, steps, _ = SL.transport(conn, per, p, vbar, np.zeros((0, conn.n_tri, nphi)), dt)
    pts, _ = SL.quadrature(p)
    X = B.triangle_points(conn.tri_xy, pts)
    assert steps.max() >= 3
    for i in range(conn.n_tri):
        for g in range(len(pts)):
            d = foot[i, g] - (X[i, g] - dt * V)
            assert np.abs(d - per * np.round(d / per)).max() < 1e-13
            hits = SL.locate(conn.tri_xy, per, foot[i, g])
            assert cell[i, g] in [h[0] for h in hits]


def test_forward_time_walks_the_other_way():
    """dt < 0: forward characteristics, the foot at x - dt v in a cell that
    contains it, crossing cells on the way."""
    conn, per = _conn(6)
    p = 1
    V = np.array([0.37, -0.21])
    vbar = np.zeros((2, conn.n_tri, B.n_phi(p)))
    vbar[0], vbar[1] = V[0], V[1]
    dt = -0.5
    foot, cell, steps, _ = SL.transport(conn, per, p, vbar, np.zeros((0, conn.n_tri, B.n_phi(p))), dt)
    pts, _ = SL.quadrature(p)
    X = B.triangle_points(conn.tri_xy, pts)
    assert steps.min() >= 1
    for i in range(conn.n_tri):
        for g in range(len(pts)):
            d = foot[i, g] - (X[i, g] - dt * V)
            assert np.abs(d - per * np.round(d / per)).max() < 1e-13
            assert cell[i, g] in [h[0] for h in SL.locate(conn.tri_xy, per, foot[i, g])]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_zero_velocity_gives_back_the_fields(p):
    conn, per = _conn(4)
    nphi = B.n_phi(p)
    c = synth.standard_normal((2, conn.n_tri, nphi), 5)
    foot, cell, steps, cstar = SL.transport(conn, per, p, np.zeros((2, conn.n_tri, nphi)), c, 0.3)
    assert steps.max() == 0 and np.array_equal(cell, np.repeat(np.arange(conn.n_tri)[:, None], cell.shape[1], 1))
    np.testing.assert_allclose(cstar, c, rtol=0, atol=1e-12)


def test_constant_field_stays_constant():
    conn, per = _conn(6)
    p = 2
    Xn = OF.main_nodes(conn, p)
    vbar = np.stack(_tg(Xn[..., 0], Xn[..., 1]))
    c = np.full((1, conn.n_tri, B.n_phi(p)), 2.5)
    _, _, steps, cstar = SL.transport(conn, per, p, vbar, c, 0.2)
    assert steps.max() >= 2
    np.testing.assert_allclose(cstar, 2.5, rtol=0, atol=1e-12)


def test_feet_converge_to_the_characteristics():
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    p, dt = 2, 0.2
    errs = []
    for N in (8, 16, 32):
        conn, per = _conn(N)
        Xn = OF.main_nodes(conn, p)
        vbar = np.stack(_tg(Xn[..., 0], Xn[..., 1]))
        nbr, trans = SL.frames(conn, per)

        def velocity(cell, xi, eta):
            return vbar[:, cell, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]

        pts, _ = SL.quadrature(p)
        X = B.triangle_points(conn.tri_xy, pts)
        rng = np.random.default_rng(0)
        e = []
        for _ in range(60):
            i, g = int(rng.integers(conn.n_tri)), int(rng.integers(len(pts)))
            xf, _, _ = SL.walk(conn.tri_xy, nbr, trans, velocity, X[i, g], i, dt)
            ex = solve_ivp(lambda t, z: -np.array(_tg(z[0], z[1])), (0.0, dt), X[i, g], rtol=1e-12, atol=1e-14)
            d = xf - ex.y[:, -1]
            e.append(np.abs(d - per * np.round(d / per)).max())
        errs.append(np.mean(e))
    assert errs[0] < 0.05
    assert errs[0] / errs[1] >= 1.5 and errs[1] / errs[2] >= 1.5, errs
