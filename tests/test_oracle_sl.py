"""Pins of the oracle's semi-Lagrangian walk and transport (Sec. 2.5, eq.
lagrtrj, eq. intstage): the frame translations carry each shared edge onto
its neighbour's copy; under a uniform velocity (exact in every DG space) the
foot is x - dt v to rounding, in the cell a brute-force point location finds;
a zero velocity gives back the fields and a constant field stays constant
(the quadrature is exact to degree 2p + 1); and for the Taylor-Green velocity
the feet converge at first order to the exact characteristics (integrated by
SciPy to 1e-12) as the mesh is refined at fixed dt.  Held trajectories: on a
source line (the velocity of two neighbours points away from their shared
edge) every backward ray that meets the edge stops at the point where it
meets it, after crossing into the neighbour and bouncing back, whatever the
time left."""
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
    nbr, trans, back = SL.frames(conn, per)
    for t in range(conn.n_tri):
        for k in range(3):
            n = nbr[t, k]
            a, b = conn.tri_xy[t, k], conn.tri_xy[t, (k + 1) % 3]
            # the neighbour holds the same two vertices (opposite orientation)
            P = conn.tri_xy[n]
            for q in (a, b):
                d = np.abs(P - (q + trans[t, k])).max(axis=1)
                assert d.min() < 1e-12
            # the neighbour sees the same edge at local index back[t, k], and back again
            kb = back[t, k]
            assert nbr[n, kb] == t and back[n, kb] == k
            np.testing.assert_allclose(trans[n, kb], -trans[t, k], rtol=0, atol=0)


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
        nbr, trans, back = SL.frames(conn, per)

        def velocity(cell, xi, eta):
            return vbar[:, cell, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]

        pts, _ = SL.quadrature(p)
        X = B.triangle_points(conn.tri_xy, pts)
        rng = np.random.default_rng(0)
        e = []
        for _ in range(60):
            i, g = int(rng.integers(conn.n_tri)), int(rng.integers(len(pts)))
            xf, _, _ = SL.walk(conn.tri_xy, nbr, trans, back, velocity, X[i, g], i, dt)
            ex = solve_ivp(lambda t, z: -np.array(_tg(z[0], z[1])), (0.0, dt), X[i, g], rtol=1e-12, atol=1e-14)
            d = xf - ex.y[:, -1]
            e.append(np.abs(d - per * np.round(d / per)).max())
        errs.append(np.mean(e))
    assert errs[0] < 0.05
    assert errs[0] / errs[1] >= 1.5 and errs[1] / errs[2] >= 1.5, errs


def source_line(conn, per, p, j, speed=1.0):
    """Velocity zero except in the two neighbours of edge j, where it is
    constant and points away from j (along l's outward normal n of j: -n in
    l, +n in r).  Returns vbar [2, Ne, Nphi] and the expected foot of every
    Gauss point of l and r whose perpendicular onto the edge's line meets the
    edge (inside by a margin): the perpendicular foot, in the start cell's
    frame (the walk crosses, bounces back and is held there)."""
    nphi = B.n_phi(p)
    l, r = conn.lr[j]
    kl, kr = int(conn.loc[j, 0]), int(conn.loc[j, 1])
    a, b = conn.tri_xy[l, kl], conn.tri_xy[l, (kl + 1) % 3]
    e = b - a
    n = np.array([e[1], -e[0]]) / np.linalg.norm(e)  # outward of l (counter-clockwise)
    vbar = np.zeros((2, conn.n_tri, nphi))
    vbar[:, l, :] = (-speed * n)[:, None]
    vbar[:, r, :] = (speed * n)[:, None]
    _, trans, _ = SL.frames(conn, per)
    pts, _ = SL.quadrature(p)
    X = B.triangle_points(conn.tri_xy, pts)
    want = {}
    for t in (l, r):
        # the edge in t's frame
        at = a if t == l else a - trans[r, kr]
        for g in range(len(pts)):
            x = X[t, g]
            q = x - ((x - at) @ n) * n
            u = (q - at) @ e / (e @ e)
            if 1e-6 < u < 1 - 1e-6:
                want[(t, g)] = q
    return vbar, want


@pytest.mark.parametrize("p", [1, 3])
def test_source_line_holds_trajectories_on_the_edge(p):
    conn, per = _conn(6)
    hits = 0
    for j in (0, 7, conn.n_edge - 1):
        vbar, want = source_line(conn, per, p, j)
        for dt in (0.5, 5.0):  # the time left is dropped
            foot, cell, steps, _ = SL.transport(conn, per, p, vbar, np.zeros((0, conn.n_tri, B.n_phi(p))), dt)
            for (t, g), q in want.items():
                assert cell[t, g] == t and steps[t, g] == 2
                np.testing.assert_allclose(foot[t, g], q, rtol=0, atol=1e-13)
                hits += 1
    assert hits >= 12


def test_source_line_would_not_end_without_the_hold():
    """The same configuration walked without the hold rule (back indices that
    never match) crosses the edge back and forth until the cap."""
    conn, per = _conn(6)
    p = 1
    vbar, want = source_line(conn, per, p, 3)
    nbr, trans, _ = SL.frames(conn, per)
    never = np.full_like(nbr, -2)
    (t, g), _ = next(iter(want.items()))
    X = B.triangle_points(conn.tri_xy, SL.quadrature(p)[0])

    def velocity(cell, xi, eta):
        return vbar[:, cell, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]

    with pytest.raises(SL.WalkError):
        SL.walk(conn.tri_xy, nbr, trans, never, velocity, X[t, g], t, 0.5, max_steps=200)
