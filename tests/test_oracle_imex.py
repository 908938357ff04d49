"""Pins of the oracle's IMEX tableaux (App. A) and stage trajectories.

The tableaux satisfy the order conditions of their formal orders (1, 2, 3)
to the six printed digits, the explicit row sums give the printed c~, and
the implicit ones are stiffly accurate.  The stage-trajectory scheme
integrates the exact Taylor-Green characteristics (SciPy to 1e-12) at
orders 1, 2, 3.  With the DG velocity: a uniform velocity gives the exact
feet (to the weights' printed sum) in the cells a brute-force point location
finds, R = 0 is one straight Euler segment from the Gauss point, a zero
velocity gives the fields back, and the sampled feet still converge at
orders 2 and 3."""
import numpy as np
import pytest

from oracle import basis as B
from oracle import fields as OF
from oracle import imex as IM
from oracle import mesh as OM
from oracle import operators as OP
from oracle import sl as SL
from paper_2401_17806_gb300 import synth

TP = 2.0 * np.pi


def _tg(x, y):
    return np.sin(TP * x) * np.cos(TP * y), -np.cos(TP * x) * np.sin(TP * y)


def test_tableau_order_conditions():
    for R, order in ((0, 1), (1, 2), (2, 3)):
        At, bt, ct, A, b, c = IM.tableau(R)
        tol = 2e-6 if R == 2 else 1e-14
        assert np.allclose(np.triu(At), 0.0)
        for W, C, M in ((bt, ct, At), (b, c, A)):
            assert abs(W.sum() - 1.0) <= tol
            if order >= 2:
                assert abs(W @ C - 0.5) <= tol
            if order >= 3:
                assert abs(W @ C ** 2 - 1.0 / 3.0) <= tol
                assert abs(W @ (M @ C) - 1.0 / 6.0) <= tol
        np.testing.assert_array_equal(bt, b)  # the semi-implicit class: one set of weights
        if R >= 1:
            np.testing.assert_array_equal(A[-1], b)  # stiffly accurate
    # the printed c~ and c columns
    g1 = 1.0 - 1.0 / np.sqrt(2.0)
    np.testing.assert_allclose(IM.tableau(1)[2], [0.0, 1.0 / (2.0 * g1)], rtol=0, atol=1e-15)
    np.testing.assert_allclose(IM.tableau(1)[5], [g1, 1.0], rtol=0, atol=1e-15)
    # (each printed entry is rounded to 5e-7: a row of three is within 1.5e-6)
    np.testing.assert_allclose(IM.tableau(2)[2], [0.0, 0.435866, 0.717933, 1.0], rtol=0, atol=1.5e-6)
    np.testing.assert_allclose(IM.tableau(2)[5], [0.435866, 0.435866, 0.717933, 1.0], rtol=0, atol=1.5e-6)


def _exact_foot(x, dt):
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    r = solve_ivp(lambda t, z: -np.array(_tg(z[0], z[1])), (0.0, dt), x, rtol=1e-12, atol=1e-14)
    return r.y[:, -1]


@pytest.mark.parametrize("R", [0, 1, 2])
def test_stage_trajectories_reach_their_order(R):
    rng = np.random.default_rng(4)
    pts = rng.random((12, 2))
    errs = []
    dts = (0.08, 0.04, 0.02)
    for dt in dts:
        e = [np.abs(IM.rk_foot(lambda y: np.array(_tg(*y)), x, dt, R) - _exact_foot(x, dt)).max() for x in pts]
        errs.append(max(e))
    # one step: local error O(dt^(R+2))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > R + 2 - 0.35) and np.all(orders < R + 2 + 0.6), orders


def _conn(N, seed=3):
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    return OM.connectivity(xy, tri, per), per


@pytest.mark.parametrize("R", [0, 1, 2])
def test_uniform_velocity_feet_and_cells(R):
    conn, per = _conn(6)
    p = 1
    V = np.array([0.37, -0.21])
    vbar = np.zeros((2, conn.n_tri, B.n_phi(p)))
    vbar[0], vbar[1] = V[0], V[1]
    dt = 0.5
    foot, cell, steps, _ = IM.rk_transport(conn, per, p, vbar, np.zeros((0, conn.n_tri, B.n_phi(p))), dt, R)
    sb = IM.tableau(R)[1].sum()
    X = B.triangle_points(conn.tri_xy, SL.quadrature(p)[0])
    assert steps.max() >= 3
    for i in range(conn.n_tri):
        for g in range(X.shape[1]):
            d = foot[i, g] - (X[i, g] - dt * sb * V)
            assert np.abs(d - per * np.round(d / per)).max() < 1e-13
            assert cell[i, g] in [h[0] for h in SL.locate(conn.tri_xy, per, foot[i, g])]


def test_euler_tableau_is_one_straight_segment():
    conn, per = _conn(7)
    p = 2
    Xn = OF.main_nodes(conn, p)
    vbar = np.stack(_tg(Xn[..., 0], Xn[..., 1]))
    dt = 0.15
    foot, cell, _, _ = IM.rk_transport(conn, per, p, vbar, np.zeros((0, conn.n_tri, B.n_phi(p))), dt, 0)
    X = B.triangle_points(conn.tri_xy, SL.quadrature(p)[0])
    phi = B.eval_phi(p, SL.quadrature(p)[0])  # [Ng, Nphi]
    for i in range(conn.n_tri):
        v0 = vbar[:, i, :] @ phi.T  # [2, Ng] the velocity at the Gauss points of i
        for g in range(X.shape[1]):
            d = foot[i, g] - (X[i, g] - dt * v0[:, g])
            assert np.abs(d - per * np.round(d / per)).max() < 1e-13


@pytest.mark.parametrize("R", [1, 2])
def test_zero_velocity_and_constant_field(R):
    conn, per = _conn(4)
    p = 3
    nphi = B.n_phi(p)
    c = synth.standard_normal((2, conn.n_tri, nphi), 5)
    _, _, steps, cs = IM.rk_transport(conn, per, p, np.zeros((2, conn.n_tri, nphi)), c, 0.3, R)
    assert steps.max() == 0
    np.testing.assert_allclose(cs, c, rtol=0, atol=1e-12)
    Xn = OF.main_nodes(conn, p)
    vbar = np.stack(_tg(Xn[..., 0], Xn[..., 1]))
    _, _, steps, cs = IM.rk_transport(conn, per, p, vbar, np.full((1, conn.n_tri, nphi), 2.5), 0.2, R)
    assert steps.max() >= 2
    np.testing.assert_allclose(cs, 2.5, rtol=0, atol=1e-12)


@pytest.mark.parametrize("R", [1, 2])
def test_dg_velocity_feet_converge_at_order(R):
    """Sampled Gauss points of a 32 x 32 mesh, p = 4: the DG velocity's own
    error (h^5) stays below the time error at these dt."""
    conn, per = _conn(32)
    p = 4
    Xn = OF.main_nodes(conn, p)
    vbar = np.stack(_tg(Xn[..., 0], Xn[..., 1]))
    nbr, trans, back = SL.frames(conn, per)
    X = B.triangle_points(conn.tri_xy, SL.quadrature(p)[0])
    At, bt = IM.tableau(R)[:2]

    def vel(cell, y):
        _, xi, eta = SL.barycentric(conn.tri_xy[cell], y)
        return vbar[:, cell, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]

    rng = np.random.default_rng(1)
    sample = [(int(rng.integers(conn.n_tri)), int(rng.integers(X.shape[1]))) for _ in range(10)]
    errs = []
    for dt in (0.16, 0.08, 0.04):
        e = []
        for i, g in sample:
            V = []
            for s in range(len(bt)):
                d = -dt * sum(At[s, j] * V[j] for j in range(s)) if s else np.zeros(2)
                y, cy, _ = IM.locate_from(conn.tri_xy, nbr, trans, back, X[i, g], i, d)
                V.append(vel(cy, y))
            xf = X[i, g] - dt * sum(bt[j] * V[j] for j in range(len(bt)))
            dd = xf - _exact_foot(X[i, g], dt)
            e.append(np.abs(dd - per * np.round(dd / per)).max())
        errs.append(max(e))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > R + 2 - 0.5), (errs, orders)


def _advdiff_setup(N, p, seed=3):
    from oracle import assemble as OA
    from oracle import operators as OP
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    conn = OM.connectivity(xy, tri, per)
    return conn, per, OP.Operators(OA.assemble(xy, tri, per, p, conn=conn))


@pytest.mark.parametrize("R", [0, 1, 2])
def test_advdiff_without_velocity_is_the_dirk(R):
    """v = 0: one step is the implicit Runge-Kutta scheme (A, b) applied to
    Mbar dC/dt = -alpha K C, written out with dense matrices."""
    conn, per, ops = _advdiff_setup(5, 2)
    p, dt, alpha = 2, 0.07, 0.3
    n = conn.n_tri * B.n_phi(p)
    C0 = synth.standard_normal(n, 21)
    got = IM.advdiff_step(ops, conn, per, p, np.zeros((2, conn.n_tri, B.n_phi(p))), C0, dt, alpha, R)
    A = IM.tableau(R)[3]
    Mb = ops.helmholtz_matrix(0.0).toarray()
    L = -alpha * np.linalg.solve(Mb, ops.K().toarray())
    U = []
    for s in range(len(A)):
        rhs = C0 + dt * sum(A[s, j] * (L @ U[j]) for j in range(s))
        U.append(np.linalg.solve(np.eye(n) - dt * A[s, s] * L, rhs))
    np.testing.assert_allclose(got, U[-1], rtol=0, atol=1e-11 * np.abs(U[-1]).max())


@pytest.mark.parametrize("R", [1, 2])
def test_advdiff_without_diffusion_is_the_stage_transport(R):
    conn, per, ops = _advdiff_setup(5, 2)
    p, dt = 2, 0.15
    Xn = OF.main_nodes(conn, p)
    vbar = np.stack(_tg(Xn[..., 0], Xn[..., 1]))
    C0 = synth.standard_normal(conn.n_tri * B.n_phi(p), 22)
    got = IM.advdiff_step(ops, conn, per, p, vbar, C0, dt, 0.0, R)
    _, _, _, cs = IM.rk_transport(conn, per, p, vbar, C0.reshape(1, conn.n_tri, -1), dt, R)
    np.testing.assert_allclose(got, cs.ravel(), rtol=0, atol=1e-12 * np.abs(cs).max())


def test_advdiff_keeps_a_constant():
    conn, per, ops = _advdiff_setup(5, 3)
    p = 3
    Xn = OF.main_nodes(conn, p)
    vbar = np.stack(_tg(Xn[..., 0], Xn[..., 1]))
    got = IM.advdiff_step(ops, conn, per, p, vbar, np.full(conn.n_tri * B.n_phi(p), 1.7), 0.1, 0.2, 2)
    np.testing.assert_allclose(got, 1.7, rtol=0, atol=1e-11)


def test_advdiff_local_order_with_a_constant_velocity():
    """C = exp(-alpha |k|^2 t) sin(k.(x - V t)) exactly; one R = 1 step on a
    16 x 16 mesh, p = 4: the local error falls faster than dt^2.3 from dt =
    0.1 to 0.05 (2.53 measured; with the shift weight as printed it falls as
    dt^1.72, the first-order scheme)."""
    conn, per, ops = _advdiff_setup(16, 4)
    p, alpha = 4, 0.2
    V = np.array([0.8, 0.5])
    k = np.array([TP, 0.0])
    lam = alpha * (k @ k)
    Xn = OF.main_nodes(conn, p)
    vbar = np.zeros((2, conn.n_tri, B.n_phi(p)))
    vbar[0], vbar[1] = V[0], V[1]

    def exact(t):
        return (np.exp(-lam * t) * np.sin(Xn[..., 0] * k[0] + Xn[..., 1] * k[1] - (k @ V) * t)).ravel()

    errs = [np.abs(IM.advdiff_step(ops, conn, per, p, vbar, exact(0.0), dt, alpha, 1) - exact(dt)).max()
            for dt in (0.1, 0.05)]
    assert np.log2(errs[0] / errs[1]) > 2.3, errs


def _tg_dual(conn, per, p):
    Xd = OF.dual_nodes(conn, p, per)
    return np.stack(_tg(Xd[..., 0], Xd[..., 1])).ravel()


@pytest.mark.parametrize("R", [0, 1, 2])
def test_ns_imex_uniform_velocity_and_divergence(R):
    """A uniform velocity is an exact steady solution; every step leaves a
    discretely divergence-free velocity (G^T v = 0 to the direct solves)."""
    conn, per, ops = _advdiff_setup(5, 2)
    nv = ops.nd * ops.npsi
    U = np.concatenate([np.full(nv, 0.3), np.full(nv, -0.2)])
    vu, _ = IM.ns_imex_step(ops, conn, per, 2, U, 0.1, 0.01, R)
    np.testing.assert_allclose(vu, U, rtol=0, atol=1e-13)
    v0 = _tg_dual(conn, per, 2)
    v1, _ = IM.ns_imex_step(ops, conn, per, 2, v0, 0.05, 0.01, R)
    assert np.linalg.norm(ops.G.T @ v1) <= 1e-12 * np.linalg.norm(v1)


def test_ns_imex_second_order_on_the_taylor_green_vortex():
    """The decaying Taylor-Green vortex (exact decay exp(-8 pi^2 nu t)) at
    t = 0.1 on a 10 x 10 mesh, p = 3: the R = 1 error falls faster than dt^2.2
    from 2 to 4 steps (2.6 measured), where R = 0 falls as dt^1."""
    conn, per, ops = _advdiff_setup(10, 3)
    nu, T = 0.01, 0.1
    v0 = _tg_dual(conn, per, 3)
    ref = v0 * np.exp(-8.0 * np.pi ** 2 * nu * T)
    errs = []
    for n in (2, 4):
        v = v0.copy()
        for _ in range(n):
            v, _ = IM.ns_imex_step(ops, conn, per, 3, v, T / n, nu, 1)
        errs.append(np.linalg.norm(v - ref) / np.linalg.norm(ref))
    assert np.log2(errs[0] / errs[1]) > 2.2, errs


def _translate_project(conn, per, p, delta):
    """Brute-force matrix of c -> proj[c(x + delta)] for main-grid scalar
    fields (eq. intstage projection of the field evaluated at the Gauss points
    moved by delta, each point located by testing every triangle)."""
    from oracle.assemble import main_mass
    pts, w = SL.quadrature(p)
    nphi = B.n_phi(p)
    X = B.triangle_points(conn.tri_xy, pts)
    phi_g = B.eval_phi(p, pts)                          # [ng, nphi]
    Mbar, _ = main_mass(conn, p)
    n = conn.n_tri * nphi
    T = np.zeros((n, n))
    for i in range(conn.n_tri):
        e1 = conn.tri_xy[i, 1] - conn.tri_xy[i, 0]
        e2 = conn.tri_xy[i, 2] - conn.tri_xy[i, 0]
        absJ = abs(e1[0] * e2[1] - e1[1] * e2[0])
        E = np.zeros((len(w), n))                       # point values as a function of c
        for g in range(len(w)):
            cell, y = SL.locate(conn.tri_xy, per, X[i, g] + delta)[0]
            _, xi, eta = SL.barycentric(conn.tri_xy[cell], y)
            E[g, cell * nphi:(cell + 1) * nphi] = B.eval_phi(p, np.array([[xi, eta]]))[0]
        rows = np.linalg.solve(Mbar[i], (phi_g.T * w) @ E * absJ)
        T[i * nphi:(i + 1) * nphi] = rows
    return T


@pytest.mark.parametrize("R", [1, 2])
def test_ns_imex_linearised_about_a_uniform_flow_is_the_stage_recurrence(R):
    """About a uniform velocity U every trajectory is the straight line
    x - tau dt U, so the step's derivative in a perturbation w is linear
    algebra: per stage s (implicit tableau (A, c) of App. A)
      w^I_s = T(c_s) w^n + sum_{j<s} dt a_{s,j} T(c_s - c_j) H_j,
      (Mbar + a_ss dt nu K) w* = Mbar w^I_s,  w^_* = L_md w*,
      S pi = G^T w^_*,  w^_s = w^_* - (a_ss dt)^2 Mhat^-1 G pi,
      H_s = L_dm[(w^_s - L_md w^I_s) / (a_ss dt)],
    with T(tau) the brute-force translation by -tau dt U and projection.
    The oracle's step at U + eps w must agree with U + eps L(w) to O(eps)
    (measured 1e-7 at eps = 1e-7, allowed 1e-5):
    a wrong shift c_s - c_j or a wrong stage flux changes L(w) at O(1), a
    wrong a_{s,j} by about its own relative error (1e-4 in one row is
    detected)."""
    conn, per, ops = _advdiff_setup(4, 2)
    p, dt, nu = 2, 0.05, 0.02
    U = np.array([0.3, -0.2])
    nv = ops.nd * ops.npsi
    Uhat = np.concatenate([np.full(nv, U[0]), np.full(nv, U[1])])
    w = synth.standard_normal(2 * nv, 17)
    eps = 1e-7
    v1, _ = IM.ns_imex_step(ops, conn, per, p, Uhat + eps * w, dt, nu, R)
    numeric = (v1 - Uhat) / eps
    _, _, _, A, _, c = IM.tableau(R)
    ns = len(c)
    Tm = {}

    def T(tau):
        key = round(float(tau), 15)
        if key not in Tm:
            Tm[key] = _translate_project(conn, per, p, -tau * dt * U)
        return Tm[key]

    wh = w.reshape(2, nv)
    wn = np.stack([ops.d2m(wh[k]) for k in range(2)])
    Hs = []
    ws = None
    for s in range(ns):
        wI = np.stack([T(c[s]) @ wn[k] + sum(dt * A[s, j] * (T(c[s] - c[j]) @ Hs[j][k]) for j in range(s))
                       for k in range(2)])
        h = A[s, s] * dt
        Hm = ops.helmholtz_matrix(nu * h)
        wst = np.stack([OP.direct_solve(Hm, ops.apply_Mbar(wI[k])) for k in range(2)])
        whs = np.concatenate([ops.m2d(wst[k]) for k in range(2)])
        pi = OP.schur_solve_direct(ops.schur_matrix(h), ops.G.T @ whs)
        ws = ops.velocity_update(whs, pi, h * h).reshape(2, nv)
        Hh = (ws - np.stack([ops.m2d(wI[k]) for k in range(2)])) / h
        Hs.append(np.stack([ops.d2m(Hh[k]) for k in range(2)]))
    lin = ws.ravel()
    print("LINEARISED", R, np.linalg.norm(numeric - lin) / np.linalg.norm(lin))
    assert np.linalg.norm(numeric - lin) <= 1e-5 * np.linalg.norm(lin), np.linalg.norm(numeric - lin) / np.linalg.norm(lin)
