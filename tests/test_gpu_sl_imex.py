"""GPU parity of the stage-trajectory transport (dgsl_sl_transport_imex:
the explicit IMEX tableaux of App. A for the characteristic equation, every
stage point and the foot reached along straight segments, eq. intstage at
the feet) against the oracle: cells exact, feet and transported fields to
1e-11, for R = 0, 1, 2 and p = 1..4; full size on sampled trajectories; the
feet's order of convergence in dt; arguments.  The kernel walks each stage
point from the previous one, the oracle from the Gauss point (the printed
definition): the cells crossed agree for R = 0 (one segment) and are
compared only there."""
import numpy as np
import pytest

from oracle import basis as B
from oracle import imex as IM
from oracle import sl as SL
from oracle.assemble import main_mass
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import dev, to_internal, to_natural  # noqa: E402
from test_gpu_sl import _setup, _tg  # noqa: E402


def _run(op, R, dt, vbar, fields):
    """As test_gpu_sl._run, through dgsl_sl_transport_imex."""
    from paper_2401_17806_gb300 import dgsl
    perm = op.maps()["perm"]
    ng = dgsl.sl_quadrature(op.p)[1].size
    nt = op.n_tri * ng
    foot = torch.zeros(2 * nt, dtype=torch.float64, device="cuda")
    cell = torch.zeros(nt, dtype=torch.int32, device="cuda")
    steps = torch.zeros(nt, dtype=torch.int32, device="cuda")
    nf = len(fields)
    c = dev(np.concatenate([to_internal(f, perm, op.n_phi) for f in fields])) if nf else None
    cs = torch.zeros_like(c) if nf else None
    vb = dev(np.concatenate([to_internal(v, perm, op.n_phi) for v in vbar]))
    op.dgsl_sl_transport_imex(R, dt, vb, c, cs, nf, foot, cell, steps)
    torch.cuda.synchronize()
    f_i = foot.cpu().numpy().reshape(op.n_tri, ng, 2)
    c_i = cell.cpu().numpy().reshape(op.n_tri, ng)
    s_i = steps.cpu().numpy().reshape(op.n_tri, ng)
    f_n, c_n, s_n = np.empty_like(f_i), np.empty_like(c_i), np.empty_like(s_i)
    f_n[perm], c_n[perm], s_n[perm] = f_i, perm[c_i], s_i
    cstar = (np.stack([to_natural(v, perm, op.n_phi).reshape(op.n_tri, op.n_phi)
                       for v in cs.cpu().numpy().reshape(nf, -1)]) if nf else None)
    return f_n, c_n, s_n, cstar


@pytest.mark.parametrize("R,N,p", [(0, 7, 2), (1, 7, 1), (1, 8, 3), (2, 9, 2), (2, 6, 4)])
def test_stage_transport_parity(dgsl_lib, R, N, p):
    op, conn, per, perm = _setup(N, p, 40 + N)
    X = B.triangle_points(conn.tri_xy, B.nodes(p))
    vbar = np.stack(_tg(X[..., 0], X[..., 1])).reshape(2, -1)
    fields = [synth.standard_normal(op.n_dof, 70 + k) for k in range(2)]
    dt = 0.2
    foot, cell, steps, cstar = _run(op, R, dt, vbar, fields)
    fo, co, so, cso = IM.rk_transport(conn, per, p, vbar.reshape(2, conn.n_tri, -1),
                                      np.stack([f.reshape(conn.n_tri, -1) for f in fields]), dt, R)
    assert so.max() >= 2
    assert np.array_equal(cell, co)
    if R == 0:
        assert np.array_equal(steps, so)
    np.testing.assert_allclose(foot, fo, rtol=0, atol=1e-11)
    np.testing.assert_allclose(cstar, cso, rtol=0, atol=1e-11 * np.abs(cso).max())


def test_uniform_velocity_and_arguments(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op, conn, per, perm = _setup(6, 2, 5)
    V = np.array([0.37, -0.21])
    vbar = [np.full(op.n_dof, V[0]), np.full(op.n_dof, V[1])]
    X = B.triangle_points(conn.tri_xy, SL.quadrature(2)[0])
    for R in (0, 1, 2):
        foot, cell, steps, _ = _run(op, R, 0.5, vbar, [])
        d = foot - (X - 0.5 * IM.tableau(R)[1].sum() * V)
        assert np.abs(d - per * np.round(d / per)).max() < 1e-13
        assert steps.max() >= 3
    vb = dev(np.concatenate(vbar))
    with pytest.raises(dgsl.DgslError) as e:
        op.dgsl_sl_transport_imex(3, 0.1, vb)
    assert e.value.code == dgsl.EINVAL
    with pytest.raises(dgsl.DgslError) as e:
        op.dgsl_sl_transport_imex(1, 1.0e6, vb)  # segments of ~10^8 cells: stopped at the cap
    assert e.value.code == dgsl.ENOTCONV
    op.dgsl_sl_transport_imex(1, 0.3, vb)  # the context is still usable


def _exact_foot(x, dt):
    solve_ivp = pytest.importorskip("scipy.integrate").solve_ivp
    r = solve_ivp(lambda t, z: -np.array(_tg(z[0], z[1])), (0.0, dt), x, rtol=1e-12, atol=1e-14)
    return r.y[:, -1]


@pytest.mark.parametrize("R", [0, 1, 2])
def test_feet_order_in_dt(dgsl_lib, R):
    """64 x 64, p = 4 (the DG velocity's own error is below the time error):
    sampled feet against the exact characteristics; one step's error falls as
    dt^(R+2)."""
    op, conn, per, perm = _setup(64, 4, 2)
    X = B.triangle_points(conn.tri_xy, B.nodes(4))
    vbar = np.stack(_tg(X[..., 0], X[..., 1])).reshape(2, -1)
    P = B.triangle_points(conn.tri_xy, SL.quadrature(4)[0])
    rng = np.random.default_rng(9)
    sample = [(int(rng.integers(conn.n_tri)), int(rng.integers(P.shape[1]))) for _ in range(16)]
    errs = []
    for dt in (0.16, 0.08, 0.04):
        foot, _, _, _ = _run(op, R, dt, vbar, [])
        e = []
        for i, g in sample:
            d = foot[i, g] - _exact_foot(P[i, g], dt)
            e.append(np.abs(d - per * np.round(d / per)).max())
        errs.append(max(e))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > R + 2 - 0.5), (errs, orders)


def test_stage_transport_full_size_sampled(dgsl_lib):
    """256 x 256, p = 3, R = 2, dt = 0.01: sampled trajectories and the
    transported velocity of sampled triangles against the oracle's stages."""
    N, p, dt, R = 256, 3, 0.01, 2
    op, conn, per, perm = _setup(N, p, 0)
    X = B.triangle_points(conn.tri_xy, B.nodes(p))
    vbar = np.stack(_tg(X[..., 0], X[..., 1])).reshape(2, -1)
    foot, cell, steps, cstar = _run(op, R, dt, vbar, [vbar[0], vbar[1]])
    nbr, trans, back = SL.frames(conn, per)
    vb = vbar.reshape(2, conn.n_tri, -1)
    At, bt = IM.tableau(R)[:2]

    def vel(c, y):
        _, xi, eta = SL.barycentric(conn.tri_xy[c], y)
        return vb[:, c, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]

    pts, w = SL.quadrature(p)
    P = B.triangle_points(conn.tri_xy, pts)
    rng = np.random.default_rng(5)
    tris = rng.choice(conn.n_tri, 30, replace=False)
    vals = np.zeros((2, len(tris), len(w)))
    for a, i in enumerate(tris):
        for g in range(len(w)):
            V, nst = [], 0
            for s in range(len(bt)):
                d = -dt * sum(At[s, j] * V[j] for j in range(s)) if s else np.zeros(2)
                y, cy, st = IM.locate_from(conn.tri_xy, nbr, trans, back, P[i, g], i, d)
                nst += st
                V.append(vel(cy, y))
            d = -dt * sum(bt[j] * V[j] for j in range(len(bt)))
            xf, cf, st = IM.locate_from(conn.tri_xy, nbr, trans, back, P[i, g], i, d)
            assert cf == cell[i, g]
            assert np.abs(xf - foot[i, g]).max() < 1e-11
            _, xi, eta = SL.barycentric(conn.tri_xy[cf], xf)
            vals[:, a, g] = vb[:, cf, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]
    assert steps.mean() > 2.0

    class Sub:
        tri_xy = conn.tri_xy[tris]

    Mbar, area2 = main_mass(Sub, p)
    phi_g = B.eval_phi(p, pts)
    for f in range(2):
        rhs = np.einsum("gl,g,ag->al", phi_g, w, vals[f]) * np.abs(area2)[:, None]
        ref = np.linalg.solve(Mbar, rhs[..., None])[..., 0]
        np.testing.assert_allclose(cstar[f][tris], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_smallest_mesh_long_trajectories(dgsl_lib):
    """3 x 3 mesh (18 triangles), dt = 0.9: trajectories wrap around the
    torus several times through the few periodic neighbours.  The walk of
    Sec. 2.5 and the stage trajectories of R = 0, 1, 2 agree with the oracle."""
    from test_gpu_sl import _run as run_walk
    op, conn, per, perm = _setup(3, 2, 1)
    X = B.triangle_points(conn.tri_xy, B.nodes(2))
    vbar = np.stack(_tg(X[..., 0], X[..., 1])).reshape(2, -1)
    fields = [synth.standard_normal(op.n_dof, 5)]
    nf = np.stack([f.reshape(conn.n_tri, -1) for f in fields])
    dt = 0.9
    foot, cell, steps, cstar = run_walk(op, dt, vbar, fields)
    fo, co, so, cso = SL.transport(conn, per, 2, vbar.reshape(2, conn.n_tri, -1), nf, dt)
    assert so.max() >= 10
    assert np.array_equal(cell, co) and np.array_equal(steps, so)
    np.testing.assert_allclose(foot, fo, rtol=0, atol=1e-11)
    np.testing.assert_allclose(cstar, cso, rtol=0, atol=1e-11 * np.abs(cso).max())
    for R in (0, 1, 2):
        foot, cell, steps, cstar = _run(op, R, dt, vbar, fields)
        fo, co, so, cso = IM.rk_transport(conn, per, 2, vbar.reshape(2, conn.n_tri, -1), nf, dt, R)
        assert np.array_equal(cell, co)
        np.testing.assert_allclose(foot, fo, rtol=0, atol=1e-11)
        np.testing.assert_allclose(cstar, cso, rtol=0, atol=1e-11 * np.abs(cso).max())
