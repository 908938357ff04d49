"""GPU parity of the semi-Lagrangian transport (Sec. 2.5, eq. lagrtrj, eq.
intstage) through the C-ABI against the oracle's element-by-element walk:
feet, containing cells and cells crossed per Gauss-point trajectory and the
transported fields, for p = 1..4 on ragged meshes with the Taylor-Green
velocity; uniform velocity (exact feet, brute-force cells); zero velocity
(fields given back); the step cap reported as a status; and sampled
trajectories and triangles of the full 256 x 256, p = 3 case."""
import numpy as np
import pytest

from oracle import basis as B
from oracle import mesh as OM
from oracle import sl as SL
from oracle.assemble import main_mass
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import dev, to_internal, to_natural  # noqa: E402


def _tg(x, y):
    tp = 2.0 * np.pi
    return np.sin(tp * x) * np.cos(tp * y), -np.cos(tp * x) * np.sin(tp * y)


def _setup(N, p, seed):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    op = dgsl.Operator(xy, tri, per, p)
    return op, OM.connectivity(xy, tri, per), per, op.maps()["perm"]


def _run(op, dt, vbar, fields):
    """GPU transport; results in the natural numbering (feet [Ne, Ng, 2],
    cells, steps [Ne, Ng], cstar [nf, Ne, Nphi])."""
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
    op.dgsl_sl_transport(dt, vb, c, cs, nf, foot, cell, steps)
    torch.cuda.synchronize()
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    f_i = foot.cpu().numpy().reshape(op.n_tri, ng, 2)
    c_i = cell.cpu().numpy().reshape(op.n_tri, ng)
    s_i = steps.cpu().numpy().reshape(op.n_tri, ng)
    f_n = np.empty_like(f_i)
    c_n = np.empty_like(c_i)
    s_n = np.empty_like(s_i)
    f_n[perm], c_n[perm], s_n[perm] = f_i, perm[c_i], s_i  # rows to natural, cell ids to natural
    cstar = (np.stack([to_natural(v, perm, op.n_phi).reshape(op.n_tri, op.n_phi)
                       for v in cs.cpu().numpy().reshape(nf, -1)]) if nf else None)
    return f_n, c_n, s_n, cstar


@pytest.mark.parametrize("N,p", [(7, 1), (9, 2), (8, 3), (6, 4)])
def test_sl_transport_parity(dgsl_lib, N, p):
    op, conn, per, perm = _setup(N, p, 20 + N)
    X = B.triangle_points(conn.tri_xy, B.nodes(p))  # natural nodes [Ne, Nphi, 2]
    vbar = np.stack(_tg(X[..., 0], X[..., 1])).reshape(2, -1)
    fields = [synth.standard_normal(op.n_dof, 90 + k) for k in range(2)]
    dt = 0.2  # 1-4 cells per trajectory at these sizes
    foot, cell, steps, cstar = _run(op, dt, vbar, fields)
    fo, co, so, cso = SL.transport(conn, per, p, vbar.reshape(2, conn.n_tri, -1),
                                   np.stack([f.reshape(conn.n_tri, -1) for f in fields]), dt)
    assert so.max() >= 2
    assert np.array_equal(cell, co)
    assert np.array_equal(steps, so)
    np.testing.assert_allclose(foot, fo, rtol=0, atol=1e-11)
    np.testing.assert_allclose(cstar, cso, rtol=0, atol=1e-11 * np.abs(cso).max())


def test_uniform_velocity_and_zero_velocity(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op, conn, per, perm = _setup(10, 2, 31)
    V = np.array([0.37, -0.21])
    vbar = [np.full(op.n_dof, V[0]), np.full(op.n_dof, V[1])]
    dt = 0.45
    foot, cell, steps, _ = _run(op, dt, vbar, [])
    pts, _ = dgsl.sl_quadrature(2)
    X = B.triangle_points(conn.tri_xy, pts)
    d = foot - (X - dt * V)
    assert np.abs(d - per * np.round(d / per)).max() < 1e-12
    assert steps.max() >= 4
    rng = np.random.default_rng(1)
    for _ in range(40):
        i, g = int(rng.integers(op.n_tri)), int(rng.integers(pts.shape[0]))
        assert cell[i, g] in [h[0] for h in SL.locate(conn.tri_xy, per, foot[i, g])]
    c = synth.standard_normal(op.n_dof, 5)
    foot, cell, steps, cstar = _run(op, dt, [np.zeros(op.n_dof), np.zeros(op.n_dof)], [c])
    assert steps.max() == 0 and np.array_equal(cell, np.repeat(np.arange(op.n_tri)[:, None], cell.shape[1], 1))
    np.testing.assert_allclose(cstar[0].ravel(), c, rtol=0, atol=1e-12 * np.abs(c).max())


def test_step_cap_and_arguments(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op, conn, per, perm = _setup(8, 1, 33)
    vb = dev(np.concatenate([np.full(op.n_dof, 1.0), np.full(op.n_dof, 0.3)]))
    with pytest.raises(dgsl.DgslError) as e:
        op.dgsl_sl_transport(1.0e6, vb)  # would cross ~10^8 cells: the walk stops at the cap
    assert e.value.code == dgsl.ENOTCONV
    op.dgsl_sl_transport(0.3, vb)  # the context is still usable
    c = dev(np.zeros(9 * op.n_dof))
    with pytest.raises(dgsl.DgslError) as e:
        op.dgsl_sl_transport(0.1, vb, c, c.clone(), 9)
    assert e.value.code == dgsl.EINVAL
    with pytest.raises(dgsl.DgslError):
        op.dgsl_sl_transport(float("nan"), vb)


def test_sl_full_size_sampled(dgsl_lib):
    """256 x 256, p = 3, dt = 0.01 (about 2.6 cells per trajectory): sampled
    trajectories and the transported velocity of sampled triangles against
    the oracle's walk."""
    N, p, dt = 256, 3, 0.01
    op, conn, per, perm = _setup(N, p, 0)
    X = B.triangle_points(conn.tri_xy, B.nodes(p))
    vbar = np.stack(_tg(X[..., 0], X[..., 1])).reshape(2, -1)
    foot, cell, steps, cstar = _run(op, dt, vbar, [vbar[0], vbar[1]])
    nbr, trans, back = SL.frames(conn, per)
    vb = vbar.reshape(2, conn.n_tri, -1)

    def velocity(c, xi, eta):
        return vb[:, c, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]

    pts, w = SL.quadrature(p)
    P = B.triangle_points(conn.tri_xy, pts)
    rng = np.random.default_rng(4)
    tris = rng.choice(conn.n_tri, 40, replace=False)
    vals = np.zeros((2, len(tris), len(w)))
    for a, i in enumerate(tris):
        for g in range(len(w)):
            xf, cf, st = SL.walk(conn.tri_xy, nbr, trans, back, velocity, P[i, g], i, dt)
            assert cf == cell[i, g] and st == steps[i, g]
            assert np.abs(xf - foot[i, g]).max() < 1e-11
            _, xi, eta = SL.barycentric(conn.tri_xy[cf], xf)
            vals[:, a, g] = vb[:, cf, :] @ B.eval_phi(p, np.array([[xi, eta]]))[0]
    assert steps.mean() > 1.0

    class Sub:
        tri_xy = conn.tri_xy[tris]

    Mbar, area2 = main_mass(Sub, p)
    phi_g = B.eval_phi(p, pts)
    for f in range(2):
        rhs = np.einsum("gl,g,ag->al", phi_g, w, vals[f]) * np.abs(area2)[:, None]
        ref = np.linalg.solve(Mbar, rhs[..., None])[..., 0]
        np.testing.assert_allclose(cstar[f][tris], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_non_unit_period_forward_time_and_determinism(dgsl_lib):
    """A 2 x 0.5 periodic domain, dt < 0 (forward characteristics): the feet
    of a uniform velocity are x - dt v modulo the periods, in cells that
    contain them; repeated calls give the same bits."""
    from paper_2401_17806_gb300 import dgsl
    xy, tri, _ = synth.jittered_periodic_mesh(9, 41)
    per = np.array([2.0, 0.5])
    xy = xy * per
    op = dgsl.Operator(xy, tri, per, 2)
    conn = OM.connectivity(xy, tri, per)
    V = np.array([-0.8, 0.33])
    dt = -0.9  # forward: about 3 cells in x, 5 in y
    foot, cell, steps, _ = _run(op, dt, [np.full(op.n_dof, V[0]), np.full(op.n_dof, V[1])], [])
    pts, _ = dgsl.sl_quadrature(2)
    X = B.triangle_points(conn.tri_xy, pts)
    d = foot - (X - dt * V)
    assert np.abs(d - per * np.round(d / per)).max() < 1e-12
    assert steps.max() >= 5
    rng = np.random.default_rng(2)
    for _ in range(40):
        i, g = int(rng.integers(op.n_tri)), int(rng.integers(pts.shape[0]))
        assert cell[i, g] in [h[0] for h in SL.locate(conn.tri_xy, per, foot[i, g])]
    Xn = B.triangle_points(conn.tri_xy, B.nodes(2))
    vb = np.stack(_tg(Xn[..., 0] / per[0], Xn[..., 1] / per[1])).reshape(2, -1)
    f = [synth.standard_normal(op.n_dof, 3)]
    a = _run(op, 0.05, vb, f)
    b = _run(op, 0.05, vb, f)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)


@pytest.mark.parametrize("p", [1, 3])
def test_held_trajectories_on_a_source_line(dgsl_lib, p):
    """Velocity pointing away from one edge on both sides: the kernel holds
    the trajectories that meet the edge where they meet it (after one
    crossing and one bounce back), like the oracle, at the perpendicular
    feet."""
    from test_oracle_sl import source_line
    op, conn, per, perm = _setup(6, p, 3)
    for j in (0, 7, conn.n_edge - 1):
        vbar, want = source_line(conn, per, p, j)
        foot, cell, steps, _ = _run(op, 5.0, vbar.reshape(2, -1), [])
        fo, co, so, _ = SL.transport(conn, per, p, vbar, np.zeros((0, conn.n_tri, B.n_phi(p))), 5.0)
        assert np.array_equal(cell, co) and np.array_equal(steps, so)
        np.testing.assert_allclose(foot, fo, rtol=0, atol=1e-13)
        for (t, g), q in want.items():
            assert cell[t, g] == t and steps[t, g] == 2
            np.testing.assert_allclose(foot[t, g], q, rtol=0, atol=1e-13)
