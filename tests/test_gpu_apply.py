"""GPU parity of the operator applies through the C-ABI against the oracle:
assembled and factored Schur matvec (FP64, rel. L2 <= 1e-13), FP32 matvec
(error reported, <= 1e-5), Helmholtz, the projections of eqs. d2m / m2d and
the divergence, with several right-hand sides, ragged sizes (row counts that
are not multiples of the CTA size) and a full-size 256 x 256, p = 3 mesh
checked on sampled rows."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import mesh as OM
from oracle import operators as OP
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _setup(N, p, seed, factored=True, store=0):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    op = dgsl.Operator(xy, tri, per, p, factored=factored, store=store)
    orc = OP.Operators(OA.assemble(xy, tri, per, p))
    return op, orc, op.maps()


def to_internal(v, perm, width):
    return v.reshape(-1, width)[perm].ravel()


def to_natural(v, perm, width):
    out = np.empty_like(v.reshape(-1, width))
    out[perm] = v.reshape(-1, width)
    return out.ravel()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def dev(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


@pytest.mark.parametrize("N,p", [(16, 1), (16, 2), (11, 3), (9, 4), (37, 2)])
def test_schur_apply_parity(dgsl_lib, N, p):
    op, orc, m = _setup(N, p, 10 + N)
    dt = 1e-2
    nrhs = 3
    xs = [synth.standard_normal(op.n_dof, 100 + k) for k in range(nrhs)]
    x = dev(np.concatenate([to_internal(v, m["perm"], op.n_phi) for v in xs]))
    for form in (0, 1):
        y = torch.full_like(x, np.nan)
        op.dgsl_apply_schur(dt, x, y, n_rhs=nrhs, form=form)
        torch.cuda.synchronize()
        yh = y.cpu().numpy().reshape(nrhs, -1)
        for k in range(nrhs):
            want = orc.apply_schur(xs[k], dt)
            got = to_natural(yh[k], m["perm"], op.n_phi)
            assert rel(got, want) <= 1e-13, (form, k, rel(got, want))


@pytest.mark.parametrize("N,p", [(16, 1), (13, 3), (9, 4)])
def test_schur_apply_f32_error(dgsl_lib, N, p):
    op, orc, m = _setup(N, p, 3, factored=False)
    x64 = synth.standard_normal(op.n_dof, 7)
    x = dev(to_internal(x64, m["perm"], op.n_phi), torch.float32)
    y = torch.zeros_like(x)
    op.dgsl_apply_schur_f32(0.5, x, y)
    torch.cuda.synchronize()
    got = to_natural(y.double().cpu().numpy(), m["perm"], op.n_phi)
    # the oracle applies the FP64 operator to the same (FP32-rounded) input
    want = orc.apply_schur(to_natural(x.double().cpu().numpy(), m["perm"], op.n_phi), 0.5)
    assert rel(got, want) <= 1e-5


@pytest.mark.parametrize("N,p", [(12, 2), (10, 3)])
def test_helmholtz_apply_parity(dgsl_lib, N, p):
    op, orc, m = _setup(N, p, 5)
    nu_dt = 3e-3
    x64 = synth.standard_normal(op.n_dof, 8)
    x = dev(to_internal(x64, m["perm"], op.n_phi))
    y = torch.zeros_like(x)
    op.dgsl_apply_helmholtz(nu_dt, x, y)
    torch.cuda.synchronize()
    got = to_natural(y.cpu().numpy(), m["perm"], op.n_phi)
    assert rel(got, orc.apply_helmholtz(x64, nu_dt)) <= 1e-13


@pytest.mark.parametrize("N,p", [(8, 1), (10, 3), (7, 4)])
def test_projections_and_divergence(dgsl_lib, N, p):
    op, orc, m = _setup(N, p, 9)
    ep = m["edge_perm"]
    # d2m right-hand side  b_i = sum_j U_ij^T vhat_j
    vh = synth.standard_normal((op.n_edge, op.n_psi), 21)
    vhd = dev(vh[ep].ravel())
    b = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    op.dgsl_project_d2m_rhs(vhd, b)
    # m2d  vhat = Mhat^{-1} (U_l vbar_l + U_r vbar_r)
    vb = synth.standard_normal(op.n_dof, 22)
    vbd = dev(to_internal(vb, m["perm"], op.n_phi))
    vo = torch.zeros(op.n_dual, dtype=torch.float64, device="cuda")
    op.dgsl_project_m2d(vbd, vo)
    # divergence y = G^T vhat for a vector dual field [2][Nd][Npsi]
    vv = synth.standard_normal((2, op.n_edge, op.n_psi), 23)
    vvd = dev(vv[:, ep].ravel())
    yd = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    op.dgsl_apply_div(vvd, yd)
    torch.cuda.synchronize()
    got_b = to_natural(b.cpu().numpy(), m["perm"], op.n_phi)
    assert rel(got_b, orc.d2m_rhs(vh.ravel())) <= 1e-13
    got_v = np.empty((op.n_edge, op.n_psi))
    got_v[ep] = vo.cpu().numpy().reshape(op.n_edge, op.n_psi)
    assert rel(got_v.ravel(), orc.m2d(vb)) <= 1e-12
    got_y = to_natural(yd.cpu().numpy(), m["perm"], op.n_phi)
    assert rel(got_y, orc.G.T @ vv.ravel()) <= 1e-13
    # and G^T is minus the paper's divergence D (D = -Q^T)
    assert rel(got_y, -(orc.Dm @ vv.ravel())) <= 1e-13


@pytest.mark.parametrize("N,p", [(8, 1), (9, 2), (10, 3), (7, 4)])
def test_velocity_update_parity(dgsl_lib, N, p):
    """v = F - c Mhat^-1 G p (eq. nc.2) against the oracle, out of place and in place."""
    from paper_2401_17806_gb300 import dgsl
    op, orc, m = _setup(N, p, 12)
    ep = m["edge_perm"]
    F = synth.standard_normal((2, op.n_edge, op.n_psi), 31)
    pr = synth.standard_normal(op.n_dof, 32)
    c = 0.37
    Fd = dev(F[:, ep].ravel())
    pd = dev(to_internal(pr, m["perm"], op.n_phi))
    vd = torch.empty_like(Fd)
    op.dgsl_velocity_update(c, Fd, pd, vd)
    torch.cuda.synchronize()
    got = np.empty_like(F)
    got[:, ep] = vd.cpu().numpy().reshape(2, op.n_edge, op.n_psi)
    want = orc.velocity_update(F.ravel(), pr, c)
    assert rel(got.ravel(), want) <= 1e-13
    op.dgsl_velocity_update(c, Fd, pd, Fd)  # in place
    torch.cuda.synchronize()
    assert torch.equal(Fd, vd)


def test_pressure_projection_divergence_free(dgsl_lib):
    """The whole projection on the device: b = G^T F, S p = b (FP32 CG + FP64
    refinement to 1e-12), v = F - dt^2 Mhat^-1 G p; the divergence of v is the
    solve's residual, checked on the device and with the oracle's separately
    assembled divergence D."""
    from paper_2401_17806_gb300 import dgsl
    op, orc, m = _setup(14, 3, 13)
    ep = m["edge_perm"]
    dt = 1e-2
    F = synth.standard_normal((2, op.n_edge, op.n_psi), 33)
    Fd = dev(F[:, ep].ravel())
    b = torch.empty(op.n_dof, dtype=torch.float64, device="cuda")
    op.dgsl_apply_div(Fd, b)
    pd = torch.zeros_like(b)
    info = op.dgsl_cg_solve(dgsl.SCHUR, dt, b, pd, opts=dgsl.solve_opts(tol=1e-12, precision=dgsl.PREC_F32_IR))[0]
    assert info.status == dgsl.OK
    vd = torch.empty_like(Fd)
    op.dgsl_velocity_update(dt * dt, Fd, pd, vd)
    y = torch.empty_like(b)
    op.dgsl_apply_div(vd, y)
    torch.cuda.synchronize()
    bn = float(torch.linalg.norm(b))
    assert float(torch.linalg.norm(y)) <= 2e-12 * bn
    v = np.empty_like(F)
    v[:, ep] = vd.cpu().numpy().reshape(2, op.n_edge, op.n_psi)
    assert np.linalg.norm(orc.Dm @ v.ravel()) <= 2e-12 * bn
    assert np.linalg.norm(v - F) > 1e-3 * np.linalg.norm(F)


def test_velocity_update_needs_factored_blocks(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op, orc, m = _setup(6, 2, 14, factored=False)
    Fd = torch.zeros(2 * op.n_dual, dtype=torch.float64, device="cuda")
    pd = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(dgsl.DgslError):
        op.dgsl_velocity_update(1.0, Fd, pd, Fd.clone())


def test_full_size_sampled_rows(dgsl_lib):
    """256 x 256 mesh, p = 3 (131,072 triangles): sampled output blocks of the
    FP64 Schur and Helmholtz applies against the oracle, row by row."""
    from paper_2401_17806_gb300 import dgsl
    N, p = 256, 3
    xy, tri, per = synth.jittered_periodic_mesh(N, 0)
    op = dgsl.Operator(xy, tri, per, p)
    conn = OM.connectivity(xy, tri, per)
    m = op.maps()
    x64 = synth.standard_normal(op.n_dof, 1)
    x = dev(to_internal(x64, m["perm"], op.n_phi))
    y = torch.zeros_like(x)
    z = torch.zeros_like(x)
    op.dgsl_apply_schur(1e-3, x, y)
    op.dgsl_apply_helmholtz(1e-6, x, z)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    ids = np.unique(np.concatenate([rng.choice(op.n_tri, 300, replace=False), [0, op.n_tri - 1]]))
    ys = to_natural(y.cpu().numpy(), m["perm"], op.n_phi).reshape(-1, op.n_phi)[ids]
    zs = to_natural(z.cpu().numpy(), m["perm"], op.n_phi).reshape(-1, op.n_phi)[ids]
    want_y = OP.sampled_rows(conn, p, x64, ids, 1e-6)
    want_z = OP.sampled_rows(conn, p, x64, ids, 1e-6, 1.0)
    assert rel(ys, want_y) <= 1e-13
    assert rel(zs, want_z) <= 1e-13
