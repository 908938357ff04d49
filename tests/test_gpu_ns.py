"""GPU parity of the first-order semi-Lagrangian Navier-Stokes step
(dgsl_ns_step: transport of the main-grid velocity, viscous solves, pressure
projection) through the C-ABI against the oracle's step composed from its own
pieces: the new dual velocity and the pressure after one step; the result is
discretely divergence-free; a uniform velocity is kept exactly; in place and
out of place give the same bits; invalid calls are rejected."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import fields as OF
from oracle import mesh as OM
from oracle import ns as NS
from oracle import operators as OP
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import dev, rel, to_natural  # noqa: E402


def _setup(N, p, seed, factored=True):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    op = dgsl.Operator(xy, tri, per, p, factored=factored)
    conn = OM.connectivity(xy, tri, per)
    orc = OP.Operators(OA.assemble(xy, tri, per, p, conn=conn))
    return op, orc, conn, per, op.maps()


def _tg(x, y):
    tp = 2.0 * np.pi
    return np.sin(tp * x) * np.cos(tp * y), -np.cos(tp * x) * np.sin(tp * y)


@pytest.mark.parametrize("N,p", [(8, 2), (7, 3)])
def test_ns_step_parity(dgsl_lib, N, p):
    from paper_2401_17806_gb300 import dgsl
    op, orc, conn, per, m = _setup(N, p, 50 + N)
    ep = m["edge_perm"]
    Xd = OF.dual_nodes(conn, p, per)
    u0, w0 = _tg(Xd[..., 0], Xd[..., 1])
    v0 = np.stack([u0, w0]) + 0.05 * synth.standard_normal((2, op.n_edge, op.n_psi), 7)
    dt, nu = 0.1, 0.01  # about one cell per trajectory
    vd = dev(v0[:, ep].ravel())
    vo = torch.empty_like(vd)
    pd = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    infos = op.dgsl_ns_step(dt, nu, vd, vo, pd, opts=dgsl.solve_opts(tol=1e-12, precision=dgsl.PREC_F32_IR))
    torch.cuda.synchronize()
    assert all(i.status == dgsl.OK for i in infos)
    got = np.empty_like(v0)
    got[:, ep] = vo.cpu().numpy().reshape(2, op.n_edge, op.n_psi)
    want, pw = NS.ns_step(orc, conn, per, p, v0.ravel(), dt, nu)
    assert rel(got.ravel(), want) <= 1e-9
    pg = to_natural(pd.cpu().numpy(), m["perm"], op.n_phi)
    assert rel(pg, pw) <= 1e-8
    assert np.linalg.norm(orc.G.T @ got.ravel()) <= 1e-9 * np.linalg.norm(orc.G.T @ v0.ravel())


def test_ns_step_uniform_velocity_in_place_and_arguments(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op, orc, conn, per, m = _setup(9, 2, 61)
    nv = op.n_edge * op.n_psi
    v = torch.cat([torch.full((nv,), 0.3), torch.full((nv,), -0.2)]).to(torch.float64).cuda()
    vo = torch.empty_like(v)
    tight = dgsl.solve_opts(tol=1e-12)
    op.dgsl_ns_step(0.4, 0.01, v, vo, opts=tight)
    torch.cuda.synchronize()
    # (exact up to the solves' tolerance: the transport, the viscous term and
    # the divergence keep a constant field)
    assert torch.allclose(vo, v, rtol=0, atol=1e-10)
    w = v + 0.1 * torch.sin(torch.arange(v.numel(), dtype=torch.float64, device="cuda"))
    a = torch.empty_like(w)
    op.dgsl_ns_step(0.05, 0.01, w, a)
    op.dgsl_ns_step(0.05, 0.01, w, w)  # in place
    torch.cuda.synchronize()
    assert torch.equal(a, w)
    with pytest.raises(dgsl.DgslError):
        op.dgsl_ns_step(-0.1, 0.01, v, vo)
    opu, _, _, _, _ = _setup(6, 1, 62, factored=False)
    z = torch.zeros(2 * opu.n_dual, dtype=torch.float64, device="cuda")
    with pytest.raises(dgsl.DgslError):
        opu.dgsl_ns_step(0.1, 0.01, z, z.clone())


def test_ns_step_pressure_warm_start(dgsl_lib):
    """Starting the pressure solve from the last step's pressure (use_x0 with
    p_out) gives the same step within the solve tolerance, in fewer
    iterations."""
    from paper_2401_17806_gb300 import dgsl
    op, _, _, _, _ = _setup(12, 2, 63)
    X = op.node_coords(1)
    u, w = _tg(X[:, 0], X[:, 1])
    v = dev(np.concatenate([u, w]))
    o = dgsl.solve_opts(tol=1e-11, precision=dgsl.PREC_F32_IR)
    p1 = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    op.dgsl_ns_step(0.02, 0.01, v, v, p1, opts=o)
    cold_v, cold_p = torch.empty_like(v), torch.zeros_like(p1)
    ic = op.dgsl_ns_step(0.02, 0.01, v, cold_v, cold_p, opts=o)
    warm_v, warm_p = torch.empty_like(v), p1.clone()
    iw = op.dgsl_ns_step(0.02, 0.01, v, warm_v, warm_p, opts=dgsl.solve_opts(tol=1e-11, precision=dgsl.PREC_F32_IR,
                                                                                  use_x0=1))
    torch.cuda.synchronize()
    assert iw[2].iters < ic[2].iters
    assert float(torch.linalg.norm(warm_p - cold_p) / torch.linalg.norm(cold_p)) <= 1e-8
    assert float(torch.linalg.norm(warm_v - cold_v) / torch.linalg.norm(cold_v)) <= 1e-10


def test_ns_step_extrapolated_pressure(dgsl_lib):
    """use_x0 = 2: the pressure solve starts from 2 p^n - p^{n-1} (the operator
    keeps the last pressure).  Four steps end at the same velocity as with the
    last pressure as the start (both solved to 1e-12), and the last step's
    pressure solve takes fewer iterations."""
    from paper_2401_17806_gb300 import dgsl
    X = None
    res = {}
    for mode in (1, 2):
        op, _, _, _, _ = _setup(16, 2, 64)
        if X is None:
            X = op.node_coords(1)
        u, w = _tg(X[:, 0], X[:, 1])
        v = dev(np.concatenate([u, w]))
        p = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
        o = dgsl.solve_opts(tol=1e-12, precision=dgsl.PREC_F64, use_x0=mode)
        for _ in range(4):
            infos = op.dgsl_ns_step(0.01, 0.01, v, v, p, opts=o)
        torch.cuda.synchronize()
        res[mode] = (v.clone(), infos[2].iters)
    assert float(torch.linalg.norm(res[2][0] - res[1][0]) / torch.linalg.norm(res[1][0])) <= 1e-9
    assert res[2][1] < res[1][1], (res[1][1], res[2][1])
