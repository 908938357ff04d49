"""GPU parity of the SL-IMEX Navier-Stokes step (dgsl_ns_imex_step) against
the oracle's step: R = 0, 1, 2 on the Taylor-Green vortex (velocity and the
last stage's pressure), divergence-free results, a uniform velocity kept, in
place equal to out of place, invalid arguments."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import fields as OF
from oracle import imex as IM
from oracle import mesh as OM
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
    ops = OP.Operators(OA.assemble(xy, tri, per, p, conn=conn))
    return op, ops, conn, per, op.maps()


def _tg(x, y):
    tp = 2.0 * np.pi
    return np.sin(tp * x) * np.cos(tp * y), -np.cos(tp * x) * np.sin(tp * y)


@pytest.mark.parametrize("R,N,p", [(0, 6, 2), (1, 6, 2), (2, 5, 2), (1, 5, 3)])
def test_ns_imex_step_parity(dgsl_lib, R, N, p):
    from paper_2401_17806_gb300 import dgsl
    op, ops, conn, per, m = _setup(N, p, 70 + N)
    ep = m["edge_perm"]
    Xd = OF.dual_nodes(conn, p, per)
    v0 = np.stack(_tg(Xd[..., 0], Xd[..., 1]))
    dt, nu = 0.05, 0.01
    vd = dev(v0[:, ep].ravel())
    vo = torch.empty_like(vd)
    pd = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    infos = op.dgsl_ns_imex_step(R, dt, nu, vd, vo, pd, opts=dgsl.solve_opts(tol=1e-12, precision=dgsl.PREC_F64))
    torch.cuda.synchronize()
    assert len(infos) == 3 * {0: 1, 1: 2, 2: 4}[R] and all(i.status == dgsl.OK for i in infos)
    got = np.empty_like(v0)
    got[:, ep] = vo.cpu().numpy().reshape(2, op.n_edge, op.n_psi)
    want, pw = IM.ns_imex_step(ops, conn, per, p, v0.ravel(), dt, nu, R)
    assert rel(got.ravel(), want) <= 1e-9
    assert rel(to_natural(pd.cpu().numpy(), m["perm"], op.n_phi), pw) <= 1e-8
    assert np.linalg.norm(ops.G.T @ got.ravel()) <= 1e-9 * np.linalg.norm(got)
    vi = vd.clone()
    op.dgsl_ns_imex_step(R, dt, nu, vi, vi, opts=dgsl.solve_opts(tol=1e-12, precision=dgsl.PREC_F64))  # in place
    torch.cuda.synchronize()
    assert torch.equal(vi, vo)


def test_ns_imex_uniform_and_arguments(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op, _, _, _, _ = _setup(8, 2, 71)
    nv = op.n_edge * op.n_psi
    v = torch.cat([torch.full((nv,), 0.3), torch.full((nv,), -0.2)]).to(torch.float64).cuda()
    for R in (0, 1, 2):
        vo = torch.empty_like(v)
        op.dgsl_ns_imex_step(R, 0.2, 0.01, v, vo, opts=dgsl.solve_opts(tol=1e-12))
        torch.cuda.synchronize()
        assert float((vo - v).abs().max()) < 1e-10
    for bad in ((3, 0.1, 0.01), (1, 0.0, 0.01), (1, 0.1, -1.0)):
        with pytest.raises(dgsl.DgslError) as e:
            op.dgsl_ns_imex_step(bad[0], bad[1], bad[2], v, v.clone())
        assert e.value.code == dgsl.EINVAL
    opu, _, _, _, _ = _setup(5, 1, 72, factored=False)
    z = torch.zeros(2 * opu.n_dual, dtype=torch.float64, device="cuda")
    with pytest.raises(dgsl.DgslError):
        opu.dgsl_ns_imex_step(1, 0.1, 0.01, z, z.clone())
