"""GPU parity of the SL-IMEX advection-diffusion step (dgsl_advdiff_step)
against the oracle's step: R = 0, 1, 2 with the Taylor-Green velocity; a
constant is kept; with a constant velocity the local error against the exact
decaying sine falls at the scheme's orders; invalid arguments."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import basis as B
from oracle import imex as IM
from oracle import mesh as OM
from oracle import operators as OP
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import dev, rel, to_internal, to_natural  # noqa: E402
from test_gpu_sl import _tg  # noqa: E402


def _setup(N, p, seed):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    op = dgsl.Operator(xy, tri, per, p)
    conn = OM.connectivity(xy, tri, per)
    return op, conn, per, op.maps()["perm"], xy, tri


@pytest.mark.parametrize("R,N,p", [(0, 6, 2), (1, 6, 3), (2, 5, 2), (1, 7, 1), (2, 4, 4)])
def test_advdiff_step_parity(dgsl_lib, R, N, p):
    from paper_2401_17806_gb300 import dgsl
    op, conn, per, perm, xy, tri = _setup(N, p, 60 + N)
    ops = OP.Operators(OA.assemble(xy, tri, per, p, conn=conn))
    X = B.triangle_points(conn.tri_xy, B.nodes(p))
    vbar = np.stack(_tg(X[..., 0], X[..., 1]))
    C0 = synth.standard_normal(op.n_dof, 80 + R)
    dt, alpha = 0.1, 0.05
    vb = dev(np.concatenate([to_internal(v.ravel(), perm, op.n_phi) for v in vbar]))
    c = dev(to_internal(C0, perm, op.n_phi))
    out = torch.empty_like(c)
    infos = op.dgsl_advdiff_step(R, dt, alpha, vb, c, out,
                                 opts=dgsl.solve_opts(tol=1e-12, precision=dgsl.PREC_F64))
    torch.cuda.synchronize()
    assert len(infos) == {0: 1, 1: 2, 2: 4}[R] and all(i.status == dgsl.OK for i in infos)
    got = to_natural(out.cpu().numpy(), perm, op.n_phi)
    want = IM.advdiff_step(ops, conn, per, p, vbar, C0, dt, alpha, R)
    assert rel(got, want) <= 1e-9
    op.dgsl_advdiff_step(R, dt, alpha, vb, c, c, opts=dgsl.solve_opts(tol=1e-12, precision=dgsl.PREC_F64))  # in place
    torch.cuda.synchronize()
    assert torch.equal(c, out)


def test_advdiff_constant_and_arguments(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op, conn, per, perm, _, _ = _setup(8, 3, 7)
    X = op.node_coords(0)
    vb = dev(np.concatenate(_tg(X[:, 0], X[:, 1])))
    c = torch.full((op.n_dof,), 1.7, dtype=torch.float64, device="cuda")
    out = torch.empty_like(c)
    op.dgsl_advdiff_step(2, 0.1, 0.2, vb, c, out)
    torch.cuda.synchronize()
    assert float((out - 1.7).abs().max()) < 1e-11
    for bad in ((3, 0.1, 0.1), (1, 0.0, 0.1), (1, 0.1, -1.0), (1, float("nan"), 0.1)):
        with pytest.raises(dgsl.DgslError) as e:
            op.dgsl_advdiff_step(bad[0], bad[1], bad[2], vb, c, out)
        assert e.value.code == dgsl.EINVAL
    with pytest.raises(dgsl.DgslError) as e:  # segments of ~10^8 cells: stopped at the cap
        op.dgsl_advdiff_step(1, 1.0e6, 0.1, vb, c, out)
    assert e.value.code == dgsl.ENOTCONV
    op.dgsl_advdiff_step(1, 0.1, 0.1, vb, c, out)  # the context is still usable


@pytest.mark.parametrize("R,order", [(1, 2.5), (2, 3.3)])
def test_advdiff_local_order(dgsl_lib, R, order):
    """C = exp(-alpha |k|^2 t) sin(k.(x - V t)), constant V, 48 x 48, p = 4:
    one step's error falls faster than dt^order from dt = 0.05 to 0.025
    (the scheme's local orders are 3 and 4)."""
    from paper_2401_17806_gb300 import dgsl
    op, conn, per, perm, _, _ = _setup(48, 4, 3)
    X = op.node_coords(0)
    V = np.array([0.8, 0.5])
    k = np.array([2.0 * np.pi, 0.0])
    alpha = 0.2
    lam = alpha * (k @ k)
    vb = dev(np.concatenate([np.full(op.n_dof, V[0]), np.full(op.n_dof, V[1])]))

    def exact(t):
        return np.exp(-lam * t) * np.sin(X @ k - (k @ V) * t)

    errs = []
    for dt in (0.1, 0.05, 0.025):
        c = dev(exact(0.0))
        op.dgsl_advdiff_step(R, dt, alpha, vb, c, c, opts=dgsl.solve_opts(tol=1e-11, precision=dgsl.PREC_F64,
                                                                          precond=dgsl.PRECOND_BLOCK_JACOBI))
        torch.cuda.synchronize()
        errs.append(np.abs(c.cpu().numpy() - exact(dt)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert orders[-1] > order, (errs, orders)
