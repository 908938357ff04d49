"""The largest single-mesh configuration: 1024 x 1024 jittered periodic mesh,
p = 2 (2,097,152 triangles, 12,582,912 pressure DOFs).  Sampled output
blocks of the FP64 Schur and Helmholtz applies against the oracle row by
row, and a full-size FP32-IR Helmholtz solve to 1e-10 whose residual the
oracle recomputes on the sampled triangles."""
import numpy as np
import pytest

from oracle import mesh as OM
from oracle import operators as OP
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import dev, rel, to_internal, to_natural  # noqa: E402


def test_max_size_sampled_rows_and_solve(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    N, p = 1024, 2
    xy, tri, per = synth.jittered_periodic_mesh(N, 0)
    op = dgsl.Operator(xy, tri, per, p)
    assert op.n_dof == 12_582_912
    conn = OM.connectivity(xy, tri, per)
    m = op.maps()
    x64 = synth.standard_normal(op.n_dof, 2)
    x = dev(to_internal(x64, m["perm"], op.n_phi))
    y = torch.zeros_like(x)
    z = torch.zeros_like(x)
    op.dgsl_apply_schur(1e-3, x, y)
    op.dgsl_apply_helmholtz(1e-6, x, z)
    torch.cuda.synchronize()
    rng = np.random.default_rng(6)
    ids = np.unique(np.concatenate([rng.choice(op.n_tri, 300, replace=False), [0, op.n_tri - 1]]))
    ys = to_natural(y.cpu().numpy(), m["perm"], op.n_phi).reshape(-1, op.n_phi)[ids]
    zs = to_natural(z.cpu().numpy(), m["perm"], op.n_phi).reshape(-1, op.n_phi)[ids]
    assert rel(ys, OP.sampled_rows(conn, p, x64, ids, 1e-6)) <= 1e-13
    assert rel(zs, OP.sampled_rows(conn, p, x64, ids, 1e-6, 1.0)) <= 1e-13
    # full-size solve: H x = b, nu dt = 1e-4
    b = x
    xs = torch.zeros_like(b)
    info = op.dgsl_cg_solve(dgsl.HELMHOLTZ, 1e-4, b, xs, opts=dgsl.solve_opts(tol=1e-10, precision=dgsl.PREC_F32_IR))[0]
    torch.cuda.synchronize()
    assert info.status == dgsl.OK and info.relres <= 1e-10
    xs_nat = to_natural(xs.cpu().numpy(), m["perm"], op.n_phi)
    hx = OP.sampled_rows(conn, p, xs_nat, ids, 1e-4, 1.0)
    bs = x64.reshape(-1, op.n_phi)[ids]
    # rigorous: the sampled residual is part of the whole, <= 1e-10 ||b||
    assert np.linalg.norm(hx - bs) <= 1e-10 * np.linalg.norm(x64)
    # a residual spread over the mesh gives the sample about the global ratio
    # (5x allowed for the sampling spread)
    assert rel(hx, bs) <= 5e-10
