"""The FP64 rounding floor a non-converged solve reports (relres_floor).

Model: every value of x carries a rounding error x_c theta_c, theta_c uniform
in [-u, u] (u = 2^-53) and independent, so E||A (x o theta)||^2 =
u^2 / 3 sum_i sum_c (a_ic x_c)^2.  The library's number is checked against a
Monte Carlo of that expectation with the ORACLE's sparse matrix (independent
assembly), and a solve asked for an unattainable tolerance must stop within a
small multiple of it."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import operators as OP
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import to_internal, to_natural  # noqa: E402

U = 2.0 ** -53


@pytest.mark.parametrize("kind,precond", [(0, 2), (0, 0), (1, 2)])
def test_floor_matches_the_rounding_model(dgsl_lib, kind, precond):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(24, 7)
    p = 3
    op = dgsl.Operator(xy, tri, per, p)
    perm = op.maps()["perm"]
    orc = OP.Operators(OA.assemble(xy, tri, per, p))
    coef = 1e-3
    A = (orc.schur_matrix(coef) if kind == 0 else orc.helmholtz_matrix(coef)).tocsr()
    b = synth.standard_normal(op.n_dof, 3)
    bd = torch.tensor(to_internal(b, perm, op.n_phi), device="cuda")
    x = torch.zeros_like(bd)
    # a tolerance no FP64 vector can meet: the refinement stalls
    info = op.dgsl_cg_solve(kind, coef, bd, x, check=False,
                            opts=dgsl.solve_opts(tol=1e-19, precision=dgsl.PREC_F64, precond=precond))[0]
    torch.cuda.synchronize()
    assert info.status == dgsl.ENOTCONV
    assert info.relres_floor > 0.0
    xn = to_natural(x.cpu().numpy(), perm, op.n_phi)
    rhs = OP.project_mean(b) if kind == 0 else b
    rng = np.random.default_rng(11)
    samples = [np.linalg.norm(A @ (xn * rng.uniform(-U, U, xn.size))) ** 2 for _ in range(8)]
    model = np.sqrt(np.mean(samples)) / np.linalg.norm(rhs)
    print(f"FLOOR kind={kind} precond={precond} library={info.relres_floor:.4e} monte_carlo={model:.4e} "
          f"stalled_relres={info.relres:.4e} ratio={info.relres / info.relres_floor:.2f}")
    assert abs(info.relres_floor / model - 1.0) <= 0.05
    # the stall sits at FP64's own accuracy: within a small multiple of the floor
    assert info.relres <= 100.0 * info.relres_floor


def test_converged_solve_reports_no_floor(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(12, 1)
    op = dgsl.Operator(xy, tri, per, 2)
    b = torch.tensor(synth.standard_normal(op.n_dof, 5), device="cuda")
    x = torch.zeros_like(b)
    info = op.dgsl_cg_solve(dgsl.SCHUR, 1e-2, b, x, opts=dgsl.solve_opts(tol=1e-10))[0]
    torch.cuda.synchronize()
    assert info.status == dgsl.OK and info.relres_floor == 0.0
