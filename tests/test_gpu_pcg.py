"""GPU parity of the block-Jacobi preconditioned CG (an extension: the paper's
CG is unpreconditioned) through the C-ABI: residual against the oracle's FP64
operator and error against its direct solve, for FP64 CG and FP32 inner CG
under FP64 refinement; the FP64 iteration count against the oracle's textbook
PCG; one step where A is block diagonal (the mass matrix, nu dt = 0); the
preconditioner rebuilt when the coefficient changes; multi-RHS results equal
to single solves; invalid options rejected; and a full-size 256 x 256, p = 3
solve checked on sampled rows."""
import numpy as np
import pytest

from oracle import mesh as OM
from oracle import operators as OP
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import dev, rel, to_internal, to_natural  # noqa: E402
from test_gpu_cg import _setup, _solve  # noqa: E402

BJ = 1  # DGSL_PRECOND_BLOCK_JACOBI


def _kappa(A):
    ev = np.linalg.eigvalsh(A.toarray())
    return ev[-1] / (ev[1] if ev[0] < 1e-12 * ev[-1] else ev[0])


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N,p", [(9, 1), (8, 2), (14, 3), (10, 4)])
def test_pcg_schur_parity(dgsl_lib, prec, N, p):
    from paper_2401_17806_gb300 import dgsl
    op, orc, m = _setup(N, p, 21)
    dt = 1e-3
    b = synth.standard_normal(op.n_dof, 61)
    x, info, _ = _solve(op, m, dgsl.SCHUR, dt, b, tol=1e-12, precision=prec, precond=BJ)
    assert info.status == dgsl.OK, info.status
    assert info.relres <= 1e-12
    S = orc.schur_matrix(dt)
    pb = OP.project_mean(b)
    kappa = _kappa(S) if op.n_dof <= 5000 else 1e6
    assert np.linalg.norm(pb - S @ x) / np.linalg.norm(pb) <= max(2e-12, 1e-13 * kappa)
    assert rel(x, OP.schur_solve_direct(S, b)) <= max(1e-10, 10 * kappa * 1e-12)
    assert abs(x.sum()) <= 1e-12 * np.abs(x).sum()
    _, info0, _ = _solve(op, m, dgsl.SCHUR, dt, b, tol=1e-12, precision=prec)
    if p >= 2:
        assert info.iters < info0.iters, (info.iters, info0.iters)
    if prec == 0:
        # one FP64 inner solve to 0.5 tol: the Chronopoulos-Gear recurrences
        # are the textbook PCG's up to rounding, so the counts agree closely
        P = OP.block_jacobi_blocks(S, op.n_phi)
        _, it_orc, _ = OP.pcg(lambda v: S @ v, b, lambda v: OP.apply_blocks(P, v), tol=0.5e-12, mean_zero=True)
        assert abs(info.iters - it_orc) <= max(3, 0.03 * it_orc), (info.iters, it_orc)


@pytest.mark.parametrize("prec", [0, 1])
def test_pcg_helmholtz_parity(dgsl_lib, prec):
    from paper_2401_17806_gb300 import dgsl
    op, orc, m = _setup(18, 3, 22)
    nu_dt = 1e-4
    b = synth.standard_normal(op.n_dof, 62)
    x, info, _ = _solve(op, m, dgsl.HELMHOLTZ, nu_dt, b, tol=1e-12, precision=prec, precond=BJ)
    assert info.status == dgsl.OK
    H = orc.helmholtz_matrix(nu_dt)
    assert np.linalg.norm(b - H @ x) / np.linalg.norm(b) <= 1e-12
    assert rel(x, OP.direct_solve(H, b)) <= 1e-10
    _, info0, _ = _solve(op, m, dgsl.HELMHOLTZ, nu_dt, b, tol=1e-12, precision=prec)
    assert info.iters < info0.iters
    if prec == 0:
        P = OP.block_jacobi_blocks(H, op.n_phi)
        _, it_orc, _ = OP.pcg(lambda v: H @ v, b, lambda v: OP.apply_blocks(P, v), tol=0.5e-12)
        assert abs(info.iters - it_orc) <= max(2, 0.03 * it_orc), (info.iters, it_orc)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_pcg_mass_matrix_in_one_step(dgsl_lib, p):
    """nu dt = 0: A = Mbar is block diagonal, the preconditioner is its exact
    inverse (in the device layout) and every inner solve stops after one step."""
    from paper_2401_17806_gb300 import dgsl
    op, orc, m = _setup(7, p, 23)
    b = synth.standard_normal(op.n_dof, 63)
    x, info, _ = _solve(op, m, dgsl.HELMHOLTZ, 0.0, b, tol=1e-13, precision=dgsl.PREC_F64, precond=BJ)
    assert info.status == dgsl.OK and info.iters == 1
    assert rel(orc.apply_Mbar(x), b) <= 1e-13
    x, info, _ = _solve(op, m, dgsl.HELMHOLTZ, 0.0, b, tol=1e-12, precision=dgsl.PREC_F32_IR, precond=BJ)
    assert info.status == dgsl.OK and info.iters == info.refinements
    assert rel(orc.apply_Mbar(x), b) <= 1e-12


def test_pcg_rebuilds_for_a_new_coefficient(dgsl_lib):
    """The operator keeps the blocks of the last four systems; every other
    coefficient (or an evicted one) gets freshly built blocks, and the results
    are the same either way."""
    from paper_2401_17806_gb300 import dgsl
    op, orc, m = _setup(10, 2, 24)
    b = synth.standard_normal(op.n_dof, 64)
    kw = dict(tol=1e-12, precision=dgsl.PREC_F32_IR, precond=BJ)
    x1, _, _ = _solve(op, m, dgsl.HELMHOLTZ, 1e-3, b, **kw)
    x2, info2, _ = _solve(op, m, dgsl.HELMHOLTZ, 1e-2, b, **kw)
    x3, _, _ = _solve(op, m, dgsl.HELMHOLTZ, 1e-3, b, **kw)
    assert np.array_equal(x1, x3)
    H2 = orc.helmholtz_matrix(1e-2)
    assert info2.status == dgsl.OK and np.linalg.norm(b - H2 @ x2) / np.linalg.norm(b) <= 1e-12
    for c in (2e-2, 3e-2, 4e-2, 5e-2):  # evicts 1e-3
        _solve(op, m, dgsl.HELMHOLTZ, c, b, **kw)
    x3, _, _ = _solve(op, m, dgsl.HELMHOLTZ, 1e-3, b, **kw)
    assert np.array_equal(x1, x3)
    # the FP64 blocks are kept beside the FP32 ones
    x4, info4, _ = _solve(op, m, dgsl.HELMHOLTZ, 1e-3, b, tol=1e-12, precision=dgsl.PREC_F64, precond=BJ)
    assert info4.status == dgsl.OK and rel(x4, x1) <= 1e-10
    x5, _, _ = _solve(op, m, dgsl.HELMHOLTZ, 1e-3, b, **kw)
    assert np.array_equal(x1, x5)


def test_pcg_multiple_rhs_and_options(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op, orc, m = _setup(12, 3, 25)
    dt = 1e-2
    bs = [synth.standard_normal(op.n_dof, 70 + k) for k in range(3)]
    b = dev(np.concatenate([to_internal(v, m["perm"], op.n_phi) for v in bs]))
    x = torch.zeros_like(b)
    opts = dgsl.solve_opts(tol=1e-11, precision=dgsl.PREC_F32_IR, precond=BJ)
    infos = op.dgsl_cg_solve(dgsl.SCHUR, dt, b, x, n_rhs=3, opts=opts)
    torch.cuda.synchronize()
    assert all(i.status == dgsl.OK for i in infos)
    xs = x.cpu().numpy().reshape(3, -1)
    for k in range(3):
        xa, _, _ = _solve(op, m, dgsl.SCHUR, dt, bs[k], tol=1e-11, precision=dgsl.PREC_F32_IR, precond=BJ)
        assert np.array_equal(xa, to_natural(xs[k], m["perm"], op.n_phi))
    bb = dev(np.zeros(op.n_dof))
    with pytest.raises(dgsl.DgslError) as e:
        op.dgsl_cg_solve(dgsl.SCHUR, dt, bb, bb.clone(), opts=dgsl.solve_opts(precond=3))
    assert e.value.code == dgsl.EINVAL
    with pytest.raises(dgsl.DgslError) as e:
        op.dgsl_cg_solve_noalloc(dgsl.SCHUR, dt, bb, bb.clone(), opts=dgsl.solve_opts(precond=BJ))
    assert e.value.code == dgsl.EINVAL
    with pytest.raises(TypeError):
        dgsl.solve_opts(preconditioner=BJ)


def test_pcg_full_size_solve_sampled_residual(dgsl_lib):
    """256 x 256, p = 3, dt = 1e-3, block-Jacobi FP32 inner CG + FP64
    refinement to 1e-10: the oracle recomputes sampled rows of the residual."""
    from paper_2401_17806_gb300 import dgsl
    N, p, dt = 256, 3, 1e-3
    xy, tri, per = synth.jittered_periodic_mesh(N, 0)
    op = dgsl.Operator(xy, tri, per, p)
    conn = OM.connectivity(xy, tri, per)
    m = op.maps()
    b64 = synth.standard_normal(op.n_dof, 12) * dt * dt
    b64 -= b64.mean()
    x, info, _ = _solve(op, m, dgsl.SCHUR, dt, b64, tol=1e-10, precision=dgsl.PREC_F32_IR, precond=BJ)
    assert info.status == dgsl.OK and info.relres <= 1e-10
    _, info0, _ = _solve(op, m, dgsl.SCHUR, dt, b64, tol=1e-10, precision=dgsl.PREC_F32_IR)
    assert info.iters < info0.iters
    rng = np.random.default_rng(3)
    ids = rng.choice(op.n_tri, 400, replace=False)
    Sx = OP.sampled_rows(conn, p, x, ids, dt * dt)
    r = b64.reshape(-1, op.n_phi)[ids] - Sx
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b64)


def test_pcg_bf16_couplings(dgsl_lib):
    """Block-Jacobi with A P rounded to BF16 (P in FP32) under FP64
    refinement: the Helmholtz system converges to 1e-10 (oracle residual);
    the Schur system converges or reports DGSL_ENOTCONV with a relative
    residual the oracle confirms."""
    from paper_2401_17806_gb300 import dgsl
    op, orc, m = _setup(12, 3, 26, store=dgsl.STORE_F64 | dgsl.STORE_BF16)
    b = synth.standard_normal(op.n_dof, 72)
    x, info, _ = _solve(op, m, dgsl.HELMHOLTZ, 1e-3, b, tol=1e-10, precision=dgsl.PREC_BF16_IR, precond=BJ)
    assert info.status == dgsl.OK
    H = orc.helmholtz_matrix(1e-3)
    assert np.linalg.norm(b - H @ x) / np.linalg.norm(b) <= 2e-10
    x, info, _ = _solve(op, m, dgsl.SCHUR, 1e-2, b, tol=1e-10, precision=dgsl.PREC_BF16_IR, precond=BJ,
                        max_refine=60)
    assert info.status in (dgsl.OK, dgsl.ENOTCONV)
    S = orc.schur_matrix(1e-2)
    pb = OP.project_mean(b)
    r = np.linalg.norm(pb - S @ x) / np.linalg.norm(pb)
    assert r <= max(2e-10, 1.01 * info.relres + 1e-12)
