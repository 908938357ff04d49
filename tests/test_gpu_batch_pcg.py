"""GPU parity of the block-Jacobi preconditioned CG inside the batched engine
and the serving loop (an extension: the paper's CG is unpreconditioned),
through the C-ABI: residuals against the oracle's FP64 operators for a mix of
meshes, degrees and kinds; fewer iterations than plain CG; every result the
same, bit for bit, alone, in the mix and inside a multi-RHS request; the
server's results equal the batch's while another solve on the same operator
rebuilds other preconditioned systems; invalid options rejected."""
import time

import numpy as np
import pytest

from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import to_internal, to_natural  # noqa: E402
from test_gpu_batch import _check_residual, _run_batch, problems  # noqa: E402,F401

BJ = 1  # DGSL_PRECOND_BLOCK_JACOBI


def test_batch_preconditioned_mixed(problems):
    from paper_2401_17806_gb300 import dgsl
    opts = dgsl.engine_opts(precision=dgsl.PREC_F32_IR, precond=BJ)
    xs, infos = _run_batch(problems, opts)
    _, plain = _run_batch(problems, dgsl.engine_opts(precision=dgsl.PREC_F32_IR))
    for (op, orc, perm, kind, coef, b), x, info, i0 in zip(problems, xs, infos, plain):
        assert info.status == dgsl.OK, info.status
        assert info.relres <= 1e-10
        _check_residual(orc, kind, coef, b, to_natural(x, perm, op.n_phi), 2e-10)
        if op.p >= 2:
            assert info.iters < i0.iters, (op.p, kind, info.iters, i0.iters)
    # alone: the same bits
    for k in (0, 3, 5):
        xa, ia = _run_batch([problems[k]], opts)
        assert ia[0].status == dgsl.OK and np.array_equal(xa[0], xs[k])


@pytest.mark.parametrize("R", [3, 8])
def test_batch_preconditioned_multi_rhs_equals_single(problems, R):
    from paper_2401_17806_gb300 import dgsl
    opts = dgsl.engine_opts(precision=dgsl.PREC_F32_IR, precond=BJ)
    for k in (2, 3):
        op, orc, perm, kind, coef, b = problems[k]
        bs = [synth.standard_normal(op.n_dof, 1900 + 17 * k + j) for j in range(R)]
        if R == 3:
            bs[1] = np.zeros(op.n_dof)
        bd = torch.tensor(np.concatenate([to_internal(v, perm, op.n_phi) for v in bs]), device="cuda")
        xd = torch.full_like(bd, np.nan)
        info = dgsl.dgsl_cg_solve_batch([dgsl.request(op, kind, coef, bd, xd, n_rhs=R)], opts)[0]
        torch.cuda.synchronize()
        assert info.status == dgsl.OK, info.status
        xs = xd.cpu().numpy().reshape(R, -1)
        singles, keep, reqs = [], [], []
        for j in range(R):
            bj = bd[j * op.n_dof:(j + 1) * op.n_dof].clone()
            xj = torch.full_like(bj, np.nan)
            keep.append(bj)
            singles.append(xj)
            reqs.append(dgsl.request(op, kind, coef, bj, xj))
        infos = dgsl.dgsl_cg_solve_batch(reqs, opts)
        torch.cuda.synchronize()
        for j in range(R):
            assert infos[j].status == dgsl.OK
            assert np.array_equal(singles[j].cpu().numpy(), xs[j])
            if not np.any(bs[j]):
                assert np.all(xs[j] == 0)
            else:
                _check_residual(orc, kind, coef, bs[j], to_natural(xs[j], perm, op.n_phi), 2e-10)


def test_batch_preconditioned_bf16(problems):
    """A P rounded to BF16 under FP64 refinement: converged, or DGSL_ENOTCONV
    with a relative residual the oracle confirms."""
    from paper_2401_17806_gb300 import dgsl
    opts = dgsl.engine_opts(precision=dgsl.PREC_BF16_IR, precond=BJ, max_refine=60)
    xs, infos = _run_batch(problems, opts)
    for (op, orc, perm, kind, coef, b), x, info in zip(problems, xs, infos):
        assert info.status in (dgsl.OK, dgsl.ENOTCONV)
        tol = 2e-10 if info.status == dgsl.OK else 1.01 * info.relres + 1e-12
        _check_residual(orc, kind, coef, b, to_natural(x, perm, op.n_phi), tol)


def test_server_preconditioned_while_the_operator_is_reused(problems):
    """Server requests hold their preconditioned systems: a solve on the same
    operator that builds five other systems meanwhile (more than the operator
    keeps) changes none of the server's results."""
    from paper_2401_17806_gb300 import dgsl
    opts = dgsl.engine_opts(precision=dgsl.PREC_F32_IR, precond=BJ, hbm_budget_bytes=2_000_000_000, idle_us=2000)
    ref, _ = _run_batch(problems, opts)
    srv = dgsl.Server(opts)
    try:
        bufs, tickets = [], []
        for rep in range(2):
            for k, (op, orc, perm, kind, coef, b) in enumerate(problems):
                bd = torch.tensor(to_internal(b, perm, op.n_phi), device="cuda")
                x = torch.full_like(bd, np.nan)
                bufs.append((k, bd, x))
                torch.cuda.synchronize()
                tickets.append(srv.dgsl_submit(dgsl.request(op, kind, coef, bd, x)))
        op1, _, perm1, _, _, b1 = problems[1]
        bb = torch.tensor(to_internal(b1, perm1, op1.n_phi), device="cuda")
        for c in (1e-3, 2e-3, 3e-3, 4e-3, 5e-3):
            xx = torch.zeros_like(bb)
            op1.dgsl_cg_solve(dgsl.HELMHOLTZ, c, bb, xx,
                              opts=dgsl.solve_opts(precision=dgsl.PREC_F32_IR, precond=BJ, tol=1e-10))
        done = {}
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 120:
            for t in tickets:
                if t not in done:
                    info = srv.dgsl_poll(t)
                    if info is not None:
                        done[t] = info
            time.sleep(0.001)
        assert len(done) == len(tickets)
        for (k, bd, x), t in zip(bufs, tickets):
            assert done[t].status == dgsl.OK
            assert np.array_equal(x.cpu().numpy(), ref[k])
        st = srv.stats()
        assert st["completed"] == len(tickets) and st["bytes_in_use"] == 0
    finally:
        srv.close()


def test_engine_rejects_bad_precond(problems):
    from paper_2401_17806_gb300 import dgsl
    op, orc, perm, kind, coef, b = problems[0]
    bd = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(dgsl.DgslError) as e:
        dgsl.dgsl_cg_solve_batch([dgsl.request(op, kind, coef, bd, bd.clone())], dgsl.engine_opts(precond=3))
    assert e.value.code == dgsl.EINVAL
    with pytest.raises(dgsl.DgslError):
        dgsl.Server(dgsl.engine_opts(precond=3))
    with pytest.raises(TypeError):
        dgsl.engine_opts(preconditioner=BJ)
