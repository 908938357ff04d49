"""GPU tests of multigrid requests in the batch call and the server: the
requests of different operators run concurrently on worker streams, each gives
the same bits as the library's own multigrid solve on the same system, the
oracle confirms the residuals, and requests submitted while other solves run
are admitted and finish (the server counts them)."""
import time

import numpy as np
import pytest

from oracle import assemble as OA
from oracle import operators as OP
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import to_internal, to_natural  # noqa: E402

CASES = [(12, 1, 0, 1e-2), (16, 2, 1, 1e-3), (20, 3, 0, 1e-3), (10, 4, 0, 2e-3), (24, 2, 0, 1e-2)]


@pytest.fixture(scope="module")
def problems(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    out = []
    for k, (N, p, kind, coef) in enumerate(CASES):
        xy, tri, per = synth.jittered_periodic_mesh(N, 60 + k)
        op = dgsl.Operator(xy, tri, per, p)
        orc = OP.Operators(OA.assemble(xy, tri, per, p))
        out.append((op, orc, op.maps()["perm"], kind, coef, synth.standard_normal(op.n_dof, 80 + k)))
    return out


def _single(op, perm, kind, coef, b, tol=1e-10):
    from paper_2401_17806_gb300 import dgsl
    bd = torch.tensor(to_internal(b, perm, op.n_phi), device="cuda")
    x = torch.zeros_like(bd)
    info = op.dgsl_cg_solve(kind, coef, bd, x, opts=dgsl.solve_opts(tol=tol, precision=dgsl.PREC_F32_IR,
                                                                    precond=dgsl.PRECOND_MULTIGRID))[0]
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


def _residual(orc, kind, coef, b, x_nat):
    A = orc.schur_matrix(coef) if kind == 0 else orc.helmholtz_matrix(coef)
    rhs = OP.project_mean(b) if kind == 0 else b
    return np.linalg.norm(rhs - A @ x_nat) / np.linalg.norm(rhs)


def test_mg_batch_runs_requests_concurrently_and_bitwise(problems):
    from paper_2401_17806_gb300 import dgsl
    reqs, xs = [], []
    for op, orc, perm, kind, coef, b in problems:
        bd = torch.tensor(to_internal(b, perm, op.n_phi), device="cuda")
        x = torch.full_like(bd, np.nan)
        reqs.append(dgsl.request(op, kind, coef, bd, x))
        xs.append((bd, x))
    infos = dgsl.dgsl_cg_solve_batch(reqs, dgsl.engine_opts(precond=dgsl.PRECOND_MULTIGRID))
    torch.cuda.synchronize()
    for (op, orc, perm, kind, coef, b), (bd, x), info in zip(problems, xs, infos):
        assert info.status == dgsl.OK and info.relres <= 1e-10
        xa, ia = _single(op, perm, kind, coef, b)
        assert np.array_equal(x.cpu().numpy(), xa)
        assert _residual(orc, kind, coef, b, to_natural(xa, perm, op.n_phi)) <= 2e-10


def test_mg_server_admits_requests_while_others_run(problems):
    from paper_2401_17806_gb300 import dgsl
    srv = dgsl.Server(dgsl.engine_opts(precond=dgsl.PRECOND_MULTIGRID, hbm_budget_bytes=4_000_000_000))
    try:
        bufs = []
        for rep in range(3):
            for k, (op, orc, perm, kind, coef, b) in enumerate(problems):
                bd = torch.tensor(to_internal(b, perm, op.n_phi), device="cuda")
                bufs.append((k, bd, torch.full_like(bd, np.nan)))
        torch.cuda.synchronize()
        tickets = []
        for rep in range(3):
            for k, bd, x in bufs[rep * len(problems):(rep + 1) * len(problems)]:
                op, orc, perm, kind, coef, b = problems[k]
                tickets.append(srv.dgsl_submit(dgsl.request(op, kind, coef, bd, x)))
            time.sleep(0.002)
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
            op, orc, perm, kind, coef, b = problems[k]
            assert done[t].status == dgsl.OK
            xa, _ = _single(op, perm, kind, coef, b)
            assert np.array_equal(x.cpu().numpy(), xa)
        st = srv.stats()
        assert st["completed"] == len(tickets) and st["queued"] == 0 and st["bytes_in_use"] == 0
        assert st["admitted_running"] >= 1, st
    finally:
        srv.close()
