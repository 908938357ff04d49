"""GPU parity of the batched persistent engine (many solves, different meshes,
degrees and kinds, in one launch; requests with several right-hand sides) and
of the serving loop (continuous batching under a memory budget), through the
C-ABI, against the oracle's FP64 operators; each result must be the same alone,
in the mix and inside a multi-RHS request."""
import time

import numpy as np
import pytest

from oracle import assemble as OA
from oracle import operators as OP
from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from test_gpu_apply import to_internal, to_natural  # noqa: E402

CASES = [(6, 1, 0, 1e-2), (9, 2, 1, 1e-3), (13, 3, 0, 1e-3), (8, 4, 1, 2e-3), (20, 2, 0, 1e-2), (11, 3, 1, 5e-4)]


@pytest.fixture(scope="module")
def problems(dgsl_lib):
    """(operator, oracle, perm, kind, coef, b_natural) for a mixed set."""
    from paper_2401_17806_gb300 import dgsl
    out = []
    for k, (N, p, kind, coef) in enumerate(CASES):
        xy, tri, per = synth.jittered_periodic_mesh(N, 40 + k)
        op = dgsl.Operator(xy, tri, per, p, store=dgsl.STORE_F64 | dgsl.STORE_F32 | dgsl.STORE_BF16)
        orc = OP.Operators(OA.assemble(xy, tri, per, p))
        b = synth.standard_normal(op.n_dof, 70 + k)
        out.append((op, orc, op.maps()["perm"], kind, coef, b))
    return out


def _run_batch(items, opts):
    from paper_2401_17806_gb300 import dgsl
    xs, reqs = [], []
    for op, orc, perm, kind, coef, b in items:
        bd = torch.tensor(to_internal(b, perm, op.n_phi), device="cuda")
        x = torch.full_like(bd, np.nan)
        reqs.append(dgsl.request(op, kind, coef, bd, x))
        xs.append((bd, x))
    infos = dgsl.dgsl_cg_solve_batch(reqs, opts)
    torch.cuda.synchronize()
    return [x.cpu().numpy() for _, x in xs], infos


def _check_residual(orc, kind, coef, b, x_nat, tol):
    if kind == 0:
        A = orc.schur_matrix(coef)
        rhs = OP.project_mean(b)
        assert abs(x_nat.sum()) <= 1e-9 * np.abs(x_nat).sum()
    else:
        A = orc.helmholtz_matrix(coef)
        rhs = b
    rel = np.linalg.norm(rhs - A @ x_nat) / np.linalg.norm(rhs)
    assert rel <= tol, rel


def test_batch_mixed_fp32(problems):
    from paper_2401_17806_gb300 import dgsl
    opts = dgsl.engine_opts(precision=dgsl.PREC_F32_IR)
    xs, infos = _run_batch(problems, opts)
    for (op, orc, perm, kind, coef, b), x, info in zip(problems, xs, infos):
        assert info.status == dgsl.OK, info.status
        assert info.relres <= 1e-10
        _check_residual(orc, kind, coef, b, to_natural(x, perm, op.n_phi), 2e-10)
        # the direct solution
        if kind == 0:
            xd = OP.schur_solve_direct(orc.schur_matrix(coef), b)
        else:
            xd = OP.direct_solve(orc.helmholtz_matrix(coef), b)
        xn = to_natural(x, perm, op.n_phi)
        ev = np.linalg.eigvalsh((orc.schur_matrix(coef) if kind == 0 else orc.helmholtz_matrix(coef)).toarray())
        kappa = ev[-1] / (ev[1] if kind == 0 else ev[0])
        assert np.linalg.norm(xn - xd) / np.linalg.norm(xd) <= max(1e-9, 10 * kappa * 1e-10)


def test_batch_results_same_alone_and_in_the_mix(problems):
    from paper_2401_17806_gb300 import dgsl
    opts = dgsl.engine_opts(precision=dgsl.PREC_F32_IR)
    mixed, _ = _run_batch(problems, opts)
    for k in (0, 3, 5):
        alone, info = _run_batch([problems[k]], opts)
        assert info[0].status == dgsl.OK
        assert np.array_equal(alone[0], mixed[k])
    # and the mix is deterministic run to run
    again, _ = _run_batch(problems, opts)
    for a, b in zip(mixed, again):
        assert np.array_equal(a, b)


def test_batch_bf16_reports_status(problems):
    from paper_2401_17806_gb300 import dgsl
    opts = dgsl.engine_opts(precision=dgsl.PREC_BF16_IR, max_refine=60)
    xs, infos = _run_batch(problems[:3], opts)
    for (op, orc, perm, kind, coef, b), x, info in zip(problems[:3], xs, infos):
        assert info.status in (dgsl.OK, dgsl.ENOTCONV)
        if info.status == dgsl.OK:
            _check_residual(orc, kind, coef, b, to_natural(x, perm, op.n_phi), 2e-10)


def test_batch_zero_rhs_and_validation(problems):
    from paper_2401_17806_gb300 import dgsl
    op, orc, perm, kind, coef, b = problems[1]
    z = [(op, orc, perm, kind, coef, np.zeros(op.n_dof))] + [problems[2]]
    xs, infos = _run_batch(z, dgsl.engine_opts())
    assert infos[0].status == dgsl.OK and np.all(xs[0] == 0)
    assert infos[1].status == dgsl.OK
    bd = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    bad = dgsl.request(op, 5, coef, bd, bd.clone())
    with pytest.raises(dgsl.DgslError):
        dgsl.dgsl_cg_solve_batch([bad], dgsl.engine_opts())


@pytest.mark.parametrize("R", [3, 8])
def test_batch_multi_rhs_equals_single(problems, R):
    """A request with R right-hand sides shares the coupling stream but gives
    every right-hand side the same result, bit for bit, as a request of its
    own; results meet the oracle's residual bar."""
    from paper_2401_17806_gb300 import dgsl
    opts = dgsl.engine_opts(precision=dgsl.PREC_F32_IR)
    for k in (1, 3, 5):
        op, orc, perm, kind, coef, b = problems[k]
        bs = [synth.standard_normal(op.n_dof, 900 + 17 * k + j) for j in range(R)]
        if R == 3:
            bs[1] = np.zeros(op.n_dof)  # a zero right-hand side inside a block
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
            keep.append(bj)  # requests hold raw pointers: the tensors must stay alive
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
        assert info.iters == max(i.iters for i in infos)
        assert info.relres == max(i.relres for i in infos)


def test_batch_rejects_bad_n_rhs(problems):
    from paper_2401_17806_gb300 import dgsl
    op, orc, perm, kind, coef, b = problems[0]
    bd = torch.zeros(9 * op.n_dof, dtype=torch.float64, device="cuda")
    with pytest.raises(dgsl.DgslError):
        dgsl.request(op, kind, coef, bd, bd.clone(), n_rhs=9)
    r = dgsl.request(op, kind, coef, bd[:op.n_dof], bd[:op.n_dof].clone())
    r.n_rhs = 9
    with pytest.raises(dgsl.DgslError):
        dgsl.dgsl_cg_solve_batch([r], dgsl.engine_opts())


def test_server_continuous_batching(problems):
    """Requests submitted while the engine runs join it (the server counts the
    requests admitted by a launch that was already running, and there are
    fewer launches than submission rounds); every result equals its
    batch-of-one result bitwise; budget and cancellation behave."""
    from paper_2401_17806_gb300 import dgsl
    # the engine idles up to 50 ms for new work, far longer than the 2 ms
    # between submission rounds, so later rounds arrive at a running launch
    opts = dgsl.engine_opts(precision=dgsl.PREC_F32_IR, hbm_budget_bytes=2_000_000_000, idle_us=50000)
    srv = dgsl.Server(opts)
    try:
        # every buffer is allocated before the first submission: a device
        # allocation (cudaMalloc) may wait for the whole device, the running
        # engine included, and would serialise the rounds
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
        ref, _ = _run_batch(problems, opts)
        for (k, bd, x), t in zip(bufs, tickets):
            assert done[t].status == dgsl.OK
            assert np.array_equal(x.cpu().numpy(), ref[k])
        st = srv.stats()
        assert st["completed"] == len(tickets) and st["queued"] == 0 and st["bytes_in_use"] == 0
        assert 1 <= st["engine_launches"] < 3
        # continuous batching: requests joined a launch already on the device
        assert st["admitted_running"] >= len(problems), st
        # a request larger than the whole budget is refused
        big = dgsl.Server(dgsl.engine_opts(hbm_budget_bytes=1_000_000))
        op, orc, perm, kind, coef, b = problems[4]
        bd = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
        with pytest.raises(dgsl.DgslError) as e:
            big.dgsl_submit(dgsl.request(op, kind, coef, bd, bd.clone()))
        assert e.value.code == dgsl.EBUDGET
        big.close()
        with pytest.raises(dgsl.DgslError):
            srv.dgsl_poll(123456789)
    finally:
        srv.close()


def test_server_budget_queues_and_cancel(problems):
    from paper_2401_17806_gb300 import dgsl
    op, orc, perm, kind, coef, b = problems[4]
    # room for the operator and about one workspace at a time
    budget = op.device_bytes + 60 * op.n_dof
    srv = dgsl.Server(dgsl.engine_opts(hbm_budget_bytes=int(budget), idle_us=0))
    try:
        bd = torch.tensor(to_internal(b, perm, op.n_phi), device="cuda")
        xs = [torch.zeros_like(bd) for _ in range(4)]
        ts = [srv.dgsl_submit(dgsl.request(op, kind, coef, bd, x)) for x in xs]
        cancelled = srv.dgsl_cancel(ts[-1])
        got = {}
        t0 = time.time()
        live = ts[:-1] if cancelled else ts
        while len(got) < len(live) and time.time() - t0 < 120:
            for t in live:
                if t not in got:
                    info = srv.dgsl_poll(t)
                    if info is not None:
                        got[t] = info
            time.sleep(0.001)
        assert len(got) == len(live)
        for t in live:
            assert got[t].status == dgsl.OK
        for x in xs[:len(live)]:
            assert np.array_equal(x.cpu().numpy(), xs[0].cpu().numpy())
    finally:
        srv.close()
