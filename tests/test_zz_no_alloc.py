"""dgsl_cg_solve_noalloc: the solve for callers that cannot allocate device
memory while they solve (services that reserve all device memory under a fixed
budget at start-up, or hosts whose own allocator owns the GPU).  It must give
the same answer as dgsl_cg_solve, bit for bit, call after call, from the
library's one fixed scratch array; leave the device's free memory unchanged;
refuse a stream that is being captured without disturbing the capture; and
refuse operators above the array's size limit.

Kept in a file that is collected last, so a run that stops at the first
failure has run every other test before it."""
import numpy as np
import pytest

from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _op(N, p, seed=3):
    from paper_2401_17806_gb300 import dgsl
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    return dgsl.Operator(xy, tri, per, p)


def _rhs(op, n_rhs, seed):
    return torch.tensor(synth.standard_normal(n_rhs * op.n_dof, seed), device="cuda")


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_bitwise_equal_to_allocating_solve_twice(dgsl_lib, prec):
    from paper_2401_17806_gb300 import dgsl
    op = _op(24, 2)
    for kind, coef, seed in [(dgsl.SCHUR, 1e-2, 1), (dgsl.HELMHOLTZ, 1e-3, 2)]:
        b = _rhs(op, 2, seed)                       # two right-hand sides in one call
        ref = torch.zeros_like(b)
        info_ref = op.dgsl_cg_solve(kind, coef, b, ref, n_rhs=2,
                                    opts=dgsl.solve_opts(tol=1e-11, precision=prec))
        for call in range(2):                       # two calls in a row share the scratch array
            x = torch.full_like(b, np.nan)
            info = op.dgsl_cg_solve_noalloc(kind, coef, b, x, n_rhs=2,
                                            opts=dgsl.solve_opts(tol=1e-11, precision=prec))
            torch.cuda.synchronize()
            for k in range(2):
                assert info[k].status == dgsl.OK, (call, k, info[k].status)
                assert info[k].relres <= 1e-11
                assert info[k].iters == info_ref[k].iters
                assert info[k].refinements == info_ref[k].refinements
                assert info[k].relres == info_ref[k].relres
            # same kernels, grids and reduction order: the same bits
            assert torch.equal(x, ref), call


def test_noalloc_leaves_free_device_memory_unchanged(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op = _op(20, 3)
    b = _rhs(op, 1, 5)
    x = torch.zeros_like(b)
    opts = dgsl.solve_opts(tol=1e-10, precision=dgsl.PREC_F32_IR)
    op.dgsl_cg_solve_noalloc(dgsl.SCHUR, 1e-2, b, x, opts=opts)   # first call: loads code, looks up the array
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        info = op.dgsl_cg_solve_noalloc(dgsl.SCHUR, 1e-2, b, x, opts=opts)[0]
        assert info.status == dgsl.OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_p1_near_the_limit_on_a_user_stream(dgsl_lib):
    """p = 1 (the CG vectors' largest share of the scratch, 32/3 n doubles) at
    259,584 DOFs, just under the 262,144 limit, two right-hand sides, on a
    stream other than the default one."""
    from paper_2401_17806_gb300 import dgsl
    op = _op(208, 1)
    assert op.n_dof == 259584
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        b = _rhs(op, 2, 9)
        ref = torch.zeros_like(b)
        x = torch.full_like(b, np.nan)
    opts = dgsl.solve_opts(tol=1e-10, precision=dgsl.PREC_F32_IR)
    info_ref = op.dgsl_cg_solve(dgsl.SCHUR, 1e-2, b, ref, n_rhs=2, opts=opts, stream=s)
    info = op.dgsl_cg_solve_noalloc(dgsl.SCHUR, 1e-2, b, x, n_rhs=2, opts=opts, stream=s)
    s.synchronize()
    for k in range(2):
        assert info[k].status == dgsl.OK and info[k].relres <= 1e-10
        assert info[k].iters == info_ref[k].iters and info[k].grid == info_ref[k].grid
    assert torch.equal(x, ref)


def test_noalloc_refuses_a_capturing_stream(dgsl_lib):
    """The solve reads residual norms back to the host every refinement step,
    so it cannot be captured: it must refuse before enqueuing anything and the
    caller's capture must still complete and replay."""
    from paper_2401_17806_gb300 import dgsl
    op = _op(12, 2)
    b = _rhs(op, 1, 4)
    x = torch.zeros_like(b)
    y = torch.zeros(16, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        y.add_(1.0)
        try:
            op.dgsl_cg_solve_noalloc(dgsl.SCHUR, 1e-2, b, x)
        except dgsl.DgslError as e:
            codes.append(e.code)
    assert codes == [dgsl.EINVAL]
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(y == 1.0)
    # the library still solves on an ordinary stream afterwards
    info = op.dgsl_cg_solve_noalloc(dgsl.SCHUR, 1e-2, b, x)[0]
    torch.cuda.synchronize()
    assert info.status == dgsl.OK


def test_noalloc_rejects_operators_above_the_limit(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op = _op(128, 3)                      # 327,680 DOFs > 262,144
    b = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(dgsl.DgslError) as e:
        op.dgsl_cg_solve_noalloc(dgsl.SCHUR, 1e-2, b, x)
    assert e.value.code == dgsl.EINVAL
    assert "262144" in str(e.value)
