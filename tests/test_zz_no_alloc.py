"""dgsl_cg_solve_noalloc: the solve for callers that cannot allocate device
memory while they solve (inside stream capture, under a fixed reserved memory
budget, or where another allocator owns the GPU).  It must give the same
answer as dgsl_cg_solve, call after call, from the library's one fixed scratch
array, and refuse operators above that array's size limit.

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


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_allocating_solve_twice(dgsl_lib, prec):
    from paper_2401_17806_gb300 import dgsl
    op = _op(24, 2)
    opts = dgsl.solve_opts(tol=1e-11, precision=prec)
    for kind, coef, seed in [(dgsl.SCHUR, 1e-2, 1), (dgsl.HELMHOLTZ, 1e-3, 2)]:
        b = torch.tensor(synth.standard_normal(op.n_dof, seed), device="cuda")
        ref = torch.zeros_like(b)
        info_ref = op.dgsl_cg_solve(kind, coef, b, ref, opts=opts)[0]
        for call in range(2):            # two calls in a row share the scratch array
            x = torch.full_like(b, np.nan)
            info = op.dgsl_cg_solve_noalloc(kind, coef, b, x, opts=dgsl.solve_opts(
                tol=1e-11, precision=prec))[0]
            torch.cuda.synchronize()
            assert info.status == dgsl.OK, (call, info.status)
            assert info.relres <= 1e-11
            xr, xn = ref.cpu().numpy(), x.cpu().numpy()
            # same tolerance as the solver parity tests
            assert np.linalg.norm(xn - xr) / np.linalg.norm(xr) <= 1e-10, call
            assert info.iters == info_ref.iters


def test_noalloc_rejects_operators_above_the_limit(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    op = _op(128, 3)                      # 327,680 DOFs > 262,144
    b = torch.zeros(op.n_dof, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(dgsl.DgslError) as e:
        op.dgsl_cg_solve_noalloc(dgsl.SCHUR, 1e-2, b, x)
    assert e.value.code == dgsl.EINVAL
    assert "262144" in str(e.value)
