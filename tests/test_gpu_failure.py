"""Failure detection on the GPU without a fault: the persistent solvers' waits
are bounded.  A grid barrier that expects a CTA that never comes and an
mbarrier that no copy completes must give up after a short limit, report
DGSL_ETIMEOUT, and leave the context usable for the next solve."""
import time

import numpy as np
import pytest

from paper_2401_17806_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_times_out_and_context_survives(dgsl_lib, which):
    from paper_2401_17806_gb300 import dgsl
    t = time.time()
    assert dgsl.dgsl_selftest_wait_timeout(which, 0.2) == dgsl.ETIMEOUT
    assert time.time() - t < 30
    # the device still solves correctly afterwards
    xy, tri, per = synth.jittered_periodic_mesh(8, 0)
    op = dgsl.Operator(xy, tri, per, 2)
    b = torch.tensor(synth.standard_normal(op.n_dof, 1), device="cuda")
    x = torch.zeros_like(b)
    info = op.dgsl_cg_solve(dgsl.SCHUR, 1e-2, b, x, opts=dgsl.solve_opts(precision=dgsl.PREC_F32_IR))[0]
    assert info.status == dgsl.OK and info.relres <= 1e-10
    assert np.isfinite(x.cpu().numpy()).all()


def test_selftest_rejects_bad_arguments(dgsl_lib):
    from paper_2401_17806_gb300 import dgsl
    with pytest.raises(dgsl.DgslError):
        dgsl.dgsl_selftest_wait_timeout(2, 0.2)
    with pytest.raises(dgsl.DgslError):
        dgsl.dgsl_selftest_wait_timeout(0, 60.0)
