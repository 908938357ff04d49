"""Pins of the oracle's condition-number estimate from CG coefficients (the
Lanczos connection of CG, used to decide which solves must meet the 1e-10
error bar): on small systems run to n steps it must give the extreme
eigenvalues of a dense eigendecomposition (for the Schur operator the
smallest nonzero one, its nullspace being span{1}); a diagonal matrix with a
known spectrum must come back exactly; and a few steps must bracket the
spectrum from inside."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import operators as OP
from paper_2401_17806_gb300 import synth


def test_known_diagonal_spectrum():
    d = np.linspace(1.0, 50.0, 40)
    lo, hi, k = OP.cg_lanczos_extremes(lambda v: d * v, np.ones(40), 40)
    assert k == 40
    assert abs(lo - 1.0) <= 1e-9 and abs(hi - 50.0) <= 1e-9


@pytest.mark.parametrize("p", [1, 2])
def test_schur_extremes_match_dense_eigh(p):
    xy, tri, per = synth.jittered_periodic_mesh(4, 3)
    op = OP.Operators(OA.assemble(xy, tri, per, p))
    dt = 1e-2
    S = op.schur_matrix(dt).toarray()
    ev = np.linalg.eigvalsh(S)
    assert ev[0] < 1e-12 * ev[-1] < ev[1]           # one zero eigenvalue
    b = synth.standard_normal(op.n, 4)
    # finite-precision CG needs more than n steps to resolve the bottom of
    # the spectrum; it stops by itself once the residual is at rounding level
    lo, hi, k = OP.cg_lanczos_extremes(lambda v: S @ v, b, 4 * op.n, mean_zero=True)
    assert abs(hi - ev[-1]) <= 1e-8 * ev[-1]
    assert abs(lo - ev[1]) <= 1e-5 * ev[1]
    # a few steps: estimates lie inside the spectrum
    lo5, hi5, _ = OP.cg_lanczos_extremes(lambda v: S @ v, b, 5, mean_zero=True)
    assert ev[1] * (1 - 1e-12) <= lo5 and hi5 <= ev[-1] * (1 + 1e-12)


def test_helmholtz_extremes_match_dense_eigh():
    xy, tri, per = synth.jittered_periodic_mesh(4, 6)
    op = OP.Operators(OA.assemble(xy, tri, per, 2))
    H = op.helmholtz_matrix(1e-3).toarray()
    ev = np.linalg.eigvalsh(H)
    lo, hi, _ = OP.cg_lanczos_extremes(lambda v: H @ v, synth.standard_normal(op.n, 2), 4 * op.n)
    assert abs(hi - ev[-1]) <= 1e-8 * ev[-1] and abs(lo - ev[0]) <= 1e-5 * ev[0]
