"""Pins of the oracle's block-Jacobi preconditioned CG (an extension: the
paper runs CG unpreconditioned).  Where A is block diagonal (the Helmholtz
operator at nu dt = 0 is the mass matrix of eq. Mi) the preconditioner is A^-1
and PCG must finish in one step; under P = I it must be plain CG, iterate for
iterate; the spectrum of P S must lie in [0, 4] with one zero eigenvalue (at
most 4 nonzero blocks per block row: the triangle and its 3 neighbours; the
nullspace span{1}); and its solution must be the direct solve's."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import assemble as OA
from oracle import operators as OP
from paper_2401_17806_gb300 import synth


def _ops(N, p, seed=5):
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    return OP.Operators(OA.assemble(xy, tri, per, p))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_block_diagonal_operator_converges_in_one_step(p):
    op = _ops(4, p)
    A = op.helmholtz_matrix(0.0)
    P = OP.block_jacobi_blocks(A, op.nphi)
    np.testing.assert_allclose(P, np.linalg.inv(op.bl.Mbar), rtol=1e-10, atol=0)
    b = synth.standard_normal(op.n, 7)
    x, it, rel = OP.pcg(lambda v: A @ v, b, lambda v: OP.apply_blocks(P, v), tol=1e-12)
    assert it == 1 and rel < 1e-12
    np.testing.assert_allclose(op.apply_Mbar(x), b, atol=1e-12 * np.abs(b).max())


def test_identity_preconditioner_is_plain_cg():
    op = _ops(6, 2)
    dt = 1e-2
    b = synth.standard_normal(op.n, 8)
    x1, it1, r1 = OP.cg(lambda v: op.apply_schur(v, dt), b, tol=1e-11, mean_zero=True)
    x2, it2, r2 = OP.pcg(lambda v: op.apply_schur(v, dt), b, lambda v: v.copy(), tol=1e-11, mean_zero=True)
    assert it1 == it2
    np.testing.assert_allclose(x2, x1, rtol=0, atol=1e-10 * np.abs(x1).max())
    assert abs(r1 - r2) <= 1e-3 * r1


@pytest.mark.parametrize("p", [1, 3])
def test_preconditioned_spectrum(p):
    op = _ops(4, p)
    S = op.schur_matrix(0.1).toarray()
    P = OP.block_jacobi_blocks(S, op.nphi)
    D = sla.block_diag(*[np.linalg.inv(Pi) for Pi in P])
    lam = sla.eigh(S, D, eigvals_only=True)
    assert lam[-1] <= 4.0 + 1e-9
    assert abs(lam[0]) < 1e-9 * lam[-1]
    assert lam[1] > 1e-6 * lam[-1]


@pytest.mark.parametrize("p", [2, 4])
def test_pcg_matches_direct_and_saves_iterations(p):
    op = _ops(8, p)
    b = synth.standard_normal(op.n, 9)
    dt = 1e-2
    S = op.schur_matrix(dt)
    P = OP.block_jacobi_blocks(S, op.nphi)
    xd = OP.schur_solve_direct(S, b)
    x, it, rel = OP.pcg(lambda v: S @ v, b, lambda v: OP.apply_blocks(P, v), tol=1e-12, mean_zero=True)
    assert rel <= 1e-12
    np.testing.assert_allclose(x, xd, atol=1e-8 * np.abs(xd).max())
    _, it0, _ = OP.cg(lambda v: S @ v, b, tol=1e-12, mean_zero=True)
    assert it < it0
    nu_dt = 1e-4
    H = op.helmholtz_matrix(nu_dt)
    PH = OP.block_jacobi_blocks(H, op.nphi)
    xh = OP.direct_solve(H, b)
    x, it, rel = OP.pcg(lambda v: H @ v, b, lambda v: OP.apply_blocks(PH, v), tol=1e-12)
    np.testing.assert_allclose(x, xh, atol=1e-10 * np.abs(xh).max())
    _, it0, _ = OP.cg(lambda v: H @ v, b, tol=1e-12)
    assert it < it0
