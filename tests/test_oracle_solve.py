"""Pins of the oracle's solves: brute-force pseudo-inverse, CG against the
direct solve, the exactness variant and manufactured convergence at order
>= p + 1/2 (the paper's scheme-level orders, Sec. 4)."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import fields as OF
from oracle import operators as OP
from paper_2401_17806_gb300 import synth


def _ops(N, p, seed=3):
    xy, tri, per = synth.jittered_periodic_mesh(N, seed)
    return OP.Operators(OA.assemble(xy, tri, per, p))


@pytest.mark.parametrize("p", [1, 3])
def test_grounded_solve_equals_pseudo_inverse(p):
    op = _ops(3, p)
    S = op.schur_matrix(0.05)
    b = synth.standard_normal(op.n, 1)
    x = OP.schur_solve_direct(S, b)
    xp = np.linalg.pinv(S.toarray(), rtol=1e-10, hermitian=True) @ b
    np.testing.assert_allclose(x, xp, atol=1e-9 * np.abs(xp).max())
    assert abs(x.sum()) < 1e-9 * np.abs(x).max()


@pytest.mark.parametrize("p", [1, 2])
def test_cg_matches_direct(p):
    op = _ops(6, p)
    dt = 1e-2
    b = synth.standard_normal(op.n, 2)
    xd = OP.schur_solve_direct(op.schur_matrix(dt), b)
    xc, it, rel = OP.cg(lambda v: op.apply_schur(v, dt), b, tol=1e-13, mean_zero=True)
    assert rel <= 1e-13
    np.testing.assert_allclose(xc, xd, atol=1e-9 * np.abs(xd).max())
    nu_dt = 1e-3
    H = op.helmholtz_matrix(nu_dt)
    xh = OP.direct_solve(H, b)
    xc, it, rel = OP.cg(lambda v: op.apply_helmholtz(v, nu_dt), b, tol=1e-13)
    np.testing.assert_allclose(xc, xh, atol=1e-10 * np.abs(xh).max())


def test_exactness_variant():
    """b = S Pi(p_ex): the mean-zero solution is Pi(p_ex) - mean."""
    p = 2
    op = _ops(8, p)
    c = op.bl.conn
    X = OF.main_nodes(c, p)
    pe = synth.manufactured_pressure(X[..., 0], X[..., 1])[0].ravel()
    S = op.schur_matrix(1e-2)
    x = OP.schur_solve_direct(S, S @ pe)
    np.testing.assert_allclose(x, pe - pe.mean(), atol=1e-9)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_manufactured_convergence_order(p):
    """K_h x = int phi f with f = -Laplace(p_ex): L2 error order >= p + 1/2."""
    errs = []
    for N in (8, 16):
        op = _ops(N, p)
        c = op.bl.conn
        f = lambda x, y: synth.manufactured_pressure(x, y)[1]
        b = OF.load_vector(c, p, f)
        x = OP.schur_solve_direct(op.K(), b)
        ones = np.ones(op.n)
        x = x - (ones @ op.apply_Mbar(x)) / (ones @ op.apply_Mbar(ones))
        errs.append(OF.l2_error(c, p, x, lambda X, Y: synth.manufactured_pressure(X, Y)[0]))
    order = np.log2(errs[0] / errs[1])
    assert order >= p + 0.5, (errs, order)


@pytest.mark.parametrize("p", [1, 2, 4])
def test_velocity_update_is_divergence_free(p):
    """Projection of eqs. nc.1-nc.2: with S p = G^T F the updated velocity
    vhat = F - dt^2 Mhat^{-1} G p has zero discrete divergence, both as G^T vhat
    and with the paper's divergence D assembled on its own (D = -Q^T)."""
    op = _ops(6, p, seed=5)
    dt = 0.02
    F = synth.standard_normal(2 * op.nd * op.npsi, 61)
    b = op.G.T @ F
    pr = OP.schur_solve_direct(op.schur_matrix(dt), b)
    v = op.velocity_update(F, pr, dt * dt)
    assert np.linalg.norm(op.G.T @ v) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(op.Dm @ v) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(v - F) > 1e-3 * np.linalg.norm(F)  # something was removed


@pytest.mark.parametrize("p", [1, 3])
def test_velocity_update_removes_discrete_gradients(p):
    """A dual field that is itself dt^2 Mhat^{-1} G q (a discrete pressure
    gradient) is projected to zero: the solve recovers q up to a constant and
    G annihilates constants."""
    op = _ops(5, p, seed=8)
    dt = 0.05
    q = synth.standard_normal(op.n, 62)
    F = dt * dt * op.apply_Mhat_inv(op.G @ q)
    pr = OP.schur_solve_direct(op.schur_matrix(dt), op.G.T @ F)
    np.testing.assert_allclose(pr, q - q.mean(), atol=1e-8 * np.abs(q).max())
    v = op.velocity_update(F, pr, dt * dt)
    assert np.linalg.norm(v) <= 1e-9 * np.linalg.norm(F)
