"""Pins of the oracle's operators (Sec. 2.3-2.4): adjointness, the mass
scalings of eqs. MassMatrixM / MassMatrixD, the 12-reference-operator
decomposition, polynomial reproduction, nullspace and invariances."""
import numpy as np
import pytest

from oracle import assemble as OA
from oracle import basis as B
from oracle import fields as OF
from oracle import operators as OP
from paper_2401_17806_gb300 import synth

_CACHE = {}


def ops(N, p, seed=1, xy_tf=None, per=None):
    key = (N, p, seed)
    if xy_tf is None and key in _CACHE:
        return _CACHE[key]
    xy, tri, period = synth.jittered_periodic_mesh(N, seed)
    if xy_tf is not None:
        xy = xy_tf(xy)
    if per is not None:
        period = per
    op = OP.Operators(OA.assemble(xy, tri, period, p))
    if xy_tf is None:
        _CACHE[key] = op
    return op


def _ref_mass(p):
    pts, w = B.duffy_rule(p + 2)
    phi = B.eval_phi(p, pts)
    return np.einsum("q,qk,ql->kl", w, phi, phi)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_adjointness(p):
    """D = -Q^T (Sec. 2.3, after eq. ad5), both assembled independently."""
    bl = ops(4, p).bl
    scale = np.abs(bl.Q).max()
    assert np.abs(bl.D + np.swapaxes(bl.Q, 2, 3)).max() <= 1e-14 * scale


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_mass_scalings(p):
    """eq. MassMatrixM: Mbar_i = A_i Mbar_ref; eq. MassMatrixD: Mhat_j =
    A_lj M^L + A_rj M^R with A_ij = A_i / 3; partition of unity."""
    bl = ops(4, p).bl
    Mref = _ref_mass(p)
    np.testing.assert_allclose(bl.Mbar, bl.area2[:, None, None] * Mref, rtol=1e-13, atol=1e-17)
    L, R = B.dual_maps(p)
    npsi = B.n_psi(p)
    ML = np.zeros((npsi, npsi))
    MR = np.zeros((npsi, npsi))
    ML[np.ix_(L, L)] = Mref
    MR[np.ix_(R, R)] = Mref
    A = bl.area2[bl.conn.lr] / 3.0
    expect = A[:, 0, None, None] * ML + A[:, 1, None, None] * MR
    np.testing.assert_allclose(bl.Mhat, expect, rtol=1e-13, atol=1e-17)
    np.testing.assert_allclose(bl.Mbar.sum((1, 2)), bl.area2 / 2, rtol=1e-13)
    np.testing.assert_allclose(bl.Mhat.sum((1, 2)), A.sum(1) / 2, rtol=1e-13)


def _reference_operators(p):
    """The 12 reference operators of Sec. 2.4 (D^{L,a,b}, D^{V,a,b}), built on
    T_ref with the dual halves mapped by node coincidence."""
    L, R = B.dual_maps(p)
    nphi, npsi = B.n_phi(p), B.n_psi(p)
    nu = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    bref = nu.mean(0)
    pts, w = B.duffy_rule(p + 2)
    tau, wt = B.gauss_legendre(p + 2)
    DL = np.zeros((3, 2, nphi, npsi))
    DV = np.zeros((3, 2, nphi, npsi, 2))
    for a in range(3):
        va, vb = nu[a], nu[(a + 1) % 3]
        xi = bref + pts[:, :1] * (va - bref) + pts[:, 1:] * (vb - bref)   # T_alpha^{-1}(zeta)
        g = B.eval_grad_phi(p, xi)
        ps = B.eval_phi(p, pts)
        xe = va + tau[:, None] * (vb - va)
        phe = B.eval_phi(p, xe)
        pse = B.eval_phi(p, np.stack([1 - tau, tau], 1))
        for b, (perm, sg) in enumerate([(L, 1.0), (R, -1.0)]):
            DV[a, b][:, perm] = np.einsum("q,qkd,qm->kmd", w, g, ps)
            DL[a, b][:, perm] = sg * np.einsum("q,qk,qm->km", wt, phe, pse)
    return DL, DV


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_reference_operator_decomposition(p):
    """D_ij = |G_j| n_j D^{L,a,b} - A_ij J_i . D^{V,a,b}  (Sec. 2.4)."""
    op = ops(4, p)
    bl = op.bl
    c = bl.conn
    DL, DV = _reference_operators(p)
    for side in range(2):
        i = c.lr[:, side]
        a = c.loc[:, side].astype(int)
        P = c.tri_xy[i]
        Jinv = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]], -1)   # J(T^{-1}) = dx/dxi
        J = np.linalg.inv(Jinv)                                        # J(T) = dxi/dx
        Aij = bl.area2[i] / 3.0
        line = (bl.length[:, None] * bl.normal)[:, None, None, :] * DL[a, side][..., None]
        # (J_i . D^V)[k,l,c] = sum_d J(T)[d, c] D^V[k,l,d]
        vol = Aij[:, None, None, None] * np.einsum("edc,ekld->eklc", J, DV[a, side])
        np.testing.assert_allclose(bl.D[:, side], line - vol, rtol=0,
                                   atol=1e-13 * np.abs(bl.D).max())


def _poly(p, seed):
    rng = np.random.default_rng(seed)
    coef = {(i, j): rng.standard_normal() for i in range(p + 1) for j in range(p + 1 - i)}

    def P(x, y):
        return sum(c * x ** i * y ** j for (i, j), c in coef.items())

    def dP(x, y):
        gx = sum(c * i * x ** (i - 1) * y ** j for (i, j), c in coef.items() if i > 0)
        gy = sum(c * j * x ** i * y ** (j - 1) for (i, j), c in coef.items() if j > 0)
        return gx + 0 * x, gy + 0 * x
    return P, dP


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_gradient_reproduces_polynomials(p):
    """For a continuous polynomial of degree <= p the jump term of eq. ad5.2
    vanishes and Mhat^{-1} (Q_l x_l + Q_r x_r) is the gradient at the dual
    nodes (the gradient lies in the C0 dual space)."""
    op = ops(5, p)
    c = op.bl.conn
    P, dP = _poly(p, 7)
    X = OF.main_nodes(c, p)
    x = P(X[..., 0], X[..., 1]).ravel()
    g = op.apply_Mhat_inv(op.G @ x).reshape(2, op.nd, op.npsi)
    Y = OF.dual_nodes(c, p)
    gx, gy = dP(Y[..., 0], Y[..., 1])
    ok = np.all(c.shift == 0, 1)
    assert ok.sum() > op.nd // 3
    scale = np.abs(gx).max() + np.abs(gy).max()
    assert np.abs(g[0][ok] - gx[ok]).max() < 1e-10 * scale
    assert np.abs(g[1][ok] - gy[ok]).max() < 1e-10 * scale


@pytest.mark.parametrize("p", [1, 2, 3])
def test_projections_reproduce_polynomials(p):
    """eq. m2d and eq. d2m are L2 projections: identity on polynomials of
    degree <= p."""
    op = ops(5, p)
    c = op.bl.conn
    P, _ = _poly(p, 11)
    X = OF.main_nodes(c, p)
    vbar = P(X[..., 0], X[..., 1]).ravel()
    Y = OF.dual_nodes(c, p)
    vhat_exact = P(Y[..., 0], Y[..., 1])
    vhat = op.m2d(vbar).reshape(op.nd, op.npsi)
    ok = np.all(c.shift == 0, 1)
    np.testing.assert_allclose(vhat[ok], vhat_exact[ok], atol=1e-10)
    back = op.d2m(vhat_exact.ravel()).reshape(c.n_tri, -1)
    tri_ok = np.all(ok[c.tri_edge], 1)
    assert tri_ok.sum() > 0
    np.testing.assert_allclose(back[tri_ok], vbar.reshape(c.n_tri, -1)[tri_ok], atol=1e-10)


@pytest.mark.parametrize("N", [3, 4])
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_schur_symmetric_semidefinite_one_dim_nullspace(N, p):
    """eq. pressure_final: symmetric, semidefinite, kernel = constants (dense
    eigendecomposition)."""
    op = ops(N, p)
    S = op.schur_matrix(0.1).toarray()
    nrm = np.abs(S).max()
    assert np.abs(S - S.T).max() <= 1e-14 * nrm
    assert np.abs(S @ np.ones(op.n)).max() <= 1e-13 * nrm
    ev = np.linalg.eigvalsh(S)
    tol = 1e-11 * ev[-1]
    assert np.sum(np.abs(ev) <= tol) == 1
    assert np.all(ev[1:] > tol)


def test_invariances():
    """S is invariant under translation, rotation by 90 degrees and uniform
    scaling of the mesh; Mbar scales with the area."""
    p = 2
    base = ops(4, p, seed=5)
    K0 = base.K().toarray()
    s = 2.5
    for tf, per, msc in [
        (lambda z: z + np.array([0.31, 0.77]), None, 1.0),
        (lambda z: np.stack([-z[:, 1], z[:, 0]], 1), None, 1.0),
        (lambda z: s * z, np.array([s, s]), s * s),
    ]:
        o = ops(4, p, seed=5, xy_tf=tf, per=per)
        np.testing.assert_allclose(o.K().toarray(), K0, atol=1e-12 * np.abs(K0).max())
        np.testing.assert_allclose(o.bl.Mbar, msc * base.bl.Mbar, rtol=1e-12,
                                   atol=1e-13 * msc * np.abs(base.bl.Mbar).max())


def test_relabelling_permutes_schur():
    """The left/right assignment is arbitrary (Sec. 2.1): relabelling the
    triangles (which swaps l and r on many edges) permutes S."""
    p = 2
    xy, tri, per = synth.jittered_periodic_mesh(4, 9)
    rng = np.random.default_rng(0)
    pi = rng.permutation(len(tri))
    o0 = OP.Operators(OA.assemble(xy, tri, per, p))
    o1 = OP.Operators(OA.assemble(xy, tri[pi], per, p))
    nphi = B.n_phi(p)
    dof = (pi[:, None] * nphi + np.arange(nphi)).ravel()
    K0 = o0.K().toarray()
    K1 = o1.K().toarray()
    np.testing.assert_allclose(K1, K0[np.ix_(dof, dof)], atol=1e-12 * np.abs(K0).max())


def test_helmholtz_zero_viscosity_is_mass():
    op = ops(4, 3)
    H = op.helmholtz_matrix(0.0).toarray()
    Mref = _ref_mass(3)
    n = B.n_phi(3)
    for i in range(op.bl.conn.n_tri):
        blk = H[i * n:(i + 1) * n, i * n:(i + 1) * n]
        np.testing.assert_allclose(blk, op.bl.area2[i] * Mref, rtol=1e-13,
                                   atol=1e-14 * op.bl.area2[i] * np.abs(Mref).max())
    off = H.copy()
    for i in range(op.bl.conn.n_tri):
        off[i * n:(i + 1) * n, i * n:(i + 1) * n] = 0
    assert np.abs(off).max() == 0
