"""Pins of the oracle's basis and quadrature (Sec. 2.2) against closed forms,
exact rational integrals, a library routine and the paper's worked example."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import basis as B

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_dof_counts_golden():
    for p, nphi, npsi in _golden("dof_counts.txt").astype(int):
        assert B.n_phi(p) == nphi == len(B.nodes(p))
        assert B.n_psi(p) == npsi
        L, R = B.dual_maps(p)
        assert len(set(L.tolist()) | set(R.tolist())) == npsi


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_matches_library(n):
    x, w = B.gauss_legendre(n)
    xr, wr = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(x, 0.5 * (xr + 1), atol=1e-15)
    np.testing.assert_allclose(w, 0.5 * wr, atol=1e-15)


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_duffy_rule_exact_monomials(n):
    pts, w = B.duffy_rule(n)
    for a in range(2 * n - 1):
        for b in range(2 * n - 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            got = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b)
            assert abs(got - exact) < 1e-15, (a, b)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_nodal_basis_delta_and_partition_of_unity(p):
    X = B.nodes(p)
    np.testing.assert_allclose(B.eval_phi(p, X), np.eye(len(X)), atol=1e-12)
    rng = np.random.default_rng(0)
    pts = rng.uniform(0, 0.5, size=(20, 2))
    np.testing.assert_allclose(B.eval_phi(p, pts).sum(-1), 1.0, atol=1e-12)
    np.testing.assert_allclose(B.eval_grad_phi(p, pts).sum(-2), 0.0, atol=1e-10)
    # gradient against central differences
    h = 1e-6
    for d in range(2):
        e = np.zeros(2)
        e[d] = h
        fd = (B.eval_phi(p, pts + e) - B.eval_phi(p, pts - e)) / (2 * h)
        np.testing.assert_allclose(B.eval_grad_phi(p, pts)[..., d], fd, atol=1e-6)


def _exact_mass_ref(p):
    """Mbar_ref by exact rational arithmetic: Vandermonde inverse in Fractions,
    monomial integrals a! b! / (a+b+2)!."""
    X = [(Fraction(a, p), Fraction(b, p)) for (a, b) in B.node_ab(p)]
    mono = B.monomials(p)
    n = len(X)
    V = [[x ** i * y ** j for (i, j) in mono] + [Fraction(int(r == c)) for c in range(n)]
         for r, (x, y) in enumerate(X)]
    for c in range(n):                        # Gauss-Jordan in exact arithmetic
        piv = next(r for r in range(c, n) if V[r][c] != 0)
        V[c], V[piv] = V[piv], V[c]
        pv = V[c][c]
        V[c] = [v / pv for v in V[c]]
        for r in range(n):
            if r != c and V[r][c] != 0:
                f = V[r][c]
                V[r] = [a - f * b for a, b in zip(V[r], V[c])]
    C = [row[n:] for row in V]                # C[m][k]: coeff of mono m in phi_k

    def mint(a, b):
        return Fraction(math.factorial(a) * math.factorial(b), math.factorial(a + b + 2))

    M = [[Fraction(0)] * n for _ in range(n)]
    for k in range(n):
        for l in range(n):
            s = Fraction(0)
            for m1, (i1, j1) in enumerate(mono):
                if C[m1][k] == 0:
                    continue
                for m2, (i2, j2) in enumerate(mono):
                    if C[m2][l] != 0:
                        s += C[m1][k] * C[m2][l] * mint(i1 + i2, j1 + j2)
            M[k][l] = s
    return np.array([[float(v) for v in row] for row in M])


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_reference_mass_exact_rational(p):
    pts, w = B.duffy_rule(p + 2)
    phi = B.eval_phi(p, pts)
    M = np.einsum("q,qk,ql->kl", w, phi, phi)
    np.testing.assert_allclose(M, _exact_mass_ref(p), rtol=0, atol=1e-15)


def test_p1_reference_mass_golden():
    gold = _golden("p1_reference_mass.txt") / 24.0
    np.testing.assert_allclose(_exact_mass_ref(1), gold, atol=0)


def test_p1_dual_basis_golden():
    """Paper's p = 1 example (Sec. 2.2) under the node-coincidence reading."""
    gold = _golden("p1_dual_basis.txt")
    L, R = B.dual_maps(1)
    for xi, eta, *vals in gold:
        psi = np.zeros(4)
        if xi + eta <= 1:
            psi[L] = B.eval_phi(1, np.array([[xi, eta]]))[0]
        else:
            psi[R] = B.eval_phi(1, np.array([[1 - xi, 1 - eta]]))[0]
        np.testing.assert_allclose(psi, vals, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_dual_basis_continuous_across_diagonal(p):
    """psi evaluated from the left half and from the right half agrees on
    xi + eta = 1 (C0 space of Sec. 2.2)."""
    L, R = B.dual_maps(p)
    t = np.linspace(0, 1, 13)
    diag = np.stack([1 - t, t], 1)
    left = np.zeros((len(t), B.n_psi(p)))
    right = np.zeros_like(left)
    left[:, L] = B.eval_phi(p, diag)
    right[:, R] = B.eval_phi(p, 1 - diag)
    np.testing.assert_allclose(left, right, atol=1e-12)
