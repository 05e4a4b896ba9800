"""Pins of the oracle's bases and quadrature against closed forms (Sec. 3)."""
import math

import numpy as np
import pytest

from oracle.basis import RefBasis, TimeBasis, gauss_legendre01, monomial_exponents
from oracle.quadrature import map_rule, ref_simplex_rule


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_nodal_basis_is_lagrange_and_partition_of_unity(dim, p):
    b = RefBasis(dim, p)
    assert b.n == math.comb(p + dim, dim)
    np.testing.assert_allclose(b.values(b.nodes), np.eye(b.n), atol=1e-11)
    rng = np.random.default_rng(0)
    x = rng.dirichlet(np.ones(dim + 1), size=50)[:, :dim]
    np.testing.assert_allclose(b.values(x).sum(axis=1), 1.0, atol=1e-12)
    np.testing.assert_allclose(b.grads(x).sum(axis=1), 0.0, atol=1e-10)


def test_node_order_lexicographic():
    b = RefBasis(2, 2)
    np.testing.assert_allclose(b.nodes, [[0, 0], [.5, 0], [1, 0], [0, .5], [.5, .5], [0, 1]])
    b3 = RefBasis(3, 1)
    np.testing.assert_allclose(b3.nodes, [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])


def test_graded_lex_monomials():
    e = monomial_exponents(2, 2)
    assert [tuple(r) for r in e] == [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]
    e3 = monomial_exponents(3, 2)
    assert [tuple(r) for r in e3][:4] == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)]
    assert [tuple(r) for r in e3][4:] == [(2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2)]


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_simplex_rule_exact_on_monomials(dim):
    # int over the unit simplex of x^a = prod(a_k!) / (|a| + dim)!
    n = 5
    pts, wts = ref_simplex_rule(dim, n)
    top = 2 * n - 1 - (dim - 1)
    for a in monomial_exponents(dim, top):
        exact = np.prod([math.factorial(int(k)) for k in a]) / math.factorial(int(a.sum()) + dim)
        got = np.sum(wts * np.prod(pts ** a, axis=1))
        assert abs(got - exact) < 1e-14 * max(1.0, exact) + 1e-16, (a, got, exact)


def test_p1_mass_closed_form():
    # P1 mass matrix on a triangle: |T|/12 [[2,1,1],[1,2,1],[1,1,2]]; on a tet |T|/20 (1 + delta)
    b = RefBasis(2, 1)
    V = np.array([[0.3, -0.1], [1.7, 0.4], [0.2, 1.1]])
    pts, wts = map_rule(V[None], *ref_simplex_rule(2, 4))
    J = (V[1:] - V[0]).T
    xi = np.linalg.solve(J, (pts[0] - V[0]).T).T
    phi = b.values(xi)
    M = np.einsum("q,qk,qm->km", wts[0], phi, phi)
    area = 0.5 * abs(np.linalg.det(J))
    np.testing.assert_allclose(M, area / 12 * (np.ones((3, 3)) + np.eye(3)), rtol=1e-13)
    b3 = RefBasis(3, 1)
    V3 = np.array([[0, 0, 0], [1.0, 0.1, 0], [0.2, 1.3, 0.1], [0.1, 0.2, 0.9]])
    pts, wts = map_rule(V3[None], *ref_simplex_rule(3, 4))
    J3 = (V3[1:] - V3[0]).T
    xi = np.linalg.solve(J3, (pts[0] - V3[0]).T).T
    phi = b3.values(xi)
    M3 = np.einsum("q,qk,qm->km", wts[0], phi, phi)
    vol = abs(np.linalg.det(J3)) / 6
    np.testing.assert_allclose(M3, vol / 20 * (np.ones((4, 4)) + np.eye(4)), rtol=1e-13)


@pytest.mark.parametrize("pg", [0, 1, 2, 3])
def test_time_basis_orthogonal_and_by_parts(pg):
    tb = TimeBasis(pg)
    tm = tb.matrices()
    _, w = gauss_legendre01(pg + 1)
    # Gauss-Legendre nodal basis is orthogonal with the quadrature weights (Sec. 3)
    np.testing.assert_allclose(tm["W"], np.diag(w), atol=1e-14)
    # integration by parts on [0,1]: K + K^T = g(1)g(1)^T - g(0)g(0)^T
    K = tm["K"]
    np.testing.assert_allclose(K + K.T, np.outer(tm["g1"], tm["g1"]) - np.outer(tm["g0"], tm["g0"]), atol=1e-12)
    np.testing.assert_allclose(tb.values(tb.nodes), np.eye(pg + 1), atol=1e-13)
