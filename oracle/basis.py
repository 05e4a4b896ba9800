"""Bases of the scheme (Sec. 3, paragraph "Space-time basis functions").

* Main grid: nodal Lagrange basis of degree p on the reference simplex
  (N_phi = C(p+d, d)), nodes equispaced and ordered z-outer, then y, x fastest;
  built by inverting the monomial Vandermonde matrix.
* Dual grid: rescaled Taylor monomials ((x - x_j)/h_j)^a, |a| <= p, in physical
  space (the paper's 3D choice, used here in 2D as well), graded-lexicographic
  order (total degree ascending; within a degree, exponent of x descending, then
  of y descending).
* Time: Lagrange polynomials through the p_gamma+1 Gauss-Legendre points of [0,1].

Pins: partition of unity and nodality, the closed-form P1 mass matrix, exactness
of Gauss-Legendre orthogonality int gamma_k gamma_m = w_k delta_km
(tests/test_oracle_basis.py).
"""
import itertools

import numpy as np


def monomial_exponents(dim, p):
    """Graded-lex exponent list of all monomials of total degree <= p."""
    out = []
    for g in range(p + 1):
        exps = [e for e in itertools.product(range(g + 1), repeat=dim) if sum(e) == g]
        exps.sort(reverse=True)
        out.extend(exps)
    return np.array(out, dtype=np.int64)


def ref_nodes(dim, p):
    """Equispaced nodes of the reference simplex, z outer, y, x fastest."""
    pts = []
    if dim == 2:
        for j in range(p + 1):
            for i in range(p + 1 - j):
                pts.append((i / p, j / p))
    else:
        for k in range(p + 1):
            for j in range(p + 1 - k):
                for i in range(p + 1 - j - k):
                    pts.append((i / p, j / p, k / p))
    return np.array(pts, dtype=np.float64)


def monomials(x, exps):
    """x: (..., dim) -> (..., n_mono) values of x^a."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones(x.shape[:-1] + (exps.shape[0],))
    for a in range(exps.shape[1]):
        out = out * x[..., a:a + 1] ** exps[:, a]
    return out


def monomial_grads(x, exps):
    """(..., n_mono, dim) derivatives d/dx_r of x^a."""
    x = np.asarray(x, dtype=np.float64)
    g = np.zeros(x.shape[:-1] + (exps.shape[0], exps.shape[1]))
    for r in range(exps.shape[1]):
        term = np.ones(x.shape[:-1] + (exps.shape[0],))
        for a in range(exps.shape[1]):
            if a == r:
                e = exps[:, a]
                term = term * e * x[..., a:a + 1] ** np.maximum(e - 1, 0)
            else:
                term = term * x[..., a:a + 1] ** exps[:, a]
        g[..., r] = term
    return g


class RefBasis:
    """Nodal P_p basis on the reference simplex."""

    def __init__(self, dim, p):
        self.dim, self.p = dim, p
        self.exps = monomial_exponents(dim, p)
        self.nodes = ref_nodes(dim, p)
        V = monomials(self.nodes, self.exps)          # V[n, a] = xi_n^a
        self.coef = np.linalg.inv(V)                   # phi_k = sum_a coef[a, k] xi^a
        self.n = self.nodes.shape[0]

    def values(self, xi):
        return monomials(xi, self.exps) @ self.coef

    def grads(self, xi):
        """(..., N, dim) reference-coordinate gradients."""
        g = monomial_grads(xi, self.exps)            # (..., a, r)
        return np.einsum("...ar,ak->...kr", g, self.coef)


def gauss_legendre01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


class TimeBasis:
    """Lagrange basis through the p_gamma+1 Gauss-Legendre points of [0,1]."""

    def __init__(self, p_gamma):
        self.n = p_gamma + 1
        self.nodes, _ = gauss_legendre01(self.n)

    def values(self, tau):
        tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
        out = np.ones((tau.size, self.n))
        for k in range(self.n):
            for m in range(self.n):
                if m != k:
                    out[:, k] *= (tau - self.nodes[m]) / (self.nodes[k] - self.nodes[m])
        return out

    def derivs(self, tau):
        tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
        out = np.zeros((tau.size, self.n))
        for k in range(self.n):
            for q in range(self.n):
                if q == k:
                    continue
                term = np.full(tau.size, 1.0 / (self.nodes[k] - self.nodes[q]))
                for m in range(self.n):
                    if m != k and m != q:
                        term *= (tau - self.nodes[m]) / (self.nodes[k] - self.nodes[m])
                out[:, k] += term
        return out

    def matrices(self):
        """Reference-interval matrices of Eqs. MD_2 - MD_2_3 (time factors).

        W[k,m]  = int_0^1 gamma_k gamma_m dtau
        K[k,m]  = int_0^1 gamma_k' gamma_m dtau      (the M^circ time factor)
        g0, g1  = gamma(0), gamma(1)
        T       = g1 g1^T - K                        (time factor of M = M^+ - M^circ)
        """
        xq, wq = gauss_legendre01(self.n + 2)
        G, dG = self.values(xq), self.derivs(xq)
        W = np.einsum("q,qk,qm->km", wq, G, G)
        K = np.einsum("q,qk,qm->km", wq, dG, G)
        g0, g1 = self.values(0.0)[0], self.values(1.0)[0]
        T = np.outer(g1, g1) - K
        return dict(W=W, K=K, g0=g0, g1=g1, T=T)
