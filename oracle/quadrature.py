"""Collapsed-coordinate (Duffy) Gauss-Legendre rules on simplices.

The paper does not state its quadrature.  All integrands of the scheme on affine
sub-cells are polynomials of degree <= 2p, so any rule exact to that degree gives
the same operator; this one uses n points per collapsed direction, exact for total
degree <= 2n - 1 - (dim - 1).  Pins: exactness on monomials against the closed form
int_T xi^a = a! / (|a| + dim)! (tests/test_oracle_basis.py).
"""
import numpy as np

from .basis import gauss_legendre01


def ref_simplex_rule(dim, n):
    """Points (Q, dim) and weights (Q,) on the unit reference simplex (weights sum 1/dim!)."""
    x, w = gauss_legendre01(n)
    if dim == 1:
        return x[:, None], w
    if dim == 2:
        u, v = np.meshgrid(x, x, indexing="ij")
        wu, wv = np.meshgrid(w, w, indexing="ij")
        xi = u
        eta = v * (1.0 - u)
        pts = np.stack([xi.ravel(), eta.ravel()], axis=1)
        wts = (wu * wv * (1.0 - u)).ravel()
        return pts, wts
    if dim == 3:
        u, v, s = np.meshgrid(x, x, x, indexing="ij")
        wu, wv, ws = np.meshgrid(w, w, w, indexing="ij")
        xi = u
        eta = v * (1.0 - u)
        zeta = s * (1.0 - u) * (1.0 - v)
        pts = np.stack([xi.ravel(), eta.ravel(), zeta.ravel()], axis=1)
        wts = (wu * wv * ws * (1.0 - u) ** 2 * (1.0 - v)).ravel()
        return pts, wts
    raise ValueError(dim)


def simplex_measure(V):
    """Measure of the k-simplex with vertices V[..., k+1, D] embedded in R^D."""
    E = V[..., 1:, :] - V[..., :1, :]
    k = E.shape[-2]
    G = np.einsum("...ad,...bd->...ab", E, E)
    fact = 1.0
    for t in range(2, k + 1):
        fact *= t
    return np.sqrt(np.abs(np.linalg.det(G))) / fact


def map_rule(V, ref_pts, ref_wts):
    """Map a reference rule onto simplices V[..., k+1, D].

    Returns physical points (..., Q, D) and weights (..., Q) summing to the measure.
    """
    k = V.shape[-2] - 1
    E = V[..., 1:, :] - V[..., :1, :]                        # (..., k, D)
    pts = V[..., None, 0, :] + np.einsum("qk,...kd->...qd", ref_pts, E)
    fact = 1.0
    for t in range(2, k + 1):
        fact *= t
    wts = ref_wts * fact * simplex_measure(V)[..., None]
    return pts, wts
