"""Per-element isotropic media (lambda, mu, rho) for the synthetic workloads."""
import numpy as np

from .meshes import unwrap_elements


def lame_from_speeds(vp, vs, rho):
    vp, vs, rho = (np.asarray(a, dtype=np.float64) for a in (vp, vs, rho))
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return lam, mu, rho


def homogeneous(n_elem, lam, mu, rho):
    return (np.full(n_elem, float(lam)), np.full(n_elem, float(mu)), np.full(n_elem, float(rho)))


def centroids(xyz, elem, period):
    return unwrap_elements(xyz, elem, period).mean(axis=1)


def layered_2d(xyz, elem, period, bounds, vp, vs, rho):
    """Horizontal layers assigned by element centroid height.

    bounds: ascending interface heights [y_1, y_2, ...]; layer k spans
    [bounds[k-1], bounds[k]) counted from the bottom.  vp, vs, rho are listed
    bottom layer first.
    """
    y = centroids(xyz, elem, period)[:, 1]
    layer = np.searchsorted(np.asarray(bounds), y, side="right")
    lam, mu, r = lame_from_speeds(np.asarray(vp)[layer], np.asarray(vs)[layer], np.asarray(rho)[layer])
    return lam, mu, r


def gaussian_random_field(points, corr_len, n_modes=256, seed=0):
    """Smooth seeded field: a sum of random Fourier modes with a Gaussian spectrum.

    Wave vectors are drawn from N(0, 1/corr_len^2) per axis, phases uniformly; the
    field is normalised to max |g| = 1 over ``points``.
    """
    rng = np.random.default_rng(seed)
    dim = points.shape[1]
    k = rng.normal(0.0, 1.0 / corr_len, size=(n_modes, dim))
    ph = rng.uniform(0.0, 2 * np.pi, size=n_modes)
    amp = rng.normal(size=n_modes)
    g = np.cos(points @ k.T + ph) @ amp
    return g / np.abs(g).max()
