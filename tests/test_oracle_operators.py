"""Pins of the oracle's operator blocks and velocity system (Sec. 4, Sec. 5.1)."""
import numpy as np
import pytest

import synth
from oracle.mesh import DualMesh
from oracle.operators import Discretization, stiffness_tensor
from oracle.stepper import Simulation


def _mesh2d(n=4, periodic=True, jitter=0.25, seed=3):
    return synth.tri_grid(n, n, 1.0, 1.0, periodic=periodic, jitter=jitter, seed=seed)


def _mesh3d(n=3, periodic=True, jitter=0.15, seed=4):
    return synth.tet_kuhn(n, 1.0, periodic=periodic, jitter=jitter, seed=seed)


def _media(n, hetero, seed=0):
    if not hetero:
        return np.full(n, 2.0), np.full(n, 1.0), np.full(n, 1.0)
    rng = np.random.default_rng(seed)
    return rng.uniform(1.0, 3.0, n), rng.uniform(0.5, 1.5, n), rng.uniform(0.7, 1.4, n)


@pytest.mark.parametrize("dim,periodic,p", [(2, True, 1), (2, False, 3), (3, True, 2), (3, False, 1)])
def test_qtilde_is_minus_D_transpose(dim, periodic, p):
    # Proof of Theorem 1: Q~_{i,j} = -D_{i,j}^T, computed here from independent integrals
    xyz, ev, per = _mesh2d(periodic=periodic) if dim == 2 else _mesh3d(periodic=periodic)
    lam, mu, rho = _media(ev.shape[0], False)
    dz = Discretization(DualMesh(xyz, ev, per), p, 0, lam, mu, rho)
    scale = np.abs(dz.D).max()
    assert np.abs(dz.Qt + np.swapaxes(dz.D, -1, -2)).max() < 1e-13 * scale


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 3), (3, 2)])
def test_constant_stress_gives_no_momentum_forcing(dim, p):
    # sum_{j in S_i} D_{i,j} . sigma = int_{dT_i} phi sigma.n - int_{T_i} grad phi . sigma = 0
    xyz, ev, per = _mesh2d(periodic=True) if dim == 2 else _mesh3d(periodic=True)
    lam, mu, rho = _media(ev.shape[0], False)
    dz = Discretization(DualMesh(xyz, ev, per), p, 0, lam, mu, rho)
    dz.spacetime(1.0)
    rng = np.random.default_rng(1)
    S = rng.normal(size=(dim, dim))
    S = S + S.T
    sig = np.zeros((dz.mesh.n_face, dim, dim, dz.Npsi))
    sig[..., 0] = S                         # psi_0 = 1: a constant stress in every dual cell
    out = dz.D_dot_sigma(sig)
    assert np.abs(out).max() < 1e-13 * np.abs(dz.D).max()


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_linear_velocity_patch(dim, p):
    # a globally linear (continuous) velocity has no jumps, so on every interior dual cell
    # M_j^{-1} E_j . Q v = dt E : grad v exactly (constant, only psi_0 nonzero)
    xyz, ev, per = _mesh2d(n=4, periodic=False) if dim == 2 else _mesh3d(n=2, periodic=False)
    lam, mu, rho = _media(ev.shape[0], False)
    sim = Simulation(xyz, ev, per, lam, mu, rho, p, 0, "cn", 0.1)
    dz = sim.disc
    G = np.arange(1, dim * dim + 1, dtype=float).reshape(dim, dim) / 7.0   # v_k = sum_l G[k,l] x_l
    nodes = np.einsum("ekd,nk->end", sim.mesh.X[:, 1:] - sim.mesh.X[:, :1], dz.ref.nodes) + sim.mesh.X[:, :1]
    v = np.einsum("kl,enl->ekn", G, nodes)
    eq = dz.E_dot_Q_v(v)
    inc = np.einsum("fyz,fabz->faby", dz.Mst_inv, eq)
    E = stiffness_tensor(2.0, 1.0, dim)
    want = 0.1 * np.einsum("abkl,kl->ab", E, G)
    inter = sim.mesh.interior
    tol = 1e-10 * np.abs(want).max()      # monomial dual mass matrices cost a few digits
    np.testing.assert_allclose(inc[inter][..., 0], np.broadcast_to(want, inc[inter][..., 0].shape), atol=tol)
    assert np.abs(inc[inter][..., 1:]).max() < tol


@pytest.mark.parametrize("dim,p,hetero,periodic", [
    (2, 1, False, True), (2, 2, True, True), (2, 3, True, False), (3, 1, False, True), (3, 2, True, False)])
def test_crank_nicolson_matrix_symmetric_positive_definite(dim, p, hetero, periodic):
    # Theorems 1 and 2 (and, with E_j constant per dual cell, the heterogeneous case)
    xyz, ev, per = _mesh2d(n=3, periodic=periodic) if dim == 2 else _mesh3d(n=3 if periodic else 2, periodic=periodic)
    lam, mu, rho = _media(ev.shape[0], hetero)
    A = Simulation(xyz, ev, per, lam, mu, rho, p, 0, "cn", 0.3).A.toarray()
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    ev_min = np.linalg.eigvalsh(0.5 * (A + A.T)).min()
    assert ev_min > 0


def test_space_time_matrix_not_symmetric():
    xyz, ev, per = _mesh2d(n=3)
    lam, mu, rho = _media(ev.shape[0], False)
    A = Simulation(xyz, ev, per, lam, mu, rho, 1, 1, "stdg", 0.2).A.toarray()
    assert np.abs(A - A.T).max() > 1e-3 * np.abs(A).max()


def test_renumbering_invariance():
    xyz, ev, per = _mesh2d(n=4, periodic=True)
    lam, mu, rho = _media(ev.shape[0], True)
    A = Simulation(xyz, ev, per, lam, mu, rho, 2, 1, "stdg", 0.1).A.toarray()
    perm = np.random.default_rng(5).permutation(ev.shape[0])
    Ap = Simulation(xyz, ev[perm], per, lam[perm], mu[perm], rho[perm], 2, 1, "stdg", 0.1).A.toarray()
    nb = A.shape[0] // ev.shape[0]
    idx = (perm[:, None] * nb + np.arange(nb)).ravel()
    np.testing.assert_allclose(Ap, A[np.ix_(idx, idx)], atol=1e-14 * np.abs(A).max())


def test_point_location_reading():
    # reading: the element whose barycentric coordinates are all >= -1e-12, the lowest index on
    # ties (edges, vertices); periodic images fold back into the element's frame
    xyz, ev, per = _mesh2d(n=4, periodic=True)
    m = DualMesh(xyz, ev, per)
    for i in range(m.n_elem):
        c = m.X[i].mean(axis=0)
        j, y = m.locate(c)
        assert j == i and np.allclose(y, c)
        j, y = m.locate(c + per * np.array([1.0, -2.0]))            # a periodic image
        assert j == i and np.allclose(y, c, atol=1e-12)
    for f in range(m.n_face):
        mid = m.face_X[f].mean(axis=0)
        j, _ = m.locate(mid)
        assert j == min(m.face_l[f], m.face_r[f])
    vert = m.X[5, 1]
    touching = [i for i in range(m.n_elem) if np.any(np.all(np.abs(
        (m.X[i] - vert + per / 2) % per - per / 2) < 1e-12, axis=1))]
    assert m.locate(vert)[0] == min(touching)
    xyz_b, ev_b, _ = _mesh2d(n=3, periodic=False)
    with pytest.raises(ValueError):
        DualMesh(xyz_b, ev_b, None).locate(np.array([1.5, 0.5]))
