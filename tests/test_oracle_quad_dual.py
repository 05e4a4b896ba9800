"""Pins of the oracle's second 2D dual basis, the paper's own (Sec. 3, space-time basis
functions): the (p+1)^2 tensor-product space on the unit square carried to each dual
quadrilateral (b_l, n_0, b_r, n_1) by its bilinear map (oracle/operators.py, dual="quad").

* the bilinear inverse undoes the forward map (corners and random interior points);
* Q~ = -D^T, a constant stress exerts no force, and the Crank-Nicolson matrix is
  symmetric positive definite with exact energy conservation (Theorems 1, 2, 5) on a
  jittered periodic mesh, where the quadrilaterals are not parallelograms and the basis
  is rational in x;
* on parallelogram cells (an unjittered grid) the tensor space contains the Taylor space
  P_p, so its L2 projection of a smooth stress field is at least as close;
* the plane wave converges at order p + 1 (p = p_gamma = 1, 2), as in Table 1.
A scrambled vertex order, a wrong map or a missing mode fails one of them.
"""
import numpy as np
import pytest

import synth
from oracle.mesh import DualMesh
from oracle.operators import Discretization, bilinear_inverse
from oracle.stepper import Simulation


def _mesh(n=4, jitter=0.25, seed=3):
    return synth.tri_grid(n, n, 1.0, 1.0, periodic=True, jitter=jitter, seed=seed)


def _disc(p, jitter=0.25, n=4, pg=0):
    xyz, ev, per = _mesh(n=n, jitter=jitter)
    ne = ev.shape[0]
    return Discretization(DualMesh(xyz, ev, per), p, pg, np.full(ne, 2.0), np.full(ne, 1.0), np.full(ne, 1.0),
                          dual="quad")


def test_bilinear_inverse_undoes_the_map():
    rng = np.random.default_rng(0)
    P = np.array([[0.0, 0.0], [1.2, 0.1], [1.0, 0.9], [-0.1, 1.1]])[None]
    uv = rng.uniform(0, 1, size=(1, 50, 2))
    u, v = uv[..., 0:1], uv[..., 1:2]
    x = (1 - u) * (1 - v) * P[:, None, 0] + u * (1 - v) * P[:, None, 1] + u * v * P[:, None, 2] + (1 - u) * v * P[:, None, 3]
    np.testing.assert_allclose(bilinear_inverse(P, x), uv, atol=1e-13)
    corners = bilinear_inverse(P, P)
    np.testing.assert_allclose(corners[0], [[0, 0], [1, 0], [1, 1], [0, 1]], atol=1e-13)
    dz = _disc(1)
    np.testing.assert_allclose(bilinear_inverse(dz.quad, dz.quad)[:, [0, 2]],
                               np.broadcast_to([[0, 0], [1, 1]], (dz.mesh.n_face, 2, 2)), atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_structure_theorems_with_the_tensor_dual_basis(p):
    dz = _disc(p)
    assert dz.Npsi == (p + 1) ** 2
    scale = np.abs(dz.D).max()
    assert np.abs(dz.Qt + np.swapaxes(dz.D, -1, -2)).max() < 1e-13 * scale
    assert np.linalg.eigvalsh(dz.Mdual).min() > 0
    dz.spacetime(1.0)
    S = np.array([[1.0, 0.3], [0.3, -0.7]])
    sig = np.zeros((dz.mesh.n_face, 2, 2, dz.Npsi))
    sig[..., 0] = S                                       # psi_0 = u^0 v^0 = 1
    assert np.abs(dz.D_dot_sigma(sig)).max() < 1e-13 * scale


@pytest.mark.parametrize("p", [1, 2])
def test_crank_nicolson_spd_and_energy_with_the_tensor_dual_basis(p):
    xyz, ev, per = _mesh(n=3)
    ne = ev.shape[0]
    rng = np.random.default_rng(2)
    lam, mu, rho = rng.uniform(1, 3, ne), rng.uniform(0.5, 1.5, ne), rng.uniform(0.7, 1.4, ne)
    sim = Simulation(xyz, ev, per, lam, mu, rho, p, 0, "cn", 0.3, dual="quad")
    A = sim.A.toarray()
    # u^a v^b on [0, 1]^2 gives worse-conditioned dual mass matrices than centred Taylor
    # monomials: the explicit inverse leaves rounding a little above 1e-13
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    sim.set_state(rng.normal(size=sim.v_tr.shape), rng.normal(size=sim.sig_tr.shape))
    e0 = sim.energy()
    sim.step(5)
    assert abs(sim.energy() - e0) <= 1e-12 * e0


@pytest.mark.parametrize("p", [1, 2])
def test_tensor_space_contains_taylor_space_on_parallelograms(p):
    xyz, ev, per = synth.tri_grid(4, 4, 1.0, 1.0, periodic=True)
    ne = ev.shape[0]
    args = (xyz, ev, per, np.full(ne, 2.0), np.full(ne, 1.0), np.full(ne, 1.0), p, 0, "cn", 0.1)
    errs = {}
    for dual in ("taylor", "quad"):
        sim = Simulation(*args, dual=dual)
        sim.set_plane_wave(0, np.array([1.0, 1.0]), None, 1.0)
        sig = sim.disc.full_from_sym(sim.sig_tr)
        # ||s - Pi s||^2 = ||s||^2 - ||Pi s||^2 with the same ||s||^2 for both spaces
        errs[dual] = -np.einsum("fabk,fkm,fabm->", sig, sim.disc.Mdual, sig)
    assert errs["quad"] <= errs["taylor"] + 1e-12 * abs(errs["taylor"])
    assert errs["quad"] < errs["taylor"] - 1e-6 * abs(errs["taylor"])    # strictly larger space


def _plane_wave_error(n, p):
    xyz, ev, per = synth.tri_grid(n, n, 1.0, 1.0, periodic=True, jitter=0.15, seed=n)
    ne = ev.shape[0]
    cp = 2.0
    steps = max(2, int(round(0.5 / cp / (0.25 / n / cp))))
    dt = 0.5 / cp / steps
    sim = Simulation(xyz, ev, per, np.full(ne, 2.0), np.full(ne, 1.0), np.full(ne, 1.0), p, p, "stdg", dt, dual="quad")
    sim.set_plane_wave(0, np.array([1.0, 0.0]), None, 1e-2)
    v0 = sim.v_tr.copy()
    sim.step(steps)
    sim2 = Simulation(xyz, ev, per, np.full(ne, 2.0), np.full(ne, 1.0), np.full(ne, 1.0), p, p, "stdg", dt, dual="quad")
    sim2.set_plane_wave(0, np.array([1.0, 0.0]), None, 1e-2, t=steps * dt)
    return np.linalg.norm(sim.v_tr - sim2.v_tr) / np.linalg.norm(v0)


@pytest.mark.parametrize("p", [1, 2])
def test_plane_wave_order_with_the_tensor_dual_basis(p):
    e1, e2 = _plane_wave_error(6, p), _plane_wave_error(12, p)
    assert np.log2(e1 / e2) > p + 1 - 0.35, (e1, e2)


@pytest.mark.parametrize("p,pg", [(1, 1), (2, 2), (2, 1)])
def test_space_time_energy_identity_with_the_tensor_dual_basis(p, pg):
    # Theorem 4 (eq. stsum4) with the paper's 2D dual space: the energy lost over a slab
    # equals the time-jump terms, which are non-negative
    xyz, ev, per = _mesh(n=4, jitter=0.2, seed=8)
    n = ev.shape[0]
    rng = np.random.default_rng(4)
    sim = Simulation(xyz, ev, per, rng.uniform(1, 3, n), rng.uniform(.5, 1.5, n), rng.uniform(.7, 1.4, n),
                     p, pg, "stdg", 0.21, dual="quad")
    sim.set_state(rng.normal(size=sim.v_tr.shape), rng.normal(size=sim.sig_tr.shape))
    e = [sim.energy()]
    jumps = []
    for _ in range(3):
        sim.step(1)
        e.append(sim.energy())
        jumps.append(sim.jump_dissipation())
    e, jumps = np.array(e), np.array(jumps)
    assert (jumps >= 0).all() and (np.diff(e) <= 1e-14 * e[0]).all()
    np.testing.assert_allclose(e[:-1] - e[1:], jumps, rtol=1e-9, atol=1e-13 * e[0])
