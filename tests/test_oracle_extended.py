"""Pins of the extended-precision operator rows (oracle/extended.py).

The module restates the oracle's A in np.longdouble so that the sliver meshes, where the
FP64 oracle's Taylor-monomial dual mass matrices (cond ~5e8) cost it ~1e-10 of accuracy,
still have a reference well below the 1e-10 bar.  Pinned here against the mathematics, not
against the module itself: Q~ = -D^T (Theorem 1 proof) to extended rounding, symmetry and
positive definiteness of the Crank-Nicolson matrix (Theorems 1, 2), agreement with the
FP64 oracle where the FP64 oracle is well conditioned, and two exact quadrature orders
agreeing far below the FP64 oracle's own spread on sliver rows.
"""
import numpy as np
import pytest

import synth
from oracle.extended import LD, PatchOperator, eps
from oracle.operators import Discretization
from oracle.stepper import Simulation


def _rel(a, b):
    a = np.asarray(a, dtype=LD).ravel()
    b = np.asarray(b, dtype=LD).ravel()
    return float(np.sqrt(np.sum((a - b) ** 2)) / np.sqrt(np.sum(b * b)))


def _media(n, seed=1):
    rng = np.random.default_rng(seed)
    return rng.uniform(1, 2, n), rng.uniform(.5, 1, n), rng.uniform(.8, 1.2, n)


@pytest.mark.parametrize("dim,p,pg,scheme", [(2, 1, 0, "cn"), (2, 2, 2, "stdg"), (2, 3, 1, "stdg"),
                                             (3, 1, 1, "stdg"), (3, 2, 0, "cn")])
def test_extended_rows_match_fp64_oracle_on_well_conditioned_meshes(dim, p, pg, scheme):
    if dim == 2:
        xyz, ev, _ = synth.tri_grid(4, 3, 2.0, 1.0, periodic=False, jitter=0.2, seed=3)
    else:
        xyz, ev, _ = synth.tet_kuhn(2, 1.0, periodic=False, jitter=0.15, seed=9)
    lam, mu, rho = _media(ev.shape[0])
    sim = Simulation(xyz, ev, None, lam, mu, rho, p, pg, scheme, 0.03)
    x = np.random.default_rng(2).normal(size=sim.A.shape[0])
    y = (sim.A @ x).reshape(ev.shape[0], -1)
    P = PatchOperator(xyz, ev, lam, mu, rho, p, pg, scheme, 0.03)
    elems = list(range(0, ev.shape[0], max(1, ev.shape[0] // 12)))
    ye = P.rows(elems, x).reshape(len(elems), -1)
    assert _rel(ye, y[elems]) < 2e-13


def test_extended_qtilde_is_minus_D_transpose_on_sliver_faces():
    # Q~ and D from independent integrals: Q~ = -D^T to the rounding of the extended format,
    # on the dual cells next to sliver elements
    w = synth.scaled("c2", ny=8, steps=1)
    P = PatchOperator(w.xyz, w.elem_vert, w.lam, w.mu, w.rho, w.p, w.p_gamma, w.scheme, w.dt)
    worst = 0.0
    for i in list(w.extra["slivers"][:6]):
        for f in range(3):
            sides, M, _ = P.face_blocks(int(i), f)
            for (_, D, Q) in sides:
                scale = np.abs(D).max()
                worst = max(worst, float(np.abs(Q + np.swapaxes(D, -1, -2)).max() / scale))
    assert worst < 1e3 * eps(), worst


def test_extended_rows_resolve_the_sliver_rounding():
    # rows of sliver elements (p = 3, Taylor dual basis): the FP64 oracle moves by ~1e-10
    # between two exact quadrature orders; the extended rows do not (they agree far below
    # the FP64 spread) and stay within that spread of the FP64 oracle
    w = synth.scaled("c2", ny=8, steps=1)
    sim = Simulation.from_workload(w)
    d2 = Discretization(sim.mesh, w.p, w.p_gamma, w.lam, w.mu, w.rho, quad_n=w.p + 5)
    x = np.random.default_rng(7).normal(size=sim.A.shape[0])
    n = w.n_elem
    y1 = (sim.A @ x).reshape(n, -1)
    y2 = (d2.assemble(w.dt, w.scheme) @ x).reshape(n, -1)
    sl = [int(i) for i in w.extra["slivers"][:8]]
    e1 = PatchOperator(w.xyz, w.elem_vert, w.lam, w.mu, w.rho, w.p, w.p_gamma, w.scheme, w.dt).rows(sl, x)
    e2 = PatchOperator(w.xyz, w.elem_vert, w.lam, w.mu, w.rho, w.p, w.p_gamma, w.scheme, w.dt,
                       quad_n=w.p + 5).rows(sl, x)
    spread64 = _rel(y1[sl], y2[sl])
    spread_ext = _rel(e1.reshape(len(sl), -1), e2.reshape(len(sl), -1))
    assert spread64 > 1e-12                     # the FP64 limit this module exists for
    # the gain follows the format: x87 80-bit (x86-64) gains ~2^11 over FP64, binary128 (aarch64) ~2^60
    gain = eps() / np.finfo(np.float64).eps
    assert spread_ext < 1e-12 and spread_ext < 100 * gain * spread64, (spread_ext, spread64)
    assert _rel(y1[sl], e1.reshape(len(sl), -1)) < 50 * spread64


@pytest.mark.parametrize("p,hetero", [(1, False), (2, True)])
def test_extended_crank_nicolson_matrix_symmetric_positive_definite(p, hetero):
    # Theorems 1 and 2: the Crank-Nicolson velocity matrix, assembled column by column from
    # the extended rows, is symmetric to extended rounding and positive definite
    xyz, ev, _ = synth.tri_grid(3, 3, 1.0, 1.0, periodic=False, jitter=0.25, seed=5)
    n = ev.shape[0]
    lam, mu, rho = _media(n) if hetero else (np.full(n, 2.0), np.full(n, 1.0), np.full(n, 1.0))
    P = PatchOperator(xyz, ev, lam, mu, rho, p, 0, "cn", 0.3)
    nb = 2 * P.b.N
    nbrs = {i: {i} for i in range(n)}
    for (i, f), ent in P.face_of.items():
        for (e, _) in ent:
            nbrs[i].add(e)
    A = np.zeros((n * nb, n * nb), dtype=LD)
    for e in range(n):
        for c in range(nb):
            x = np.zeros(n * nb)
            x[e * nb + c] = 1.0
            for i in sorted(nbrs[e]):
                A[i * nb:(i + 1) * nb, e * nb + c] = P.row(i, x).ravel()
    scale = np.abs(A).max()
    assert float(np.abs(A - A.T).max() / scale) < 1e3 * eps()
    assert np.linalg.eigvalsh(A.astype(np.float64)).min() > 0
