"""Pins of the oracle's Appendix A preconditioners (Eqs. pre1, APPRE1, APPRE2).

Each pin follows from the definition alone, not from how the oracle forms an inverse:
  * (P_1 A x)_i = x_i when x lives on element i only;
  * (P_2 A x)_i = x_i when x lives on the stencil S_i only (A x restricted to S_i is A_i x);
  * on a mesh covered by one stencil, P_2's block row of that element is A^{-1}'s;
  * without off-diagonal blocks P_2 is P_1.
A dropped neighbour, a wrong block row of A_i^{-1} or a transposed block fails one of them.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle.precond import pre1, pre2, stencil
from oracle.stepper import Simulation


def _sim(dim, p, pg, scheme, periodic, seed=0):
    if dim == 2:
        xyz, ev, per = synth.tri_grid(4, 3, 1.0, 0.75, periodic=periodic, jitter=0.25, seed=seed)
    else:
        xyz, ev, per = synth.tet_kuhn(2, 1.0, periodic=periodic, jitter=0.15, seed=seed)
    rng = np.random.default_rng(seed + 1)
    ne = ev.shape[0]
    lam, mu, rho = rng.uniform(1.0, 3.0, ne), rng.uniform(0.5, 1.5, ne), rng.uniform(0.7, 1.4, ne)
    return Simulation(xyz, ev, per, lam, mu, rho, p, pg, scheme, 0.05)


CASES = [(2, 2, 2, "stdg", False), (2, 1, 0, "cn", True), (2, 3, 1, "stdg", True), (3, 1, 1, "stdg", False)]


@pytest.mark.parametrize("dim,p,pg,scheme,periodic", CASES)
def test_pre1_inverts_the_element_block(dim, p, pg, scheme, periodic):
    sim = _sim(dim, p, pg, scheme, periodic)
    A, ne = sim.A.tocsr(), sim.mesh.n_elem
    nb = A.shape[0] // ne
    P = pre1(A, ne)
    rng = np.random.default_rng(7)
    for e in rng.choice(ne, 4, replace=False):
        x = np.zeros(A.shape[0])
        x[e * nb:(e + 1) * nb] = rng.normal(size=nb)
        y = P @ (A @ x)
        assert np.abs(y[e * nb:(e + 1) * nb] - x[e * nb:(e + 1) * nb]).max() < 1e-9 * np.abs(x).max()


@pytest.mark.parametrize("dim,p,pg,scheme,periodic", CASES)
def test_pre2_inverts_on_the_stencil(dim, p, pg, scheme, periodic):
    sim = _sim(dim, p, pg, scheme, periodic)
    A, ne = sim.A.tocsr(), sim.mesh.n_elem
    nb = A.shape[0] // ne
    P = pre2(A, ne, sim.mesh.elem_nbr)
    rng = np.random.default_rng(8)
    for e in rng.choice(ne, 4, replace=False):
        st = stencil(e, sim.mesh.elem_nbr)
        assert len(st) >= 2
        x = np.zeros(A.shape[0])
        for g in st:
            x[g * nb:(g + 1) * nb] = rng.normal(size=nb)
        y = P @ (A @ x)
        assert np.abs(y[e * nb:(e + 1) * nb] - x[e * nb:(e + 1) * nb]).max() < 1e-9 * np.abs(x).max()
        # a vector on the stencil's complement does not reach element e through P_2
        x2 = rng.normal(size=A.shape[0])
        for g in st:
            x2[g * nb:(g + 1) * nb] = 0.0
        assert np.abs((P @ x2)[e * nb:(e + 1) * nb]).max() == 0.0


def test_pre2_is_the_exact_inverse_when_one_stencil_covers_the_mesh():
    # a triangle and its three face neighbours: the centre element's stencil is the mesh
    xyz = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 0.8], [0.5, -0.6], [1.2, 0.7], [-0.2, 0.7]])
    ev = np.array([[0, 1, 2], [0, 3, 1], [1, 4, 2], [2, 5, 0]], dtype=np.int32)
    sim = Simulation(xyz, ev, None, np.full(4, 2.0), np.full(4, 1.0), np.array([1.0, 1.3, 0.8, 1.1]), 2, 1, "stdg", 0.1)
    A, ne = sim.A.tocsr(), 4
    nb = A.shape[0] // ne
    assert sorted(stencil(0, sim.mesh.elem_nbr)) == [0, 1, 2, 3]
    P = pre2(A, ne, sim.mesh.elem_nbr).toarray()
    Ainv = np.linalg.inv(A.toarray())
    assert np.abs(P[:nb] - Ainv[:nb]).max() < 1e-10 * np.abs(Ainv).max()
    # the outer elements' stencils miss two elements each: their rows are not A^{-1}'s
    assert np.abs(P[nb:2 * nb] - Ainv[nb:2 * nb]).max() > 1e-6 * np.abs(Ainv).max()


def test_pre2_reduces_to_pre1_without_coupling():
    sim = _sim(2, 2, 1, "stdg", True)
    A, ne = sim.A.tocsr(), sim.mesh.n_elem
    nb = A.shape[0] // ne
    Abd = sp.block_diag([A[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb] for e in range(ne)], format="csr")
    P1 = pre1(Abd, ne).toarray()
    P2 = pre2(Abd, ne, sim.mesh.elem_nbr).toarray()
    assert np.abs(P1 - P2).max() < 1e-12 * np.abs(P1).max()


def _face_pairs(ev):
    """Element pairs sharing a face (sorted vertex tuples of the d-1 faces), as e1 * n + e2, e1 < e2."""
    ne, nv = ev.shape
    faces = np.concatenate([np.delete(ev, f, axis=1) for f in range(nv)])
    faces.sort(axis=1)
    owner = np.tile(np.arange(ne), nv)
    key = np.unique(faces, axis=0, return_inverse=True)[1].ravel()
    order = np.argsort(key, kind="stable")
    k, o = key[order], owner[order]
    same = k[1:] == k[:-1]
    a, b = o[:-1][same], o[1:][same]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    return lo, hi


@pytest.mark.parametrize("name", ["c1", "c2", "c3", "c4", "c5", "ragged"])
def test_face_neighbours_never_share_a_face(name):
    # The GPU forms Pre2's first block row by eliminating the neighbours one by one, which is
    # exact when no two face neighbours of an element are face neighbours of each other
    # (the local system is then an "arrow"); this holds for every workload mesh.
    w = {"c1": lambda: synth.c1_periodic_pwave(), "c2": lambda: synth.c2_layered_slivers(),
         "c3": lambda: synth.c3_cube_swave(n=16), "c4": lambda: synth.c4_multishot(n_shots=1),
         "c5": lambda: synth.c5_adjoint(), "ragged": lambda: synth.ragged_union(ks=range(0, 16, 5))[0]}[name]()
    ev = np.asarray(w.elem_vert, dtype=np.int64)
    ne = ev.shape[0]
    lo, hi = _face_pairs(ev)
    pairs = np.unique(lo * ne + hi)
    # neighbours of every element, padded with -1
    deg = np.bincount(np.concatenate([lo, hi]), minlength=ne)
    assert deg.max() <= ev.shape[1]
    tab = np.full((ne, ev.shape[1]), -1, dtype=np.int64)
    src = np.concatenate([lo, hi])
    dst = np.concatenate([hi, lo])
    order = np.argsort(src, kind="stable")
    src, dst = src[order], dst[order]
    start = np.searchsorted(src, np.arange(ne))
    slot = np.arange(len(src)) - start[src]
    tab[src, slot] = dst
    for p in range(ev.shape[1]):
        for q in range(p + 1, ev.shape[1]):
            a, b = tab[:, p], tab[:, q]
            ok = (a >= 0) & (b >= 0) & (a != b)
            key = np.minimum(a[ok], b[ok]) * ne + np.maximum(a[ok], b[ok])
            assert not np.isin(key, pairs).any(), name
