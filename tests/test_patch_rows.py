"""CPU check of the patch construction that the full-size GPU test relies on: rows of the
oracle's operator computed on the patch {i and its face neighbours} equal the rows of the
fully assembled operator (2D sliver mesh at p = 3, 3D bounded mesh), and the face
neighbours agree with the oracle's connectivity."""
import numpy as np
import pytest

import synth
from helpers import face_neighbours, oracle_sim, patch_operator_rows


def _tet():
    xyz, ev, per = synth.tet_kuhn(2, 1.0, periodic=False, jitter=0.15, seed=9)
    n = ev.shape[0]
    rng = np.random.default_rng(1)
    return synth.Workload("tet", 3, xyz, ev, per, rng.uniform(1, 2, n), rng.uniform(.5, 1, n),
                          rng.uniform(.8, 1.2, n), p=2, p_gamma=1, scheme="stdg", dt=0.03, n_steps=1, h=0.5)


@pytest.mark.parametrize("make", [lambda: synth.scaled("c2", ny=8, steps=2), _tet], ids=["c2_slivers_p3", "tet_p2"])
def test_patch_rows_equal_the_assembled_rows(make):
    w = make()
    sim = oracle_sim(w)
    m = sim.mesh
    nb = face_neighbours(w.elem_vert)
    assert (nb >= 0).sum() == 2 * m.interior.sum()
    for j in np.where(m.interior)[0]:
        assert m.face_r[j] in nb[m.face_l[j]] and m.face_l[j] in nb[m.face_r[j]]
    x = np.random.default_rng(1).normal(size=sim.A.shape[0])
    y = (sim.A @ x).reshape(w.n_elem, -1)
    elems = np.arange(0, w.n_elem, 5)
    rows = patch_operator_rows(w, elems, x, nb)
    err = np.abs(rows - y[elems]).max(axis=1) / np.abs(y[elems]).max(axis=1)
    assert err.max() < 1e-11, err.max()
