"""The sliver study of Sec. 6.5 (printed values in tests/golden/sliver_iterations.txt) on
the oracle's assembled systems -- slow (minutes of GMRES in Python), so it runs only with
STDG_SLOW_TESTS=1.

The paper's setup: (p, p_gamma) = (4, 2), dt = 0.014, a plane P wave along (1, 0) on an
almost uniform mesh of [-1.5, 1.5]^2 (mesh 1) and the same mesh with two slivers whose
incircle radius is 70.53 times smaller (mesh 2).  Ours: a jittered 12 x 12 x 2 mesh (its
vertices on the boundary fixed), two slivers made by moving the vertex opposite the
longest edge towards it.  Right-preconditioned GMRES(30) to 1e-8 from a zero guess on the
first three slabs' systems, with none, the block-Jacobi Pre1 and the stencil Pre2 of
Appendix A (oracle/precond.py).  Checked against the table: on both meshes none > Pre1 >
Pre2, and the sliver factor (mesh 2 / mesh 1) falls from none to Pre1 to Pre2.  Not
reproduced: the table's factor 1.00 for Pre2 (ours about 3, with Pre2 built as printed;
our sliver construction also deforms the sliver's neighbours, which the stencil contains
only in part).
"""
import functools

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle.precond import pre1, pre2
from oracle.stepper import Simulation
from synth.meshes import add_slivers
from test_golden_tables import load_sliver

pytestmark = pytest.mark.slow

CAP = 6000                 # iterations; the unpreconditioned sliver case reaches it (a lower bound)


def _mesh(n, slivers, seed=3):
    xyz, ev, _ = synth.tri_grid(n, n, 3.0, 3.0, periodic=False, jitter=0.2, seed=seed)
    xyz = xyz - 1.5
    on_boundary = (np.abs(np.abs(xyz[:, 0]) - 1.5) < 1e-12) | (np.abs(np.abs(xyz[:, 1]) - 1.5) < 1e-12)
    if slivers:
        xyz, chosen = add_slivers(xyz, ev, 3.0 / n, 2.0 / ev.shape[0], ratio=70.53, seed=seed,
                                  fixed_vertex=on_boundary)
        assert len(chosen) == 2
    return xyz, ev


@functools.lru_cache(maxsize=None)
def mean_iterations(slivers, pre, n=12, steps=3):
    xyz, ev = _mesh(n, slivers)
    ne = ev.shape[0]
    lam, mu, rho = synth.homogeneous(ne, 2.0, 1.0, 1.0)
    sim = Simulation(xyz, ev, None, lam, mu, rho, 4, 2, "stdg", 0.014)
    sim.set_plane_wave(0, np.array([1.0, 0.0]), None, 1e-2)
    A = sim.A.tocsr()
    P = {0: None, 1: lambda: pre1(A, ne), 2: lambda: pre2(A, ne, sim.mesh.elem_nbr)}[pre]
    P = P() if P else None
    op = A if P is None else spla.LinearOperator(A.shape, matvec=lambda y: A @ (P @ y))
    counts = []
    for _ in range(steps):
        b = sim.rhs()
        k = [0]

        def count(_r):
            k[0] += 1
        spla.gmres(op, b, rtol=1e-8, restart=30, maxiter=CAP // 30, callback=count, callback_type="pr_norm")
        counts.append(k[0])
        sim.step(1)
    return float(np.mean(counts))


def test_sliver_table_trends():
    paper = load_sliver()
    ours = {name: (mean_iterations(False, pre), mean_iterations(True, pre))
            for name, pre in (("none", 0), ("pre1", 1), ("pre2", 2))}
    print("ours", ours, "paper", paper)
    for k in (0, 1):
        assert ours["none"][k] > ours["pre1"][k] > ours["pre2"][k]
        assert paper["none"][k] > paper["pre1"][k] > paper["pre2"][k]
    factor = {name: v[1] / v[0] for name, v in ours.items()}
    assert factor["none"] > factor["pre1"] > factor["pre2"]
