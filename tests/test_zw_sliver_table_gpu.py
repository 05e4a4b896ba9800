"""The sliver-element study of Sec. 6.5 (Table NT5.1) on the GPU, on meshes of our own: GMRES
iterations per slab without preconditioner, with the block-Jacobi Pre1 and with the
stencil Pre2, (p, p_gamma) = (4, 2) as in the paper, on a jittered layered mesh without
and with 1% sliver elements (incircle reduced ~70x), the same plane P wave and slab size
on both.  Checked here: slivers multiply the unpreconditioned and the Pre1 counts most, and
Pre2 is the least sensitive and the cheapest.  The paper's table reports a Pre2 factor of
1.00 (mesh-independent); on these meshes, with many more slivers than the paper's two,
Pre2's factor stays above 1 (about 2), and the test does not claim mesh independence."""
import numpy as np
import pytest

import synth
from synth.workloads import _layered_mesh, explicit_cfl_dt
from helpers import need_gpu

pytestmark = pytest.mark.gpu


def _iterations(slivers, pre, ny=24, steps=3):
    from paper_1802_04516_gb300.binding import Solver, StdgError
    xyz, ev, per, lam, mu, rho, h, _ = _layered_mesh(2 * ny, ny, seed=77, slivers=slivers)
    lam, mu, rho = synth.homogeneous(ev.shape[0], 2.0, 1.0, 1.0)
    dt = 10.0 * explicit_cfl_dt(h, 2, 4, 2.0)
    s = Solver(2, 4, 2, "stdg", "fp64", rel_tol=1e-8, max_iters=4000, gmres_restart=30, preconditioner=pre)
    s.set_mesh(xyz, ev, per)
    s.set_material(lam, mu, rho)
    s.set_shots(1)
    s.set_plane_wave(0, [1.0, 0.0], amp=1e-2)
    its = []
    for _ in range(steps):
        try:
            its.append(s.step(dt, 1)["iters_max"])
        except StdgError:
            its.append(4000)
    s.close()
    return float(np.mean(its))


def test_pre2_least_sliver_sensitive_and_cheapest():
    need_gpu()
    table = {pre: (_iterations(False, pre), _iterations(True, pre)) for pre in (0, 1, 2)}
    for pre, (u, sl) in table.items():
        print("preconditioner", pre, "uniform %.1f" % u, "slivers %.1f" % sl, "factor %.2f" % (sl / u))
    none_f = table[0][1] / table[0][0]
    pre1_f = table[1][1] / table[1][0]
    pre2_f = table[2][1] / table[2][0]
    assert none_f > 1.5 and pre1_f > 1.2           # slivers hurt without the stencil preconditioner
    assert pre2_f < min(none_f, pre1_f)            # Pre2 is the least sensitive
    assert table[2][1] < table[1][1] < table[0][1]  # and the cheapest in iterations on slivers
