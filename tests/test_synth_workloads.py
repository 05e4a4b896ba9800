"""The synthetic workloads have the sizes and structure their recipes state (CPU)."""
import numpy as np

import synth
from synth.workloads import explicit_cfl_dt


def _signed_areas(w):
    X = w.xyz[w.elem_vert]
    a = X[:, 1] - X[:, 0]
    b = X[:, 2] - X[:, 0]
    return 0.5 * (a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])


def _n_faces(ev):
    nv = ev.shape[1]
    faces = np.concatenate([np.delete(ev, f, axis=1) for f in range(nv)])
    faces.sort(axis=1)
    return np.unique(faces, axis=0).shape[0]


def test_benchmark_mesh():
    w = synth.c2_layered_slivers()
    assert w.n_elem == 448 * 224 * 2 == 200704
    assert _n_faces(w.elem_vert) == 301728
    area = _signed_areas(w)
    assert area.min() > 0                                      # no inverted element
    h = 1.0 / 224
    q = area / (0.5 * h * h)
    n_sliver = int(np.sum(q < 0.05))
    assert 0.007 * w.n_elem < n_sliver < 0.013 * w.n_elem      # about 1% slivers
    assert abs(w.dt - 10 * explicit_cfl_dt(h, 2, 3, 4.0)) < 1e-15
    assert abs(w.dt - 7.97e-4) < 1e-6
    vp = np.sqrt((w.lam + 2 * w.mu) / w.rho)
    assert np.allclose(sorted(set(np.round(vp, 6))), [2.0, 3.0, 4.0])


def test_multishot_and_ragged_batches():
    w = synth.c4_multishot()
    assert w.n_shots == 64 and w.p == w.p_gamma == 2 and w.n_elem == 200704
    assert np.allclose(w.shots_xs[:, 0], 0.05 + 1.9 * np.arange(64) / 63) and np.allclose(w.shots_xs[:, 1], 0.85)
    u, spans = synth.ragged_union()
    sizes = [n for _, n in spans]
    assert len(sizes) == 16 and sizes == sorted(sizes)
    assert sizes[0] < 5500 and sizes[-1] > 75000 and u.n_elem == sum(sizes) == 449864
    assert [s for s, _ in spans] == list(np.cumsum([0] + sizes[:-1]))
    assert u.extra["part_sources"].shape == (16, 2)
    assert _signed_areas(u).min() > 0


def test_inversion_workload():
    w = synth.c5_adjoint()
    wt = synth.c5_adjoint(true_model=True)
    assert w.n_elem == 244 * 123 * 2 == 60024 and w.n_shots == 8 and len(w.receivers) == 100
    for a, base in ((w.lam, 2.0), (w.mu, 1.0), (w.rho, 1.0)):
        assert np.all(np.abs(a / base - 1.0) <= 0.2 + 1e-12)   # +-20% random field
    bump = wt.lam / w.lam - 1.0
    assert 0.04 < bump.max() <= 0.05 and bump.min() >= 0.0    # +5% Gaussian bump in the true model


def test_generators_are_deterministic():
    # every input is a pure function of its seed: two calls agree bit for bit, another seed differs
    a, b = synth.c2_layered_slivers(ny=16), synth.c2_layered_slivers(ny=16)
    for k in ("xyz", "elem_vert", "lam", "mu", "rho", "receivers", "shots_xs"):
        assert np.array_equal(getattr(a, k), getattr(b, k)), k
    c = synth.c2_layered_slivers(ny=16, seed=7)
    assert not np.array_equal(a.xyz, c.xyz)
    u1, s1 = synth.ragged_union(ks=[0, 3], scale=0.02)
    u2, s2 = synth.ragged_union(ks=[0, 3], scale=0.02)
    assert s1 == s2 and np.array_equal(u1.xyz, u2.xyz) and np.array_equal(u1.elem_vert, u2.elem_vert)
    m1, m2 = synth.c5_adjoint(ny=12), synth.c5_adjoint(ny=12)
    assert np.array_equal(m1.lam, m2.lam) and np.array_equal(m1.mu, m2.mu) and np.array_equal(m1.rho, m2.rho)
