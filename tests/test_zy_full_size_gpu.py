"""GPU vs oracle at the benchmark's full size: the 200,704-triangle layered sliver mesh at
p = p_gamma = 3, the configuration bench.py times.  The oracle cannot assemble A at this
size, but row i of A couples only element i and its face neighbours, through the faces of
i: the oracle's assembled operator on that patch gives (A x)_i exactly (up to rounding;
tests/helpers.py checks this against the full assembly on CPU).  Sampled rows: 12 elements
drawn at random and 12 slivers.  FP64 (the FP64 path's face and mass kernels) within 20x
the oracle's own rounding spread on those rows, never worse than 1e-10 where the spread
allows it (the rule of the small-mesh operator tests); FP32 (the single-shot TMA face
kernel and mass kernel of the mixed path's inner solve) within 1e-6 on the random rows
(measured on a GB300: FP64 8.5e-13 and 2.7e-10 against bars of 2.3e-11 and 9.9e-9, FP32
9.3e-8)."""
import numpy as np
import pytest

import synth
from helpers import face_neighbours, gpu_solver, need_gpu, patch_operator_rows, rel_l2

pytestmark = pytest.mark.gpu


def _samples(w, rng):
    X = w.xyz[w.elem_vert]
    a, b = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
    area = 0.5 * (a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    h = w.xyz[:, 1].max() / 224
    slivers = np.where(area / (0.5 * h * h) < 0.05)[0]
    return rng.choice(w.n_elem, 12, replace=False), rng.choice(slivers, 12, replace=False)


def _bar(spread):
    return max(1e-12, 20 * spread) if spread > 5e-12 else max(1e-12, min(1e-10, 20 * spread))


def test_full_size_operator_rows_match_oracle():
    torch = need_gpu()
    w = synth.c2_layered_slivers()
    assert w.n_elem == 200704
    nb = face_neighbours(w.elem_vert)
    rng = np.random.default_rng(3)
    groups = _samples(w, rng)
    s = gpu_solver(w, with_sources=False, with_receivers=False)
    x = rng.normal(size=s.nvel)
    y = s.apply_operator(w.dt, x).reshape(w.n_elem, -1)
    s.close()
    refs = []
    for idx in groups:
        r1 = patch_operator_rows(w, idx, x, nb)
        r2 = patch_operator_rows(w, idx, x, nb, quad_n=w.p + 5)
        tol = _bar(rel_l2(r2, r1))
        err = rel_l2(y[idx], r1)
        print("FP64 rows: error %.3g, bar %.3g" % (err, tol))
        assert err < tol
        refs.append(r1)
    m = gpu_solver(w, precision="mixed", with_sources=False, with_receivers=False)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.zeros_like(xd)
    torch.cuda.synchronize()
    m.apply_operator_device(w.dt, xd.data_ptr(), yd.data_ptr(), fp32=True)
    torch.cuda.synchronize()
    y32 = yd.cpu().numpy().astype(np.float64).reshape(w.n_elem, -1)
    m.close()
    err32 = rel_l2(y32[groups[0]], refs[0])
    print("FP32 rows: error %.3g" % err32)
    assert err32 < 1e-6
