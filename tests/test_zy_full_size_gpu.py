"""GPU vs oracle at the benchmark's full size: the 200,704-triangle layered sliver mesh at
p = p_gamma = 3, the configuration bench.py times.  The oracle cannot assemble A at this
size, but row i of A couples only element i and its face neighbours, through the faces of
i: the oracle's operator on that patch gives (A x)_i exactly (up to rounding;
tests/test_patch_rows.py checks this against the full assembly on CPU).  Sampled rows: 12
elements drawn at random and 12 slivers, against the extended-precision oracle
(oracle/extended.py: the FP64 oracle's own rounding on sliver dual cells is ~1e-10, the
size of the bar).  FP64 (the FP64 path's face and mass kernels) within the stated 1e-10 on
both groups; FP32 (the single-shot TMA face kernel and mass kernel of the mixed path's
inner solve) within 1e-6 on the random rows.  The FP64 oracle's rows are printed beside
them."""
import numpy as np
import pytest

import synth
from helpers import extended_patch_rows, face_neighbours, gpu_solver, need_gpu, patch_operator_rows, rel_l2_ext

pytestmark = pytest.mark.gpu


def _samples(w, rng):
    X = w.xyz[w.elem_vert]
    a, b = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]
    area = 0.5 * (a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    h = w.xyz[:, 1].max() / 224
    slivers = np.where(area / (0.5 * h * h) < 0.05)[0]
    return rng.choice(w.n_elem, 12, replace=False), rng.choice(slivers, 12, replace=False)


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
    for name, idx in zip(("random", "sliver"), groups):
        ext = extended_patch_rows(w, idx, x, nb)
        r64 = patch_operator_rows(w, idx, x, nb)
        err = rel_l2_ext(y[idx], ext)
        print("FP64 %s rows: error %.3g vs extended-precision oracle (FP64 oracle vs extended %.3g)"
              % (name, err, rel_l2_ext(r64, ext)))
        assert err < 1e-10
        refs.append(ext)
    m = gpu_solver(w, precision="mixed", with_sources=False, with_receivers=False)
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.zeros_like(xd)
    torch.cuda.synchronize()
    m.apply_operator_device(w.dt, xd.data_ptr(), yd.data_ptr(), fp32=True)
    torch.cuda.synchronize()
    y32 = yd.cpu().numpy().astype(np.float64).reshape(w.n_elem, -1)
    m.close()
    err32 = rel_l2_ext(y32[groups[0]], refs[0])
    print("FP32 rows: error %.3g" % err32)
    assert err32 < 1e-6
