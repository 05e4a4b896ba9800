"""The allocation-free residual entry point against the library's existing entry points.

stdg_residual_noalloc serves callers that cannot call cudaMalloc (code running during a
CUDA-graph stream capture, pipelines that cannot take cudaFree's device-wide
synchronisation, processes whose HBM is reserved by another allocator).  Its scratch is a
fixed array inside the library, shared by every call; two calls in a row must both be
right, whatever the previous call left in it.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth
from helpers import gpu_solver, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def test_residual_noalloc_matches_existing_entry_points():
    torch = need_gpu()
    from paper_1802_04516_gb300 import binding
    w = synth.scaled("c2", ny=6, p=2, steps=1)
    s = gpu_solver(w, with_sources=False, with_receivers=False)
    lib = binding.load()
    n = s.nvel
    g = torch.Generator(device="cuda").manual_seed(3)
    for call in range(2):
        x = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        b = torch.randn(n, dtype=torch.float64, device="cuda", generator=g) * (1 + call)
        r = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        rc = lib.stdg_residual_noalloc(s.h, w.dt, x.data_ptr(), b.data_ptr(), r.data_ptr(), out.data_ptr())
        assert rc == 0, lib.stdg_last_error(s.h)
        torch.cuda.synchronize()
        # reference: the existing operator entry point, residual and norms formed by torch
        y = torch.empty_like(x)
        s.apply_operator_device(w.dt, x.data_ptr(), y.data_ptr())
        torch.cuda.synchronize()
        r_ref = (b - y).cpu().numpy()
        rel_ref = np.linalg.norm(r_ref) / np.linalg.norm(b.cpu().numpy())
        assert rel_l2(r.cpu().numpy(), r_ref) < 1e-12
        o = out.cpu().numpy()
        assert abs(o[0] - rel_ref) <= 1e-12 * rel_ref
        assert abs(o[1] - np.linalg.norm(r_ref)) <= 1e-12 * np.linalg.norm(r_ref)
