"""Shared helpers of the test-suite: build the oracle and the library on one workload."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "stdg.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\*)\s+(stdg_\w+)\s*\(", text, re.M)))


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_04516_gb300 import build
    build.build()
    return torch


def rel_l2(a, b):
    a, b = np.asarray(a).ravel(), np.asarray(b).ravel()
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def gpu_solver(w, **kw):
    from paper_1802_04516_gb300.binding import solver_from_workload
    return solver_from_workload(w, **kw)


def oracle_sim(w, dt=None):
    from oracle.stepper import Simulation
    sim = Simulation.from_workload(w, dt=dt)
    if w.plane_wave is not None:
        pw = w.plane_wave
        sim.set_plane_wave(pw["kind"], pw["n"], pw.get("pol"), pw["amp"])
    return sim


def stress_field_rel(sig, ref, disc):
    """Relative L2 difference of two stress fields given by Taylor-monomial DOFs.

    sum_j int_{R_j} |sigma - ref|^2 (full tensor) / sum_j int_{R_j} |ref|^2, with the oracle's
    dual mass matrices; insensitive to the ill-conditioned directions of the monomial basis.
    """
    from oracle.operators import SYM
    w = np.array([1.0 if a == b else 2.0 for (a, b) in SYM[disc.dim]])
    d = np.asarray(sig) - np.asarray(ref)
    num = np.einsum("c,fcm,fmn,fcn->", w, d, disc.Mdual, d)
    den = np.einsum("c,fcm,fmn,fcn->", w, ref, disc.Mdual, ref)
    return float(np.sqrt(abs(num) / den)) if den > 0 else float(np.sqrt(abs(num)))


def oracle_rounding_spread(sim, w):
    """Relative difference of A x between two oracle evaluations that differ only by rounding.

    The second evaluation integrates with two more quadrature points per direction: both
    rules are exact for the integrands, so the difference measures how far FP64 rounding
    (amplified by cond(M_j) of the Taylor-monomial dual basis) moves the assembled A.
    """
    from oracle.operators import Discretization
    d2 = Discretization(sim.mesh, w.p, w.p_gamma, w.lam, w.mu, w.rho, quad_n=w.p + 5)
    A2 = d2.assemble(w.dt, w.scheme)
    x = np.random.default_rng(11).normal(size=A2.shape[0])
    return rel_l2(A2 @ x, sim.A @ x)
