"""Shared helpers of the test-suite: build the oracle and the library on one workload."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    with open(os.path.join(ROOT, "include", "stdg.h")) as f:
        text = f.read()
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


def face_neighbours(elem_vert):
    """Face neighbours of every element of a mesh without periodic faces: (n_elem, d+1)
    array, -1 where the face is on the boundary (faces matched by sorted vertex tuples)."""
    ev = np.asarray(elem_vert)
    ne, nv = ev.shape
    faces = np.concatenate([np.sort(np.delete(ev, k, axis=1), axis=1) for k in range(nv)])   # (nv*ne, d)
    owner = np.tile(np.arange(ne), nv)
    local = np.repeat(np.arange(nv), ne)
    _, inv, cnt = np.unique(faces, axis=0, return_inverse=True, return_counts=True)
    inv = inv.ravel()
    order = np.argsort(inv, kind="stable")
    nb = np.full((ne, nv), -1, dtype=np.int64)
    first = np.concatenate([[0], np.cumsum(cnt)[:-1]])
    for g in np.where(cnt == 2)[0]:
        a, b = order[first[g]], order[first[g] + 1]
        nb[owner[a], local[a]] = owner[b]
        nb[owner[b], local[b]] = owner[a]
    return nb


def patch_operator_rows(w, elems, x, nb=None, quad_n=None):
    """(A x)_i for the sampled elements i of a large mesh, each from the oracle's assembled
    operator on the patch {i and its face neighbours}: row i of A couples only those
    elements, through the faces of i, whose dual cells and E_j the patch reproduces (the
    patch numbers its elements differently, which changes l(j)/r(j) but not A).  Meshes
    without periodic faces only.  Returns (len(elems), d * N_gamma * N_phi)."""
    from oracle.mesh import DualMesh
    from oracle.operators import Discretization
    assert w.period is None
    nb = face_neighbours(w.elem_vert) if nb is None else nb
    xe = np.asarray(x).reshape(w.n_elem, -1)
    rows = []
    for i in elems:
        P = np.concatenate([[i], np.sort(nb[i][nb[i] >= 0])])
        verts, ev = np.unique(w.elem_vert[P], return_inverse=True)
        ev = ev.reshape(len(P), -1).astype(np.int32)
        dz = Discretization(DualMesh(w.xyz[verts], ev, None), w.p, w.p_gamma, w.lam[P], w.mu[P], w.rho[P],
                            quad_n=quad_n)
        A = dz.assemble(w.dt, w.scheme)
        rows.append((A @ xe[P].ravel()).reshape(len(P), -1)[0])
    return np.array(rows)


def extended_patch_rows(w, elems, x, nb=None, quad_n=None):
    """(A x)_i for the sampled elements in extended precision (oracle/extended.py), each on
    the patch {i and its face neighbours} as in patch_operator_rows.  Meshes without periodic
    faces only.  Returns an np.longdouble array (len(elems), d * N_gamma * N_phi)."""
    from oracle.extended import PatchOperator
    assert w.period is None
    nb = face_neighbours(w.elem_vert) if nb is None else nb
    xe = np.asarray(x).reshape(w.n_elem, -1)
    rows = []
    for i in elems:
        P = np.concatenate([[i], np.sort(nb[i][nb[i] >= 0])])
        verts, ev = np.unique(w.elem_vert[P], return_inverse=True)
        ev = ev.reshape(len(P), -1)
        op = PatchOperator(w.xyz[verts], ev, w.lam[P], w.mu[P], w.rho[P], w.p, w.p_gamma, w.scheme, w.dt,
                           quad_n=quad_n)
        rows.append(op.row(0, xe[P].ravel()).ravel())
    return np.array(rows)


def rel_l2_ext(a, ref):
    """rel_l2 with the reference kept in its own (extended) precision."""
    ref = np.asarray(ref)
    a = np.asarray(a).astype(ref.dtype)
    return float(np.sqrt(np.sum((a - ref) ** 2)) / np.sqrt(np.sum(ref * ref)))
