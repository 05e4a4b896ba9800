"""The library's host-side mesh code on CPU, bit for bit against the oracle: row a1 (mesh
connectivity, Sec. 3: stdg_mesh_faces, the code stdg_set_mesh runs) on small 2D/3D,
periodic and bounded meshes and on the full 200,704-triangle benchmark mesh, with its
rejections of bad meshes; the location of sources and receivers (rows a8/a9:
stdg_locate_points, the code the source and receiver calls run); and the reference mass
matrix and time factors of row a2 (stdg_reference_tables)."""
import ctypes

import numpy as np
import pytest

import synth
from oracle.mesh import DualMesh


def _faces(xyz, ev, per):
    from paper_1802_04516_gb300 import build
    from paper_1802_04516_gb300.binding import load, mesh_faces
    load(build.build())
    return mesh_faces(xyz, ev, per)


CASES = {
    "2d_periodic_jittered": lambda: synth.tri_grid(5, 4, 1.0, 0.8, periodic=True, jitter=0.25, seed=1),
    "2d_bounded": lambda: synth.tri_grid(6, 3, 2.0, 1.0, periodic=False, jitter=0.2, seed=2),
    "3d_periodic": lambda: synth.tet_kuhn(3, 1.0, periodic=True, jitter=0.15, seed=3),
    "3d_bounded": lambda: synth.tet_kuhn(3, 1.0, periodic=False, jitter=0.1, seed=4),
    "2d_sliver_layers": lambda: (lambda w: (w.xyz, w.elem_vert, w.period))(synth.scaled("c2", ny=10, steps=1)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_face_table_matches_oracle(name):
    xyz, ev, per = CASES[name]()
    m = DualMesh(xyz, ev, per)
    fl, fr = _faces(xyz, ev, per)
    assert np.array_equal(fl, m.face_l) and np.array_equal(fr, m.face_r)


def test_face_table_matches_oracle_on_the_benchmark_mesh():
    w = synth.c2_layered_slivers()
    m = DualMesh(w.xyz, w.elem_vert, w.period)
    fl, fr = _faces(w.xyz, w.elem_vert, w.period)
    assert len(fl) == m.n_face == 301728
    assert np.array_equal(fl, m.face_l) and np.array_equal(fr, m.face_r)


def _rc(xyz, ev, per=None, cap=None, arrays=True):
    from paper_1802_04516_gb300 import build
    from paper_1802_04516_gb300.binding import load
    lib = load(build.build())
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    ev = np.ascontiguousarray(ev, dtype=np.int32)
    per_p = None if per is None else np.ascontiguousarray(per, dtype=np.float64).ctypes.data_as(
        ctypes.POINTER(ctypes.c_double))
    n = ctypes.c_int64(cap if cap is not None else 0)
    fl = np.zeros(max(cap or 0, 1), dtype=np.int32)
    fr = np.zeros(max(cap or 0, 1), dtype=np.int32)
    i32 = ctypes.POINTER(ctypes.c_int32)
    rc = lib.stdg_mesh_faces(ev.shape[1] - 1, xyz.shape[0], xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                             ev.shape[0], ev.ctypes.data_as(i32), per_p, ctypes.byref(n),
                             fl.ctypes.data_as(i32) if arrays else None, fr.ctypes.data_as(i32) if arrays else None)
    return rc, n.value


def test_rejections():
    xyz, ev, _ = synth.tri_grid(3, 3, 1.0, 1.0, periodic=False)
    rc, n = _rc(xyz, ev, arrays=False)
    assert rc == 0 and n == DualMesh(xyz, ev, None).n_face
    assert _rc(xyz, ev, cap=n) == (0, n)
    assert _rc(xyz, ev, cap=n - 1) == (-1, n)                  # capacity too small: count still set
    bad = ev.copy()
    bad[4] = bad[4, [0, 2, 1]]                                 # one element turned clockwise
    assert _rc(xyz, bad)[0] == -2
    bad = ev.copy()
    bad[0, 1] = xyz.shape[0]                                   # vertex index out of range
    assert _rc(xyz, bad)[0] == -1
    nan = xyz.copy()
    nan[ev[2, 0], 0] = np.nan
    assert _rc(nan, ev)[0] == -1
    # a face shared by three triangles
    tri3 = np.array([[0.0, 0.0], [1.0, 0.0], [0.5, 1.0], [0.5, -1.0], [0.6, 2.0]])
    ev3 = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], dtype=np.int32)
    assert _rc(tri3, ev3)[0] == -2


def _locate_lib(xyz, ev, pts, per):
    from paper_1802_04516_gb300 import build
    from paper_1802_04516_gb300.binding import load, locate_points
    load(build.build())
    return locate_points(xyz, ev, pts, per)


def _locate_oracle(m, pts):
    out = []
    for x in pts:
        try:
            out.append(m.locate(x)[0])
        except ValueError:
            out.append(-1)
    return np.array(out)


@pytest.mark.parametrize("name", ["2d_periodic_jittered", "2d_bounded", "3d_periodic", "3d_bounded"])
def test_point_location_matches_oracle(name):
    # rows a8/a9 (receivers, point sources): the element of every point, bit for bit, with the
    # reading's ties -- element centroids, face midpoints, vertices, random and outside points
    xyz, ev, per = CASES[name]()
    m = DualMesh(xyz, ev, per)
    rng = np.random.default_rng(8)
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    pts = np.concatenate([m.X.mean(axis=1), m.face_X.mean(axis=1), m.X[::3, 0],
                          rng.uniform(lo, hi, size=(60, xyz.shape[1])),
                          rng.uniform(lo - 0.5, hi + 0.5, size=(20, xyz.shape[1]))])
    got = _locate_lib(xyz, ev, pts, per)
    want = _locate_oracle(m, pts)
    assert np.array_equal(got, want)
    assert (want >= 0).sum() > len(pts) // 2


def test_workload_sources_and_receivers_match_oracle():
    for w in (synth.scaled("c2", ny=10, steps=1), synth.scaled("c4", ny=8, steps=1, n_shots=16),
              synth.scaled("c5", ny=10, steps=1)):
        m = DualMesh(w.xyz, w.elem_vert, w.period)
        pts = np.concatenate([w.shots_xs, w.receivers])
        got = _locate_lib(w.xyz, w.elem_vert, pts, w.period)
        assert np.array_equal(got, _locate_oracle(m, pts)) and (got >= 0).all()


@pytest.mark.parametrize("dim,p,pg", [(2, 1, 1), (2, 2, 2), (2, 3, 3), (2, 4, 2), (3, 1, 0), (3, 2, 2), (3, 3, 1)])
def test_reference_tables_match_oracle(dim, p, pg):
    # row a2 on the host: the reference mass matrix of the nodal basis and the time factors
    # (Eqs. MD_2 - MD_2_3) that every kernel uses, against the oracle's own bases and rules
    from oracle.basis import RefBasis, TimeBasis
    from oracle.quadrature import ref_simplex_rule
    from paper_1802_04516_gb300 import build
    from paper_1802_04516_gb300.binding import load, reference_tables
    load(build.build())
    lib = reference_tables(dim, p, pg)
    rp, rw = ref_simplex_rule(dim, p + 3)
    phi = RefBasis(dim, p).values(rp)
    Mref = np.einsum("q,qk,qm->km", rw, phi, phi)
    tm = TimeBasis(pg).matrices()
    W, T, g0, g1 = tm["W"], tm["T"], tm["g0"], tm["g1"]
    Tinv = np.linalg.inv(T)
    ref = dict(Mref=Mref, W=np.diag(W), T=T, S=W @ Tinv @ W, kappa=g1 @ Tinv @ g0, u=g1 @ Tinv @ W)
    assert np.abs(W - np.diag(np.diag(W))).max() < 1e-15          # the nodal time basis is orthogonal
    for k, v in ref.items():
        assert np.allclose(lib[k], v, rtol=1e-12, atol=1e-13 * np.abs(v).max()), k
