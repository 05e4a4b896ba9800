"""Structured-then-jittered simplex meshes (2D triangles, 3D Kuhn tetrahedra).

Conventions shared by every consumer:
  * vertices are unique; on a periodic axis the vertex at the far end is identified
    with the one at the near end (it is not duplicated), so an element that crosses
    the seam lists vertices whose coordinates lie a period apart;
  * ``period`` is ``None`` (no periodic axis) or a length-``dim`` float array whose
    entry is the period of that axis, or 0 where the axis is not periodic;
  * every element is positively oriented once unwrapped (see ``unwrap_elements``).
"""
import itertools

import numpy as np


def unwrap_elements(xyz, elem_vert, period):
    """Vertex coordinates per element, shifted by whole periods next to vertex 0.

    Returns an array (n_elem, dim+1, dim).  Pure geometry bookkeeping.
    """
    X = xyz[elem_vert].astype(np.float64)
    if period is None:
        return X
    per = np.asarray(period, dtype=np.float64)
    for a in range(X.shape[2]):
        if per[a] > 0:
            delta = X[:, :, a] - X[:, :1, a]
            X[:, :, a] -= per[a] * np.round(delta / per[a])
    return X


def _signed_volume(X):
    d = X.shape[2]
    J = X[:, 1:, :] - X[:, :1, :]
    return np.linalg.det(J) / (1 if d == 1 else (2 if d == 2 else 6))


def tri_grid(nx, ny, Lx=1.0, Ly=1.0, periodic=False, jitter=0.0, seed=0):
    """nx*ny cells, each split along its (0,0)-(1,1) diagonal into two CCW triangles.

    jitter: vertices move by a seeded uniform offset in [-jitter*h, jitter*h] per axis
    (h = cell size along that axis); on a non-periodic box, boundary vertices move
    only tangentially and corners stay fixed.
    Returns (xyz[n_vert,2], elem_vert[n_elem,3] int32, period or None).
    """
    hx, hy = Lx / nx, Ly / ny
    nvx, nvy = (nx, ny) if periodic else (nx + 1, ny + 1)
    jj, ii = np.meshgrid(np.arange(nvy), np.arange(nvx), indexing="ij")
    xyz = np.stack([ii.ravel() * hx, jj.ravel() * hy], axis=1).astype(np.float64)
    if jitter > 0:
        rng = np.random.default_rng(seed)
        off = rng.uniform(-jitter, jitter, size=xyz.shape) * np.array([hx, hy])
        if not periodic:
            iv, jv = ii.ravel(), jj.ravel()
            off[(iv == 0) | (iv == nx), 0] = 0.0
            off[(jv == 0) | (jv == ny), 1] = 0.0
        xyz = _apply_jitter(xyz, off, elem_fn=lambda: _tri_elems(nx, ny, nvx, nvy, periodic),
                            period=np.array([Lx, Ly]) if periodic else None)

    elem = _tri_elems(nx, ny, nvx, nvy, periodic)
    period = np.array([Lx, Ly]) if periodic else None
    return xyz, elem, period


def _apply_jitter(xyz, off, elem_fn, period):
    """Add ``off``; halve the offsets of vertices of inverted elements until none is."""
    elem = elem_fn()
    off = off.copy()
    for _ in range(60):
        vol = _signed_volume(unwrap_elements(xyz + off, elem, period))
        bad = vol <= 0
        if not bad.any():
            break
        off[np.unique(elem[bad])] *= 0.5
    return xyz + off


def _tri_elems(nx, ny, nvx, nvy, periodic):
    def vid(i, j):
        if periodic:
            return (j % nvy) * nvx + (i % nvx)
        return j * nvx + i

    jc, ic = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    ic, jc = ic.ravel(), jc.ravel()
    v00, v10 = vid(ic, jc), vid(ic + 1, jc)
    v01, v11 = vid(ic, jc + 1), vid(ic + 1, jc + 1)
    ta = np.stack([v00, v10, v11], axis=1)
    tb = np.stack([v00, v11, v01], axis=1)
    return np.stack([ta, tb], axis=1).reshape(-1, 3).astype(np.int32)


def add_slivers(xyz, elem, h, fraction, ratio=70.0, seed=0, fixed_vertex=None):
    """Turn a seeded ``fraction`` of triangles into slivers (no two share a vertex).

    For each chosen triangle the vertex opposite its longest edge is moved along the
    edge normal until its distance to that edge is h/ratio; a move that would invert
    any triangle around that vertex is rejected.  ``fixed_vertex`` (bool per vertex)
    marks vertices that must not move (e.g. the boundary of a non-periodic box).
    Returns (new xyz, indices of the sliver triangles).
    """
    xyz = xyz.copy()
    n_elem = elem.shape[0]
    target = int(round(fraction * n_elem))
    rng = np.random.default_rng(seed)
    order = rng.permutation(n_elem)
    used = np.zeros(xyz.shape[0], dtype=bool)
    if fixed_vertex is None:
        fixed_vertex = np.zeros(xyz.shape[0], dtype=bool)
    v2e = [[] for _ in range(xyz.shape[0])]
    for e, tri in enumerate(elem):
        for v in tri:
            v2e[v].append(e)
    chosen = []
    for e in order:
        if len(chosen) >= target:
            break
        tri = elem[e]
        if used[tri].any():
            continue
        P = xyz[tri]
        lens = [np.linalg.norm(P[(k + 2) % 3] - P[(k + 1) % 3]) for k in range(3)]
        k = int(np.argmax(lens))  # vertex k is opposite the longest edge
        a = tri[k]
        if fixed_vertex[a]:
            continue
        b, c = P[(k + 1) % 3], P[(k + 2) % 3]
        t = c - b
        t = t / np.linalg.norm(t)
        foot = b + np.dot(P[k] - b, t) * t
        nrm = P[k] - foot
        dist = np.linalg.norm(nrm)
        if dist <= h / ratio:
            continue
        old = xyz[a].copy()
        xyz[a] = foot + nrm / dist * (h / ratio)
        ok = True
        for e2 in v2e[a]:
            Q = xyz[elem[e2]]
            area = 0.5 * ((Q[1, 0] - Q[0, 0]) * (Q[2, 1] - Q[0, 1]) - (Q[1, 1] - Q[0, 1]) * (Q[2, 0] - Q[0, 0]))
            if area <= 0:
                ok = False
                break
        if not ok:
            xyz[a] = old
            continue
        used[tri] = True
        chosen.append(e)
    return xyz, np.array(chosen, dtype=np.int64)


def tet_kuhn(n, L=1.0, periodic=False, jitter=0.0, seed=0):
    """n^3 cubes, each split into the 6 Kuhn tetrahedra sharing its main diagonal.

    Returns (xyz[n_vert,3], elem_vert[n_elem,4] int32, period or None); elements are
    cube-major (x fastest, then y, then z), 6 per cube, positively oriented.
    """
    h = L / n
    nv = n if periodic else n + 1
    kk, jj, ii = np.meshgrid(np.arange(nv), np.arange(nv), np.arange(nv), indexing="ij")
    xyz = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64) * h
    if jitter > 0:
        rng = np.random.default_rng(seed)
        off = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
        if not periodic:
            for a, idx in enumerate([ii.ravel(), jj.ravel(), kk.ravel()]):
                off[(idx == 0) | (idx == n), a] = 0.0
        xyz = _apply_jitter(xyz, off, elem_fn=lambda: _tet_elems(n, nv, periodic),
                            period=np.array([L, L, L]) if periodic else None)
    elem = _tet_elems(n, nv, periodic)
    period = np.array([L, L, L]) if periodic else None
    return xyz, elem, period


def _tet_elems(n, nv, periodic):
    def vid(i, j, k):
        if periodic:
            return ((k % nv) * nv + (j % nv)) * nv + (i % nv)
        return (k * nv + j) * nv + i

    kc, jc, ic = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ic, jc, kc = ic.ravel(), jc.ravel(), kc.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        cur = [0, 0, 0]
        path = [tuple(cur)]
        for ax in perm:
            cur[ax] = 1
            path.append(tuple(cur))
        ids = [vid(ic + p[0], jc + p[1], kc + p[2]) for p in path]
        # a Kuhn simplex is positively oriented iff its axis permutation is even
        inversions = sum(1 for x in range(3) for y in range(x + 1, 3) if perm[x] > perm[y])
        if inversions % 2 == 1:
            ids[2], ids[3] = ids[3], ids[2]
        tets.append(np.stack(ids, axis=1))
    return np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)


def check_positive(xyz, elem, period):
    vol = _signed_volume(unwrap_elements(xyz, elem, period))
    return bool((vol > 0).all()), vol
