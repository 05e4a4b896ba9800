"""The five synthetic workloads (plus scaled copies of the same construction).

Each builder returns a ``Workload``: mesh, per-element media, discretisation
orders, scheme, time step, initial data (plane wave or zero), Ricker shots and
receivers.  Seeds are 1234 + workload number unless given.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .media import gaussian_random_field, homogeneous, layered_2d, centroids
from .meshes import add_slivers, tet_kuhn, tri_grid


@dataclass
class Workload:
    name: str
    dim: int
    xyz: np.ndarray
    elem_vert: np.ndarray
    period: Optional[np.ndarray]
    lam: np.ndarray
    mu: np.ndarray
    rho: np.ndarray
    p: int
    p_gamma: int
    scheme: str            # "cn" (p_gamma = 0, Crank-Nicolson) or "stdg"
    dt: float
    n_steps: int
    h: float               # nominal structured spacing
    plane_wave: Optional[dict] = None   # {"kind": 0|1, "n": dim, "pol": dim, "amp": a}
    shots_xs: Optional[np.ndarray] = None    # (n_shots, dim)
    shots_dir: Optional[np.ndarray] = None   # (n_shots, dim)
    f0: float = 10.0
    t_delay: float = 0.116
    a1: float = 1.0
    receivers: Optional[np.ndarray] = None   # (n_rec, dim)
    extra: dict = field(default_factory=dict)

    @property
    def n_elem(self):
        return int(self.elem_vert.shape[0])

    @property
    def n_shots(self):
        return 1 if self.shots_xs is None else int(self.shots_xs.shape[0])


def explicit_cfl_dt(h, dim, p, vp_max):
    """Reading of "the explicit CFL": h / (d (2p+1) vp_max)."""
    return h / (dim * (2 * p + 1) * vp_max)


LAYERS = dict(bounds=[1.0 / 3.0, 2.0 / 3.0], vp=[4.0, 3.0, 2.0], vs=[2.3, 1.7, 1.2], rho=[2.0, 1.5, 1.0])


def c1_periodic_pwave(n=20, p=1, steps=10, dt=0.05):
    xyz, ev, per = tri_grid(n, n, 1.0, 1.0, periodic=True)
    lam, mu, rho = homogeneous(ev.shape[0], 2.0, 1.0, 1.0)
    return Workload("c1_periodic_pwave_p%d_%dtri" % (p, ev.shape[0]), 2, xyz, ev, per, lam, mu, rho,
                    p=p, p_gamma=0, scheme="cn", dt=dt, n_steps=steps, h=1.0 / n,
                    plane_wave={"kind": 0, "n": np.array([1.0, 0.0]), "pol": None, "amp": 1e-2})


def _layered_mesh(nx, ny, seed, slivers=True):
    xyz, ev, per = tri_grid(nx, ny, 2.0, 1.0, periodic=False, jitter=0.3, seed=seed)
    h = 1.0 / ny
    if slivers:
        nvx = nx + 1
        vid = np.arange(xyz.shape[0])
        iv, jv = vid % nvx, vid // nvx
        fixed = (iv == 0) | (iv == nx) | (jv == 0) | (jv == ny)
        xyz, sl = add_slivers(xyz, ev, h, 0.01, ratio=70.0, seed=seed + 1, fixed_vertex=fixed)
    else:
        sl = np.zeros(0, dtype=np.int64)
    lam, mu, rho = layered_2d(xyz, ev, per, **LAYERS)
    return xyz, ev, per, lam, mu, rho, h, sl


def c2_layered_slivers(ny=224, p=3, steps=200, seed=1236):
    nx = 2 * ny
    xyz, ev, per, lam, mu, rho, h, sl = _layered_mesh(nx, ny, seed)
    dt = 10.0 * explicit_cfl_dt(h, 2, p, 4.0)
    rec = np.stack([0.1 + 1.8 * np.arange(16) / 15.0, np.full(16, 0.95)], axis=1)
    return Workload("c2_layered_slivers_p%d_%dtri" % (p, ev.shape[0]), 2, xyz, ev, per, lam, mu, rho,
                    p=p, p_gamma=p, scheme="stdg", dt=dt, n_steps=steps, h=h,
                    shots_xs=np.array([[1.0, 0.85]]), shots_dir=np.array([[0.0, 1.0]]),
                    f0=10.0, t_delay=1.16 / 10.0, a1=1.0, receivers=rec, extra={"slivers": sl})


def c3_cube_swave(n=64, p=2, steps=50, dt=0.02, seed=1237):
    xyz, ev, per = tet_kuhn(n, 1.0, periodic=True, jitter=0.2, seed=seed)
    lam, mu, rho = homogeneous(ev.shape[0], 1.0, 1.0, 1.0)
    return Workload("c3_cube_swave_p%d_%dtet" % (p, ev.shape[0]), 3, xyz, ev, per, lam, mu, rho,
                    p=p, p_gamma=p, scheme="stdg", dt=dt, n_steps=steps, h=1.0 / n,
                    plane_wave={"kind": 1, "n": np.array([1.0, 0.0, 0.0]),
                                "pol": np.array([0.0, 1.0, 0.0]), "amp": 1e-2})


def c4_multishot(ny=224, p=2, steps=200, n_shots=64, seed=1236):
    nx = 2 * ny
    xyz, ev, per, lam, mu, rho, h, sl = _layered_mesh(nx, ny, seed)
    dt = 10.0 * explicit_cfl_dt(h, 2, p, 4.0)
    xs = np.stack([0.05 + 1.9 * np.arange(n_shots) / max(n_shots - 1, 1), np.full(n_shots, 0.85)], axis=1)
    rec = np.stack([0.1 + 1.8 * np.arange(16) / 15.0, np.full(16, 0.95)], axis=1)
    return Workload("c4_multishot%d_p%d_%dtri" % (n_shots, p, ev.shape[0]), 2, xyz, ev, per, lam, mu, rho,
                    p=p, p_gamma=p, scheme="stdg", dt=dt, n_steps=steps, h=h,
                    shots_xs=xs, shots_dir=np.tile([0.0, 1.0], (n_shots, 1)),
                    f0=10.0, t_delay=0.116, a1=1.0, receivers=rec)


def c4_ragged(k, p=2, steps=200, seed=1300, scale=1.0):
    """Mesh k of the ragged batch: ~5000 * 16^(k/15) triangles (times ``scale``)."""
    n_tri = 5000.0 * 16.0 ** (k / 15.0) * scale
    ny = max(3, int(round(np.sqrt(n_tri / 4.0))))
    nx = 2 * ny
    xyz, ev, per = tri_grid(nx, ny, 2.0, 1.0, periodic=False, jitter=0.3, seed=seed + k)
    lam, mu, rho = homogeneous(ev.shape[0], 1.12, 1.44, 1.0)
    h = 1.0 / ny
    dt = 10.0 * explicit_cfl_dt(h, 2, p, 2.0)
    return Workload("c4_ragged%d_p%d_%dtri" % (k, p, ev.shape[0]), 2, xyz, ev, per, lam, mu, rho,
                    p=p, p_gamma=p, scheme="stdg", dt=dt, n_steps=steps, h=h,
                    shots_xs=np.array([[1.0, 0.5]]), shots_dir=np.array([[0.0, 1.0]]),
                    f0=10.0, t_delay=0.116, a1=1.0,
                    receivers=np.array([[0.5, 0.9], [1.5, 0.9]]))


def c5_adjoint(ny=123, nx=None, p=2, steps=300, n_shots=8, n_rec=100, seed=1239, true_model=False):
    nx = 2 * ny - 2 if nx is None else nx
    xyz, ev, per = tri_grid(nx, ny, 2.0, 1.0, periodic=False, jitter=0.3, seed=seed)
    c = centroids(xyz, ev, per)
    g = [gaussian_random_field(c, 0.2, 256, seed=seed + 10 + k) for k in range(3)]
    base = np.array([2.0, 1.0, 1.0])
    lam, mu, rho = (base[k] * (1.0 + 0.2 * g[k]) for k in range(3))
    if true_model:
        bump = 0.05 * np.exp(-np.sum((c - np.array([1.0, 0.5])) ** 2, axis=1) / 0.15 ** 2)
        lam, mu, rho = lam * (1 + bump), mu * (1 + bump), rho * (1 + bump)
    h = 1.0 / ny
    vp_max = float(np.sqrt((lam + 2 * mu) / rho).max())
    dt = 10.0 * explicit_cfl_dt(h, 2, p, vp_max)
    xs = np.stack([0.125 + 0.25 * np.arange(n_shots), np.full(n_shots, 0.85)], axis=1)
    rec = np.stack([0.02 + 1.96 * np.arange(n_rec) / max(n_rec - 1, 1), np.full(n_rec, 0.95)], axis=1)
    return Workload("c5_adjoint_p%d_%dtri" % (p, ev.shape[0]), 2, xyz, ev, per, lam, mu, rho,
                    p=p, p_gamma=p, scheme="stdg", dt=dt, n_steps=steps, h=h,
                    shots_xs=xs, shots_dir=np.tile([0.0, 1.0], (n_shots, 1)),
                    f0=10.0, t_delay=0.116, a1=1.0, receivers=rec)


def scaled(name, **kw):
    """Small copies of the same constructions, sized for the oracle."""
    if name == "c1":
        return c1_periodic_pwave(**kw)
    if name == "c2":
        kw.setdefault("ny", 28)
        kw.setdefault("steps", 5)
        return c2_layered_slivers(**kw)
    if name == "c3":
        kw.setdefault("n", 4)
        kw.setdefault("steps", 3)
        return c3_cube_swave(**kw)
    if name == "c4":
        kw.setdefault("ny", 12)
        kw.setdefault("steps", 3)
        kw.setdefault("n_shots", 4)
        return c4_multishot(**kw)
    if name == "c5":
        kw.setdefault("ny", 8)
        kw.setdefault("steps", 6)
        kw.setdefault("n_shots", 2)
        kw.setdefault("n_rec", 5)
        return c5_adjoint(**kw)
    raise KeyError(name)


def ragged_union(ks=range(16), p=2, steps=200, scale=1.0, seed=1300, gap=0.5):
    """The ragged batch as one input: meshes c4_ragged(k) placed side by side (x-shifted by
    their width plus ``gap``) as one disconnected mesh, so that one context -- and one launch
    per kernel -- advances all of them.  ``dt`` is the smallest part's time step; extra
    ``part_dt`` holds each part's own (10x CFL) step and ``alpha`` the per-element ratio
    part_dt / dt, the time scale that lets every part advance at its own step.
    Returns (Workload, list of (first element, element count) per part)."""
    parts = [c4_ragged(k, p=p, steps=steps, seed=seed, scale=scale) for k in ks]
    xyz, ev, lam, mu, rho, xs, rec, spans = [], [], [], [], [], [], [], []
    voff, eoff, xoff = 0, 0, 0.0
    for w in parts:
        shift = np.array([xoff, 0.0])
        xyz.append(w.xyz + shift)
        ev.append(w.elem_vert + voff)
        lam.append(w.lam); mu.append(w.mu); rho.append(w.rho)
        xs.append(w.shots_xs[0] + shift)
        rec.append(w.receivers + shift)
        spans.append((eoff, w.n_elem))
        voff += w.xyz.shape[0]
        eoff += w.n_elem
        xoff += 2.0 + gap
    dt = min(w.dt for w in parts)
    alpha = np.concatenate([np.full(w.n_elem, w.dt / dt) for w in parts])
    u = Workload("c4_ragged_union%d_p%d_%dtri" % (len(parts), p, eoff), 2, np.concatenate(xyz),
                 np.concatenate(ev).astype(np.int32), None, np.concatenate(lam), np.concatenate(mu),
                 np.concatenate(rho), p=p, p_gamma=p, scheme="stdg", dt=dt, n_steps=steps, h=parts[0].h,
                 shots_xs=None, shots_dir=None, receivers=np.concatenate(rec),
                 extra={"part_sources": np.array(xs), "spans": spans, "part_dt": [w.dt for w in parts],
                        "alpha": alpha})
    return u, spans


def permuted(w, seed=0):
    """The same workload with its elements and vertices renumbered by a seeded random
    permutation (the same mesh, media, sources and receivers in an unfavourable order)."""
    import dataclasses
    rng = np.random.default_rng(seed)
    pe = rng.permutation(w.n_elem)
    pv = rng.permutation(w.xyz.shape[0])            # new id of old vertex v: inv[v]
    inv = np.empty_like(pv)
    inv[pv] = np.arange(pv.size)
    return dataclasses.replace(w, name=w.name + "_permuted", xyz=w.xyz[pv], elem_vert=inv[w.elem_vert[pe]].astype(np.int32),
                               lam=w.lam[pe], mu=w.mu[pe], rho=w.rho[pe])
