"""Pins of the oracle's misfit gradient (oracle/adjoint.py).

* every transpose passes a dot-product test <y, F x> = <F^T y, x> with random vectors;
* the slab matrix satisfies A^T = J A J, J the reversal of the time nodes (the Lagrange
  basis on the symmetric Gauss-Legendre points gives T^T = J T J and S^T = J S J), which
  the GPU adjoint uses to solve with A^T;
* the gradient matches central finite differences of the misfit with direct solves
  (relative steps 1e-4 and 5e-5, Richardson-extrapolated) for lambda, mu and rho on
  seeded elements.
A dropped term, a wrong sign, a missing mirror entry or a transposed block fails one of them.
"""
import numpy as np
import pytest

import synth
from oracle import adjoint as adj
from oracle.stepper import Simulation


def _tiny(p=1, pg=1, ny=5, steps=12, n_shots=2, n_rec=6):
    w = synth.c5_adjoint(ny=ny, p=p, steps=steps, n_shots=n_shots, n_rec=n_rec)
    w_true = synth.c5_adjoint(ny=ny, p=p, steps=steps, n_shots=n_shots, n_rec=n_rec, true_model=True)
    return w, w_true, pg


def _geom(w, pg):
    return (w.xyz, w.elem_vert, w.period, w.p, pg, w.dt)


def _sources(w):
    return [(w.shots_xs[k], w.shots_dir[k]) for k in range(w.n_shots)]


@pytest.mark.parametrize("p,pg", [(1, 1), (2, 2)])
def test_transposes_pass_dot_product_tests(p, pg):
    w, _, _ = _tiny(p=p, pg=pg)
    sim = Simulation(w.xyz, w.elem_vert, w.period, w.lam, w.mu, w.rho, p, pg, "stdg", w.dt)
    dz, m = sim.disc, sim.mesh
    rng = np.random.default_rng(3)
    d, ne, nf = dz.dim, m.n_elem, m.n_face
    vel_st = (ne, d, dz.Ng * dz.Nphi)
    ful_st = (nf, d, d, dz.Ng * dz.Npsi)
    sym_st = (nf, dz.s, dz.Ng * dz.Npsi)
    sym_tr = (nf, dz.s, dz.Npsi)
    ful_tr = (nf, d, d, dz.Npsi)
    vel_tr = (ne, d, dz.Nphi)
    pairs = [
        (dz.D_dot_sigma, lambda u: adj.D_dot_sigma_T(dz, u), ful_st, vel_st),
        (lambda v: adj.Q_gather(dz, v), lambda G: adj.Q_gather_T(dz, G), vel_st, ful_st),
        (lambda G: adj.E_contract(dz.E, G), lambda Y: adj.E_contract_T(dz.E, Y), ful_st, ful_st),
        (dz.full_from_sym, lambda f: adj.full_from_sym_T(dz, f), sym_st, ful_st),
        (dz.sym_from_full, lambda s: adj.sym_from_full_T(dz, s), ful_st, sym_st),
        (lambda Y: adj.minv(dz, Y), lambda Y: adj.minv_T(dz, Y), ful_st, ful_st),
        (lambda S: adj.mminus(dz, S), lambda Y: adj.mminus_T(dz, Y), ful_tr, ful_st),
        (lambda y: adj.trace_time(dz, y, dz.Npsi), lambda t: adj.trace_time_T(dz, t), sym_st, sym_tr),
        (lambda s: adj.Bs_apply(dz, s), lambda l: adj.Bs_T(dz, l), sym_tr, vel_st),
        (lambda s: adj.Cs_apply(dz, s), lambda a: adj.Cs_T(dz, a), sym_tr, sym_tr),
        (lambda x: adj.Cx_apply(dz, x), lambda a: adj.Cx_T(dz, a), vel_st, sym_tr),
        (lambda v: adj.Bv_apply(dz, v), lambda l: adj.Bv_T(dz, l), vel_tr, vel_st),
    ]
    for F, FT, sin, sout in pairs:
        x = rng.normal(size=sin)
        y = rng.normal(size=sout)
        lhs = np.sum(y * F(x))
        rhs = np.sum(FT(y) * x)
        assert abs(lhs - rhs) <= 1e-11 * (np.linalg.norm(y) * np.linalg.norm(F(x)) + 1e-300), (F, lhs, rhs)
    # the stepper's own slab maps agree with the composed ones
    sig = rng.normal(size=sym_tr)
    sim.sig_tr = sig.copy()
    sim.v_tr = np.zeros(vel_tr)
    x = rng.normal(size=vel_st)
    st = sim.stress_update(x)
    ref = adj.trace_time(dz, st, dz.Npsi)
    assert np.abs(ref - adj.Cs_apply(dz, sig) - adj.Cx_apply(dz, x)).max() <= 1e-12 * np.abs(ref).max()
    # receivers
    sim.set_receivers(w.receivers)
    res = rng.normal(size=(len(w.receivers), d))
    v = rng.normal(size=vel_tr)
    sim.v_tr = v
    assert abs(np.sum(res * sim.receiver_values()) - np.sum(adj.receivers_T(sim, res) * v)) < 1e-12 * np.abs(res).sum()


@pytest.mark.parametrize("p,pg", [(1, 1), (2, 2), (3, 3), (2, 1)])
def test_slab_matrix_transpose_is_time_reversal(p, pg):
    w, _, _ = _tiny(p=p, pg=pg)
    sim = Simulation(w.xyz, w.elem_vert, w.period, w.lam, w.mu, w.rho, p, pg, "stdg", w.dt)
    dz = sim.disc
    ng, nphi = dz.Ng, dz.Nphi
    idx = np.arange(sim.A.shape[0]).reshape(-1, ng, nphi)
    perm = idx[:, ::-1, :].ravel()              # J: time node a -> N_gamma - 1 - a
    A = sim.A.toarray()
    JAJ = A[np.ix_(perm, perm)]
    assert np.abs(A.T - JAJ).max() <= 1e-12 * np.abs(A).max()
    if pg >= 1:
        assert np.abs(A.T - A).max() > 1e-6 * np.abs(A).max()   # A itself is not symmetric


def test_gradient_matches_central_differences():
    w, w_true, pg = _tiny()
    geom = _geom(w, pg)
    src = _sources(w)
    data = np.array([adj.forward(adj.make_sim(_geom(w_true, pg), w_true.lam, w_true.mu, w_true.rho), w.n_steps,
                                 s, w.f0, w.t_delay, w.a1, w.receivers)[0] for s in src])
    L, g_lam, g_mu, g_rho = adj.misfit_gradient(geom, w.lam, w.mu, w.rho, w.n_steps, src, w.f0, w.t_delay, w.a1,
                                                w.receivers, data)
    assert L > 0
    rng = np.random.default_rng(21)
    for name, g in (("lam", g_lam), ("mu", g_mu), ("rho", g_rho)):
        big = np.where(np.abs(g) >= 1e-3 * np.abs(g).max())[0]
        for e in rng.choice(big, 4, replace=False):
            base = {"lam": w.lam, "mu": w.mu, "rho": w.rho}
            fds = []
            for h in (1e-4 * base[name][e], 0.5e-4 * base[name][e]):
                Ls = []
                for sgn in (1.0, -1.0):
                    q = {k: v.copy() for k, v in base.items()}
                    q[name][e] += sgn * h
                    Ls.append(adj.misfit(geom, q["lam"], q["mu"], q["rho"], w.n_steps, src, w.f0, w.t_delay, w.a1,
                                         w.receivers, data))
                fds.append((Ls[0] - Ls[1]) / (2 * h))
            # Richardson: the O(h^2) term of the central difference cancels (the misfit of a small
            # model perturbation is strongly curved: at h_rel = 1e-4 that term alone is ~4e-6 relative)
            fd = (4.0 * fds[1] - fds[0]) / 3.0
            assert abs(fd - g[e]) <= 1e-6 * abs(g[e]) + 1e-9 * np.abs(g).max(), (name, e, fd, g[e])


def test_source_gradient_matches_differences_and_homogeneity():
    # dL/d(amplitude), dL/d(force direction), dL/d(position) of each shot's point source
    # (Sec. 6.3).  The source vector is linear in the amplitude and the direction, so the misfit
    # is quadratic in them and a central difference is exact up to rounding; the position enters
    # through phi(x_s) (Richardson-extrapolated differences, the source staying in its element).
    # Homogeneity: a1 dL/da1 = d . dL/dd.
    w, w_true, pg = _tiny()
    geom = _geom(w, pg)
    src = _sources(w)
    data = np.array([adj.forward(adj.make_sim(_geom(w_true, pg), w_true.lam, w_true.mu, w_true.rho), w.n_steps,
                                 s, w.f0, w.t_delay, w.a1, w.receivers)[0] for s in src])
    L, _, _, _, g_src = adj.misfit_gradient(geom, w.lam, w.mu, w.rho, w.n_steps, src, w.f0, w.t_delay, w.a1,
                                            w.receivers, data, source_grad=True)
    d = w.dim
    assert g_src.shape == (len(src), 1 + 2 * d)

    def Lk(k, xs, dr, a1):   # the misfit of shot k alone (the only term its source enters)
        return adj.misfit(geom, w.lam, w.mu, w.rho, w.n_steps, [(xs, dr)], w.f0, w.t_delay, a1, w.receivers,
                          data[k:k + 1])

    for k, (xs, dr) in enumerate(src):
        xs, dr = np.asarray(xs, float), np.asarray(dr, float)
        g = g_src[k]
        assert abs(w.a1 * g[0] - dr @ g[1:1 + d]) <= 1e-10 * (abs(w.a1 * g[0]) + 1e-300)
        h = 1e-3 * w.a1
        fd = (Lk(k, xs, dr, w.a1 + h) - Lk(k, xs, dr, w.a1 - h)) / (2 * h)
        assert abs(fd - g[0]) <= 1e-6 * abs(g[0]), ("a1", k, fd, g[0])
        for l in range(d):
            e = np.eye(d)[l] * 1e-3
            fd = (Lk(k, xs, dr + e, w.a1) - Lk(k, xs, dr - e, w.a1)) / 2e-3
            assert abs(fd - g[1 + l]) <= 1e-6 * np.abs(g[1:1 + d]).max(), ("dir", k, l, fd, g[1 + l])
            fds = []
            for hx in (2e-5, 1e-5):
                ex = np.eye(d)[l] * hx
                fds.append((Lk(k, xs + ex, dr, w.a1) - Lk(k, xs - ex, dr, w.a1)) / (2 * hx))
            fd = (4.0 * fds[1] - fds[0]) / 3.0
            assert abs(fd - g[1 + d + l]) <= 1e-5 * np.abs(g[1 + d:]).max(), ("x_s", k, l, fd, g[1 + d + l])
