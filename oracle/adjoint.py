"""Receiver misfit and its exact gradient with respect to per-element lambda, mu, rho and the
point sources (amplitude, force direction, position of each shot's source).

TEST INFRASTRUCTURE ONLY (see the package header).

The paper has no adjoint; this module differentiates the oracle's own discrete forward
map (space-time DG, Eq. velocity.sys then Eq. NM26, one Simulation per material):

  b^n      = Bv v^n + Bs sigma^n + s^n          Bv = rho Mbar^-,   Bs = D . (M^st)^{-1} M^- full(.)
  x^{n+1}  = A^{-1} b^n
  sigma^{n+1} = Cs sigma^n + Cx x^{n+1}         traced: gamma(1)^T sym((M^st)^{-1}(M^- full(sigma) + E . Q x))
  v^{n+1}  = Gam x^{n+1}                        Gam = gamma(1)^T (x) I
  L        = 1/2 sum_shots sum_{n=1..N} sum_r |R v^n - d^n|^2

Backward recursion (a_v, a_s = dL/dv^n, dL/dsigma^n through all later slabs):
  a_x = Gam^T a_v^{n+1} + Cx^T a_s^{n+1};   A^T lam = a_x  (the same LU, trans='T')
  a_v^n = Bv^T lam + R^T (R v^n - d^n),     a_s^n = Bs^T lam + Cs^T a_s^{n+1}
  dL/dtheta += lam^T dBv/dtheta v^n - lam^T dA/dtheta x^{n+1} + a_s^{n+1 T} dCx/dtheta x^{n+1}.
The point source enters the right-hand side only (Sec. 6.3): dL/dtheta_src += lam^T ds^n/dtheta_src,
s^n linear in the amplitude and the force direction, polynomial in the position through phi(x_s).
rho enters A and Bv through the element mass; lambda and mu enter A and Cx through E_j,
which is linear in the dual-cell values (lambda_j, mu_j) = sub-cell-weighted means of the
two elements' values (the dual-material reading).  Every transpose below is written out
from its forward map and pinned by a dot-product test; the gradient is pinned by central
finite differences with direct solves (tests/test_oracle_adjoint.py).
"""
import numpy as np

from .basis import gauss_legendre01
from .operators import SYM, stiffness_tensor
from .stepper import Simulation, ricker


# ---- transposes of the stepper's pieces (each checked by a dot-product test) -------------
def D_dot_sigma_T(dz, u):
    """Transpose of Discretization.D_dot_sigma: velocity (ne, d, Ng*Nphi) -> (nf, d, d, Ng*Npsi)."""
    m, d = dz.mesh, dz.dim
    out = np.zeros((m.n_face, d, d, dz.Ng * dz.Npsi))
    for s in (0, 1):
        el = m.face_l if s == 0 else m.face_r
        ok = el >= 0
        out[ok] += np.einsum("flxz,fkx->fklz", dz.Dst[ok, s], u[el[ok]])
    return out


def Q_gather(dz, v):
    """G[f, k, l] = sum_sides Q^st[l] v_k: the velocity-to-tensor map inside E_dot_Q_v."""
    m = dz.mesh
    G = np.zeros((m.n_face, dz.dim, dz.dim, dz.Ng * dz.Npsi))
    for s in (0, 1):
        el = m.face_l if s == 0 else m.face_r
        ok = el >= 0
        G[ok] += np.einsum("flzx,fkx->fklz", dz.Qst[ok, s], v[el[ok]])
    return G


def Q_gather_T(dz, G):
    """Transpose of Q_gather: (nf, d, d, Ng*Npsi) -> velocity (ne, d, Ng*Nphi)."""
    m = dz.mesh
    out = np.zeros((m.n_elem, dz.dim, dz.Ng * dz.Nphi))
    for s in (0, 1):
        el = m.face_l if s == 0 else m.face_r
        ok = el >= 0
        np.add.at(out, el[ok], np.einsum("flzx,fklz->fkx", dz.Qst[ok, s], G[ok]))
    return out


def E_contract(E, G):
    return np.einsum("fabkl,fklz->fabz", E, G)


def E_contract_T(E, Y):
    return np.einsum("fabkl,fabz->fklz", E, Y)


def full_from_sym_T(dz, full):
    """Transpose of full_from_sym: (nf, d, d, .) -> (nf, s, .), both mirror entries summed."""
    out = np.zeros((full.shape[0], dz.s) + full.shape[3:])
    for c, (a, b) in enumerate(SYM[dz.dim]):
        out[:, c] += full[:, a, b]
        if a != b:
            out[:, c] += full[:, b, a]
    return out


def sym_from_full_T(dz, sym):
    """Transpose of sym_from_full: (nf, s, .) -> (nf, d, d, .), the listed (a, b) entry only."""
    out = np.zeros((sym.shape[0], dz.dim, dz.dim) + sym.shape[2:])
    for c, (a, b) in enumerate(SYM[dz.dim]):
        out[:, a, b] += sym[:, c]
    return out


def minv(dz, Y):        # (M^st)^{-1} per face
    return np.einsum("fyz,fabz->faby", dz.Mst_inv, Y)


def minv_T(dz, Y):
    return np.einsum("fzy,fabz->faby", dz.Mst_inv, Y)


def mminus(dz, S):      # M^- : (nf, d, d, Npsi) -> (nf, d, d, Ng*Npsi)
    return np.einsum("fzm,fabm->fabz", dz.Mminus, S)


def mminus_T(dz, Y):
    return np.einsum("fzm,fabz->fabm", dz.Mminus, Y)


def trace_time(dz, y, n):   # gamma(1)^T over the time index: (., c, Ng*n) -> (., c, n)
    return np.einsum("a,fcam->fcm", dz.tm["g1"], y.reshape(y.shape[0], y.shape[1], dz.Ng, n))


def trace_time_T(dz, t):
    return np.einsum("a,fcm->fcam", dz.tm["g1"], t).reshape(t.shape[0], t.shape[1], -1)


# ---- forward pieces written as the linear maps above --------------------------------------
def Bs_apply(dz, sig):
    return dz.D_dot_sigma(minv(dz, mminus(dz, dz.full_from_sym(sig))))


def Bs_T(dz, lam):
    return full_from_sym_T(dz, mminus_T(dz, minv_T(dz, D_dot_sigma_T(dz, lam))))


def Cs_apply(dz, sig):
    return trace_time(dz, dz.sym_from_full(minv(dz, mminus(dz, dz.full_from_sym(sig)))), dz.Npsi)


def Cs_T(dz, a):
    return full_from_sym_T(dz, mminus_T(dz, minv_T(dz, sym_from_full_T(dz, trace_time_T(dz, a)))))


def Cx_apply(dz, x, E=None):
    E = dz.E if E is None else E
    return trace_time(dz, dz.sym_from_full(minv(dz, E_contract(E, Q_gather(dz, x)))), dz.Npsi)


def Cx_T(dz, a):
    return Q_gather_T(dz, E_contract_T(dz.E, minv_T(dz, sym_from_full_T(dz, trace_time_T(dz, a)))))


def Bv_apply(dz, v):
    return dz.rho[:, None, None] * np.einsum("exm,ecm->ecx", dz.Mbar_minus, v)


def Bv_T(dz, lam):
    return dz.rho[:, None, None] * np.einsum("exm,ecx->ecm", dz.Mbar_minus, lam)


def receivers_T(sim, res):
    """R^T: (n_rec, d) residuals -> trace-shaped velocity (ne, d, Nphi)."""
    out = np.zeros_like(sim.v_tr)
    for (i, ph), rr in zip(sim.receivers, res):
        out[i] += rr[:, None] * ph[None, :]
    return out


# ---- misfit and gradient ---------------------------------------------------------------------
def make_sim(geom, lam, mu, rho):
    xyz, ev, per, p, pg, dt = geom
    return Simulation(xyz, ev, per, lam, mu, rho, p, pg, "stdg", dt)


def forward(sim, n_steps, source, f0, td, a1, receivers, keep=False):
    """One shot from the zero state: receiver records (n_steps, n_rec, d) and, with keep, the
    trace states v^n (n = 0..N-1) and slab solutions x^{n+1}."""
    dz = sim.disc
    sim.v_tr = np.zeros_like(sim.v_tr)
    sim.sig_tr = np.zeros_like(sim.sig_tr)
    sim.t, sim.step_index, sim.records = 0.0, 0, []
    sim.set_source(source[0], source[1], f0, td, a1)
    sim.set_receivers(receivers)
    V, X = [], []
    for _ in range(n_steps):
        if keep:
            V.append(sim.v_tr.copy())
        sim.step(1)
        if keep:
            X.append(sim.last_v.copy())
    return np.array(sim.records), V, X


def misfit(geom, lam, mu, rho, n_steps, sources, f0, td, a1, receivers, data):
    sim = make_sim(geom, lam, mu, rho)
    L = 0.0
    for s, src in enumerate(sources):
        rec, _, _ = forward(sim, n_steps, src, f0, td, a1, receivers)
        L += 0.5 * np.sum((rec - data[s]) ** 2)
    return L


def source_derivatives(sim, t0):
    """Derivatives of the slab's point-source vector (Sec. 6.3: (rho S)_i = d phi(x_s) dt int gamma S)
    for the slab [t0, t0 + dt], each shaped like the vector (ne, d, Ng*Nphi): with respect to
    the amplitude a1 (the vector at unit amplitude), the force direction d_l and the position
    x_s,m (the element containing x_s held fixed)."""
    dz, s = sim.disc, sim.sources
    xq, wq = gauss_legendre01(8)
    g = dz.tb.values(xq)
    unit = sim.dt * np.einsum("q,qa,q->a", wq, g, ricker(t0 + xq * sim.dt, s["f0"], s["t_delay"], 1.0))
    _, grad = dz.phi(np.array([s["elem"]]), s["x_local"][None, None, :])
    dphi = grad[0, 0]                                                   # (Nphi, d)
    shape = (sim.mesh.n_elem, dz.dim, dz.Ng, dz.Nphi)
    d_a1 = np.zeros(shape)
    d_a1[s["elem"]] = np.einsum("k,a,n->kan", s["dir"], unit, s["phi"])
    d_dir, d_xs = [], []
    for l in range(dz.dim):
        u = np.zeros(shape)
        u[s["elem"], l] = s["a1"] * np.einsum("a,n->an", unit, s["phi"])
        d_dir.append(u.reshape(shape[0], dz.dim, -1))
        u = np.zeros(shape)
        u[s["elem"]] = s["a1"] * np.einsum("k,a,n->kan", s["dir"], unit, dphi[:, l])
        d_xs.append(u.reshape(shape[0], dz.dim, -1))
    return d_a1.reshape(shape[0], dz.dim, -1), d_dir, d_xs


def misfit_gradient(geom, lam, mu, rho, n_steps, sources, f0, td, a1, receivers, data, source_grad=False):
    """(L, dL/dlambda, dL/dmu, dL/drho) per element, summed over the shots; with source_grad
    also dL/d(source) per shot, (n_shots, 1 + 2 d): the shot's amplitude a1, its force
    direction and its position, from lam^T ds^n/dtheta (the source enters b^n only)."""
    sim = make_sim(geom, lam, mu, rho)
    dz, m = sim.disc, sim.mesh
    d, ne = dz.dim, m.n_elem
    c = 1.0
    E1 = stiffness_tensor(np.ones(m.n_face), np.zeros(m.n_face), d)
    E2 = stiffness_tensor(np.zeros(m.n_face), np.ones(m.n_face), d)
    g_rho = np.zeros(ne)
    g_lf = np.zeros(m.n_face)
    g_mf = np.zeros(m.n_face)
    L = 0.0
    g_src = np.zeros((len(sources), 1 + 2 * d))
    for s, src in enumerate(sources):
        rec, V, X = forward(sim, n_steps, src, f0, td, a1, receivers, keep=True)
        res = rec - data[s]
        L += 0.5 * np.sum(res ** 2)
        a_v = receivers_T(sim, res[n_steps - 1])
        a_s = np.zeros_like(sim.sig_tr)
        for n in range(n_steps - 1, -1, -1):
            x, v = X[n], V[n]
            a_x = trace_time_T(dz, a_v) + Cx_T(dz, a_s)
            lam_ = sim.lu.solve(a_x.ravel(), trans="T").reshape(x.shape)
            # rho: lam^T (dBv/drho) v - lam^T (dA/drho) x
            g_rho += np.einsum("ecx,exm,ecm->e", lam_, dz.Mbar_minus, v)
            g_rho -= np.einsum("ecx,exy,ecy->e", lam_, dz.Mbar_st, x)
            # lambda_j, mu_j: -lam^T (dA/dtheta) x + a_s^T (dCx/dtheta) x, A_face = -c D.(M^st)^{-1} E.Q
            DTl = D_dot_sigma_T(dz, lam_)
            G = Q_gather(dz, x)
            for Ek, gk in ((E1, g_lf), (E2, g_mf)):
                h = minv(dz, E_contract(Ek, G))
                gk += c * np.einsum("fabz,fabz->f", DTl, h)
                gk += np.einsum("fcm,fcm->f", a_s, trace_time(dz, dz.sym_from_full(h), dz.Npsi))
            if source_grad:   # b^n = ... + s^n: dL/dtheta += lam^T ds^n/dtheta
                d_a1, d_dir, d_xs = source_derivatives(sim, n * sim.dt)
                g_src[s, 0] += np.sum(lam_ * d_a1)
                for l in range(d):
                    g_src[s, 1 + l] += np.sum(lam_ * d_dir[l])
                    g_src[s, 1 + d + l] += np.sum(lam_ * d_xs[l])
            a_s = Bs_T(dz, lam_) + Cs_T(dz, a_s)
            a_v = Bv_T(dz, lam_)
            if n >= 1:
                a_v = a_v + receivers_T(sim, res[n - 1])
    # dual-cell values -> elements: lambda_j = (w_l lambda_l + w_r lambda_r) / (w_l + w_r)
    wl = m.sub_vol[m.face_l]
    wr = np.where(m.interior, m.sub_vol[np.maximum(m.face_r, 0)], 0.0)
    g_lam = np.zeros(ne)
    g_mu = np.zeros(ne)
    for side, w in ((m.face_l, wl), (m.face_r, wr)):
        ok = side >= 0
        np.add.at(g_lam, side[ok], (w / (wl + wr) * g_lf)[ok])
        np.add.at(g_mu, side[ok], (w / (wl + wr) * g_mf)[ok])
    if source_grad:
        return L, g_lam, g_mu, g_rho, g_src
    return L, g_lam, g_mu, g_rho
