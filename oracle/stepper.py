"""Time stepping with direct solves (Sec. 4; Sec. 6.3 for the point source).

Space-time DG (p_gamma >= 0, Eq. velocity.sys then Eq. NM26), per slab n -> n+1:
  b_i   = Mbar^-_i rho_i v_tr,i + sum_{j in S_i} D^st_{i,j} . (M^st_j)^{-1} (M^-_j sigma_tr,j) + (rho S)_i
  A v   = b                                                    (SuperLU, factored once per dt)
  sigma_j = (M^st_j)^{-1} (M^-_j sigma_tr,j + E_j . sum_{i'} Q^st_{i',j} v_{i'})   (no stress source)
  traces v_tr = sum_a gamma_a(1) v_a, sigma_tr likewise (the t^{n+1,-} values, Eq. NM13).
Crank-Nicolson (p_gamma = 0, Eq. velocity.sys.cn then Eq. NM26.cn):
  b     = rho Mbar v^n + sum D . sigma^n + 1/4 sum D . M^{-1} E . Q v^n + (rho S)
  sigma^{n+1} = sigma^n + M^{-1} E . Q v^{n+1/2},  v^{n+1/2} = (v^n + v^{n+1}) / 2.
Energy (Eq. SP3F / eq. stsum5): 1/2 sum_i rho_i int v_tr^2 + 1/2 sum_j int sigma_tr : E_j^{-1} sigma_tr.
Point source (Sec. 6.3): (rho S)_{i,k,a,n} = d_k phi_n(x_s) dt int_0^1 gamma_a(tau) S(t^n + tau dt) dtau,
with the Ricker wavelet read as S(t) = a1 (0.5 + a2 (t - t_D)^2) exp(a2 (t - t_D)^2),
a2 = -(pi f0)^2 (the printed formula lacks the exponential), the slab integral by
8-point Gauss-Legendre.  Receivers record v_h(x_r, t^{n+1,-}).
Pins (tests/test_oracle_stepper.py): exact energy preservation for CN (Theorem 5),
energy decrease equal to the time-jump terms of eq. stsum4 for space-time DG
(Theorem 4), the plane-wave exact solution and its convergence order (Sec. 6.2),
linearity and superposition of sources.
"""
import numpy as np
import scipy.sparse.linalg as spla

from .basis import gauss_legendre01
from .mesh import DualMesh
from .operators import Discretization, compliance_apply, SYM
from .quadrature import map_rule, ref_simplex_rule


def ricker(t, f0, t_delay, a1):
    a2 = -(np.pi * f0) ** 2
    tau = t - t_delay
    return a1 * (0.5 + a2 * tau * tau) * np.exp(a2 * tau * tau)


def plane_wave_fields(x, t, kind, n, pol, amp, lam, mu, rho):
    """Exact plane P (kind 0) or S (kind 1) wave, Eqs. NT2.1 / NT2.2 with the unit normal.

    U = amp * r * sin(k . x - c |k| t), k = 2 pi n; P: v = -c_p nh, sigma = lam I + 2 mu nh nh^T;
    S: v = -c_s e, sigma = mu (nh e^T + e nh^T), e = pol (2D default (-n_y, n_x)).
    Returns v (..., d) and the full stress (..., d, d).
    """
    n = np.asarray(n, dtype=np.float64)
    d = n.size
    nh = n / np.linalg.norm(n)
    k = 2 * np.pi * n
    if kind == 0:
        c = np.sqrt((lam + 2 * mu) / rho)
        rv = -c * nh
        rs = lam * np.eye(d) + 2 * mu * np.outer(nh, nh)
    else:
        c = np.sqrt(mu / rho)
        e = np.array([-nh[1], nh[0]]) if pol is None else np.asarray(pol, dtype=np.float64)
        e = e / np.linalg.norm(e)
        rv = -c * e
        rs = mu * (np.outer(nh, e) + np.outer(e, nh))
    ph = np.sin(x @ k - c * np.linalg.norm(k) * t)
    return amp * ph[..., None] * rv, amp * ph[..., None, None] * rs


class Simulation:
    """One mesh, one medium, n_shots right-hand sides; direct solves."""

    def __init__(self, xyz, elem_vert, period, lam, mu, rho, p, p_gamma, scheme, dt, dual="taylor"):
        if scheme == "cn" and p_gamma != 0:
            raise ValueError("Crank-Nicolson needs p_gamma = 0")
        self.mesh = DualMesh(xyz, elem_vert, period)
        self.disc = Discretization(self.mesh, p, p_gamma, lam, mu, rho, dual=dual)
        self.scheme, self.dt = scheme, dt
        self.A = self.disc.assemble(dt, scheme)
        self._lu = None
        self.t = 0.0
        self.step_index = 0
        dz = self.disc
        self.v_tr = np.zeros((self.mesh.n_elem, dz.dim, dz.Nphi))
        self.sig_tr = np.zeros((self.mesh.n_face, dz.s, dz.Npsi))
        self.sources = None
        self.receivers = None
        self.records = []

    @classmethod
    def from_workload(cls, w, dt=None):
        return cls(w.xyz, w.elem_vert, w.period, w.lam, w.mu, w.rho, w.p, w.p_gamma, w.scheme,
                   w.dt if dt is None else dt)

    @property
    def lu(self):
        if self._lu is None:
            self._lu = spla.splu(self.A.tocsc())
        return self._lu

    # ---- initial data --------------------------------------------------------------
    def set_plane_wave(self, kind, n, pol, amp, t=0.0, quad_n=None):
        """L2 projections of the exact plane wave onto the velocity and dual bases."""
        m, dz = self.mesh, self.disc
        d = dz.dim
        qn = quad_n or (2 * dz.p + 8)
        rp, rw = ref_simplex_rule(d, qn)
        pts, wts = map_rule(m.X, rp, rw)
        lam0, mu0, rho0 = dz.lam_e[0], dz.mu_e[0], dz.rho[0]
        v, _ = plane_wave_fields(pts, t, kind, n, pol, amp, lam0, mu0, rho0)
        val, _ = dz.phi(np.arange(m.n_elem), pts)
        rhs = np.einsum("eq,eqk,eqc->eck", wts, val, v)
        self.v_tr = np.linalg.solve(dz.Mbar[:, None], rhs[..., None])[..., 0]
        rhs_s = np.zeros((m.n_face, d, d, dz.Npsi))
        for side in (0, 1):
            faces = np.arange(m.n_face) if side == 0 else np.where(m.interior)[0]
            if faces.size == 0:
                continue
            elems = m.face_l[faces] if side == 0 else m.face_r[faces]
            F = m.face_X[faces] - (m.shift[faces][:, None, :] if side == 1 else 0.0)
            sub = np.concatenate([F, m.bary[elems][:, None, :]], axis=1)
            ps, ws = map_rule(sub, rp, rw)
            off = m.shift[faces][:, None, :] if side == 1 else 0.0
            psi = dz.psi(faces, ps + off)
            _, s = plane_wave_fields(ps, t, kind, n, pol, amp, lam0, mu0, rho0)
            rhs_s[faces] += np.einsum("fq,fqm,fqab->fabm", ws, psi, s)
        full = np.linalg.solve(dz.Mdual[:, None, None], rhs_s[..., None])[..., 0]
        self.sig_tr = dz.sym_from_full(full)
        self.t = t

    def set_state(self, v_tr, sig_tr):
        self.v_tr = np.array(v_tr, dtype=np.float64).reshape(self.v_tr.shape)
        self.sig_tr = np.array(sig_tr, dtype=np.float64).reshape(self.sig_tr.shape)

    # ---- sources / receivers --------------------------------------------------------
    def set_source(self, xs, direction, f0, t_delay, a1):
        i, y = self.mesh.locate(xs)
        phi, _ = self.disc.phi(np.array([i]), y[None, None, :])
        self.sources = dict(elem=i, phi=phi[0, 0], dir=np.asarray(direction, dtype=np.float64),
                            f0=f0, t_delay=t_delay, a1=a1, x_local=y)

    def source_vector(self, t0):
        """(rho S)_i for the slab [t0, t0 + dt]; zero except in the source element."""
        dz = self.disc
        out = np.zeros((self.mesh.n_elem, dz.dim, dz.Ng, dz.Nphi))
        if self.sources is None:
            return out.reshape(self.mesh.n_elem, dz.dim, -1)
        s = self.sources
        xq, wq = gauss_legendre01(8)
        g = dz.tb.values(xq)                                  # (8, Ng)
        St = ricker(t0 + xq * self.dt, s["f0"], s["t_delay"], s["a1"])
        tint = self.dt * np.einsum("q,qa,q->a", wq, g, St)    # dt int gamma_a S
        out[s["elem"]] = np.einsum("k,a,n->kan", s["dir"], tint, s["phi"])
        return out.reshape(self.mesh.n_elem, dz.dim, -1)

    def set_receivers(self, xr):
        self.receivers = []
        for x in np.atleast_2d(xr):
            i, y = self.mesh.locate(x)
            phi, _ = self.disc.phi(np.array([i]), y[None, None, :])
            self.receivers.append((i, phi[0, 0]))

    def receiver_values(self):
        return np.array([[self.v_tr[i, k] @ ph for k in range(self.disc.dim)] for (i, ph) in self.receivers])

    # ---- one slab --------------------------------------------------------------------
    def rhs(self):
        dz, m = self.disc, self.mesh
        ne = m.n_elem
        src = self.source_vector(self.t)
        if self.scheme == "cn":
            v = self.v_tr
            mass = self.disc.rho[:, None, None] * np.einsum("ekm,ecm->eck", dz.Mbar, v)
            sig_full = dz.full_from_sym(self.sig_tr)
            ds = dz.D_dot_sigma(sig_full)
            schur = self._D_Minv(dz.E_dot_Q_v(v))
            return (mass + ds + 0.25 * schur + src).reshape(-1)
        mass = dz.rho[:, None, None] * np.einsum("exm,ecm->ecx", dz.Mbar_minus, self.v_tr)
        sig_full = dz.full_from_sym(self.sig_tr)                        # (nf, d, d, Npsi)
        carried = np.einsum("fzm,fabm->fabz", dz.Mminus, sig_full)       # M^-_j sigma_tr,j
        carried = np.einsum("fyz,fabz->faby", dz.Mst_inv, carried)
        ds = dz.D_dot_sigma(carried)
        return (mass + ds + src).reshape(ne * dz.dim * dz.Ng * dz.Nphi)

    def _D_Minv(self, full):
        dz = self.disc
        return dz.D_dot_sigma(np.einsum("fyz,fabz->faby", dz.Mst_inv, full))

    def stress_update(self, v_new):
        dz = self.disc
        eq = dz.E_dot_Q_v(v_new)                                        # (nf, d, d, Ng*Npsi)
        if self.scheme == "cn":
            eqh = 0.5 * (eq + dz.E_dot_Q_v(self.v_tr))
            inc = np.einsum("fyz,fabz->faby", dz.Mst_inv, eqh)
            return self.sig_tr + dz.sym_from_full(inc)
        sig_full = dz.full_from_sym(self.sig_tr)
        carried = np.einsum("fzm,fabm->fabz", dz.Mminus, sig_full)
        sig = np.einsum("fyz,fabz->faby", dz.Mst_inv, carried + eq)
        return dz.sym_from_full(sig)                                    # (nf, s, Ng*Npsi)

    def step(self, n_steps=1):
        dz = self.disc
        g1 = dz.tm["g1"]
        for _ in range(n_steps):
            b = self.rhs()
            v = self.lu.solve(b).reshape(self.mesh.n_elem, dz.dim, dz.Ng * dz.Nphi)
            sig = self.stress_update(v)
            self.last_v, self.last_sig = v, sig
            self.v_start = np.einsum("a,ecam->ecm", dz.tm["g0"], v.reshape(v.shape[0], dz.dim, dz.Ng, dz.Nphi))
            self.sig_start = np.einsum("a,fcam->fcm", dz.tm["g0"],
                                       sig.reshape(sig.shape[0], dz.s, dz.Ng, dz.Npsi))
            self.v_prev, self.sig_prev = self.v_tr, self.sig_tr
            self.v_tr = np.einsum("a,ecam->ecm", g1, v.reshape(v.shape[0], dz.dim, dz.Ng, dz.Nphi))
            self.sig_tr = np.einsum("a,fcam->fcm", g1, sig.reshape(sig.shape[0], dz.s, dz.Ng, dz.Npsi))
            self.t += self.dt
            self.step_index += 1
            if self.receivers is not None:
                self.records.append(self.receiver_values())

    # ---- energy -----------------------------------------------------------------------
    def energy(self, v_tr=None, sig_tr=None):
        dz = self.disc
        v = self.v_tr if v_tr is None else v_tr
        s = self.sig_tr if sig_tr is None else sig_tr
        kin = 0.5 * np.einsum("e,eck,ekm,ecm->", dz.rho, v, dz.Mbar, v)
        full = dz.full_from_sym(s)                                       # (nf, d, d, Npsi)
        eps = compliance_apply(np.moveaxis(full, -1, 1), dz.lam_f[:, None], dz.mu_f[:, None], dz.dim)
        eps = np.moveaxis(eps, 1, -1)
        ela = 0.5 * np.einsum("fabk,fkm,fabm->", full, dz.Mdual, eps)
        return kin + ela

    def jump_dissipation(self):
        """Time-jump terms of eq. stsum4 for the last slab (space-time DG)."""
        return self.energy(self.v_start - self.v_prev, self.sig_start - self.sig_prev)

    def apply_A(self, x):
        return self.A @ x
