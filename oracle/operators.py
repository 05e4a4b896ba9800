"""Discrete operators and the Schur velocity system (Sec. 4, Eqs. MD_2 - SD_1,
Eq. velocity.sys, Eq. velocity.sys.cn).

Definitions implemented (spatial factors; the space-time blocks are their tensor
products with the time-basis integrals, because every basis function is a product
phi(x) gamma(tau) and t = t^n + tau dt):
  Mbar_i[k,m]     = int_{T_i} phi_k phi_m                                  (Eq. MD_2)
  M_j[k,m]        = int_{R_j} psi_k psi_m                                  (Eq. MD_2)
  D_{i,j}[l][k,m] = int_{Gamma_j} phi_k psi_m (n_{i,j})_l - int_{T_{i,j}} d_l phi_k psi_m
                                                                           (Eq. MD_3)
  Q~_{i,j}[l][m,k]= int_{T_{i,j}} psi_m d_l phi_k - int_{Gamma_j} psi_m phi_k s_{i,j} (n_j)_l
                                                                           (Eq. qtilde)
  time factors    W = int gamma gamma, K = int gamma' gamma, T = gamma(1)gamma(1)^T - K
  space-time      D^st = kron(dt W, D), Q^st = kron(dt W, Q~), M^st = kron(T, M),
                  Mbar^st = kron(T, Mbar), M^- = kron(gamma(0), M)         (Eqs. MD_2_1 - MD_2_3)
The material on the dual mesh is E_j, constant per dual cell: the sub-cell
measure-weighted mean of the isotropic tensors of l(j) and r(j) (a reading; with E_j
constant only the constant coefficient of E_h in Eq. MD_6 survives, so Q_{i,j}
reduces to Q~_{i,j}).  rho_i is constant per element.  A free-surface boundary face
drops the face integrals (zero traction, no jump term).

The velocity system is assembled explicitly as a SciPy sparse matrix:
  A = blockdiag(rho_i Mbar^st_i (x) I_d) - c * sum_j D^st_{i,j} (M^st_j)^{-1} E_j . Q^st_{i',j}
with c = 1 (space-time DG, Eq. velocity.sys) or c = 1/4 (Crank-Nicolson, Eq.
velocity.sys.cn).  "E . Q v" contracts the full tensor: (E.G)_{ab} = E_{abkl} G_{kl},
G_{kl} = Q[l] v_k, and "D . sigma" is sum_l D[l] sigma_{kl}.
Layouts: velocity  [elem][component][time node][space node];
         stress    [face][component][time node][dual mode], components
         2D (xx, yy, xy), 3D (xx, yy, zz, xy, yz, xz).
Pins (tests/test_oracle_operators.py): Q~ = -D^T (Theorem 1 proof), symmetry and
positive definiteness of the Crank-Nicolson matrix by brute force (Theorems 1, 2),
zero momentum forcing by a constant stress, the linear-velocity patch test, and
invariance under element renumbering; for the paper's 2D tensor dual basis
(dual="quad"), tests/test_oracle_quad_dual.py.
"""
import numpy as np
import scipy.sparse as sp

from .basis import RefBasis, TimeBasis, monomial_exponents, monomials
from .quadrature import map_rule, ref_simplex_rule

SYM = {2: [(0, 0), (1, 1), (0, 1)], 3: [(0, 0), (1, 1), (2, 2), (0, 1), (1, 2), (0, 2)]}


def sym_index(dim):
    """(dim, dim) table: full-tensor entry (a, b) -> symmetric component index."""
    t = np.zeros((dim, dim), dtype=np.int64)
    for c, (a, b) in enumerate(SYM[dim]):
        t[a, b] = t[b, a] = c
    return t


def stiffness_tensor(lam, mu, dim):
    """Isotropic E_{abkl} = lam d_ab d_kl + mu (d_ak d_bl + d_al d_bk) (Eq. 1.1b)."""
    I = np.eye(dim)
    lam = np.asarray(lam)[..., None, None, None, None]
    mu = np.asarray(mu)[..., None, None, None, None]
    return (lam * np.einsum("ab,kl->abkl", I, I)
            + mu * (np.einsum("ak,bl->abkl", I, I) + np.einsum("al,bk->abkl", I, I)))


def compliance_apply(sig, lam, mu, dim):
    """E^{-1} : sigma for isotropic E (inverse of Eq. 1.1b; plane strain in 2D)."""
    tr = np.trace(sig, axis1=-2, axis2=-1)
    lam = np.asarray(lam)
    mu = np.asarray(mu)
    coef = lam / (dim * lam + 2.0 * mu)
    return (sig - (coef * tr)[..., None, None] * np.eye(dim)) / (2.0 * np.asarray(mu)[..., None, None])


def bilinear_inverse(P, x, iters=40):
    """Reference coordinates (u, v) in [0, 1]^2 of points x (..., q, 2) under the bilinear map
    F(u, v) = (1-u)(1-v) P0 + u(1-v) P1 + u v P2 + (1-u) v P3 of the quadrilaterals P (..., 4, 2),
    by Newton's method from the centre (the map is one-to-one on a convex quadrilateral)."""
    P0, P1, P2, P3 = (P[..., k, None, :] for k in range(4))
    a, b, c = P1 - P0, P3 - P0, P0 - P1 + P2 - P3          # F = P0 + u a + v b + u v c
    u = np.full(x.shape[:-1], 0.5)
    v = np.full(x.shape[:-1], 0.5)
    for _ in range(iters):
        r = P0 + u[..., None] * a + v[..., None] * b + (u * v)[..., None] * c - x
        Fu = a + v[..., None] * c
        Fv = b + u[..., None] * c
        det = Fu[..., 0] * Fv[..., 1] - Fu[..., 1] * Fv[..., 0]
        du = (r[..., 0] * Fv[..., 1] - r[..., 1] * Fv[..., 0]) / det
        dv = (Fu[..., 0] * r[..., 1] - Fu[..., 1] * r[..., 0]) / det
        u, v = u - du, v - dv
    r = P0 + u[..., None] * a + v[..., None] * b + (u * v)[..., None] * c - x
    scale = np.abs(P - P.mean(axis=-2, keepdims=True)).max()
    if np.abs(r).max() > 1e-12 * scale:
        raise ValueError("bilinear inverse did not converge (non-convex dual quadrilateral?)")
    return np.stack([u, v], axis=-1)


class Discretization:
    """Blocks of Sec. 4 on a DualMesh.  dual="taylor": the dual basis is the rescaled
    monomials of total degree <= p in physical space (the paper's 3D choice, used in 2D as
    well).  dual="quad" (2D, meshes without boundary faces): the paper's 2D choice of Sec. 3
    (paragraph on space-time basis functions), the (p+1)^2 tensor-product space on the unit
    square carried to the dual quadrilateral (b_l, face vertex 0, b_r, face vertex 1) by its
    bilinear map, spanned here by u^a v^b, 0 <= a, b <= p (the same space as the tensor
    nodal basis).  The discrete solution depends on the space only, not on the basis."""

    def __init__(self, mesh, p, p_gamma, lam, mu, rho, quad_n=None, dual="taylor"):
        d = self.dim = mesh.dim
        self.mesh, self.p, self.p_gamma = mesh, p, p_gamma
        self.lam_e = np.asarray(lam, dtype=np.float64)
        self.mu_e = np.asarray(mu, dtype=np.float64)
        self.rho = np.asarray(rho, dtype=np.float64)
        self.ref = RefBasis(d, p)
        self.dual = dual
        if dual == "taylor":
            self.exps = monomial_exponents(d, p)
        elif dual == "quad":
            if d != 2 or not mesh.interior.all():
                raise ValueError("the tensor dual basis needs a 2D mesh without boundary faces")
            self.exps = np.array([(a, b) for b in range(p + 1) for a in range(p + 1)], dtype=np.int64)
            # quadrilateral (b_l, n_0, b_r, n_1) of every dual cell, in the frame of l(j)
            self.quad = np.stack([mesh.bary[mesh.face_l], mesh.face_X[:, 0],
                                  mesh.bary[mesh.face_r] + mesh.shift, mesh.face_X[:, 1]], axis=1)
        else:
            raise ValueError("dual must be 'taylor' or 'quad'")
        self.Nphi, self.Npsi = self.ref.n, self.exps.shape[0]
        self.tb = TimeBasis(p_gamma)
        self.Ng = self.tb.n
        self.tm = self.tb.matrices()
        self.s = 3 if d == 2 else 6
        # the tensor basis has degree 2p in the reference square (rational in x on a
        # non-parallelogram cell): more points
        n = quad_n or (p + 3 if dual == "taylor" else 2 * p + 3)
        self.vol_rule = ref_simplex_rule(d, n)
        self.face_rule = ref_simplex_rule(d - 1, n)
        self._element_mass()
        self._pair_blocks()
        self._dual_material()

    # ---- basis evaluation -----------------------------------------------------------
    def phi(self, i, x):
        """Values (..., Nphi) and physical gradients (..., Nphi, d) of phi^(i) at x (i frame)."""
        m = self.mesh
        xi = np.einsum("...rd,...qd->...qr", m.Jinv[i], x - m.X[i, 0][..., None, :])
        val = self.ref.values(xi)
        g = self.ref.grads(xi)                                  # (..., q, k, r)
        grad = np.einsum("...qkr,...rl->...qkl", g, m.Jinv[i])
        return val, grad

    def psi(self, j, x_lframe):
        """Dual basis (..., Npsi) of face j at points given in the frame of l(j)."""
        m = self.mesh
        if self.dual == "quad":
            return monomials(bilinear_inverse(self.quad[j], x_lframe), self.exps)
        y = (x_lframe - m.xc[j][..., None, :]) / m.hj[j][..., None, None]
        return monomials(y, self.exps)

    # ---- spatial blocks -----------------------------------------------------------
    def _element_mass(self):
        m = self.mesh
        rp, rw = self.vol_rule
        pts, wts = map_rule(m.X, rp, rw)
        idx = np.arange(m.n_elem)
        val, _ = self.phi(idx, pts)
        self.Mbar = np.einsum("eq,eqk,eqm->ekm", wts, val, val)

    def _pair_blocks(self):
        m, d = self.mesh, self.dim
        nf = m.n_face
        self.D = np.zeros((nf, 2, d, self.Nphi, self.Npsi))
        self.Qt = np.zeros((nf, 2, d, self.Npsi, self.Nphi))
        self.Mdual = np.zeros((nf, self.Npsi, self.Npsi))
        rp, rw = self.vol_rule
        fp, fw = self.face_rule
        for side in (0, 1):
            faces = np.arange(nf) if side == 0 else np.where(m.interior)[0]
            if faces.size == 0:
                continue
            elems = m.face_l[faces] if side == 0 else m.face_r[faces]
            F = m.face_X[faces] - (m.shift[faces][:, None, :] if side == 1 else 0.0)
            sub = np.concatenate([F, m.bary[elems][:, None, :]], axis=1)   # T_{i,j}
            ps, ws = map_rule(sub, rp, rw)
            off = m.shift[faces][:, None, :] if side == 1 else 0.0
            psi_s = self.psi(faces, ps + off)
            phi_s, gphi_s = self.phi(elems, ps)
            pf, wf = map_rule(F, fp, fw)
            psi_f = self.psi(faces, pf + off)
            phi_f, _ = self.phi(elems, pf)
            sgn = 1.0 if side == 0 else -1.0
            nj = m.normal[faces]
            inter = m.interior[faces].astype(np.float64)
            face_term = np.einsum("fq,fqk,fqm->fkm", wf, phi_f, psi_f) * inter[:, None, None]
            vol_term = np.einsum("fq,fqkl,fqm->flkm", ws, gphi_s, psi_s)
            self.D[faces, side] = face_term[:, None] * (sgn * nj)[:, :, None, None] - vol_term
            vol_q = np.einsum("fq,fqm,fqkl->flmk", ws, psi_s, gphi_s)
            face_q = np.einsum("fq,fqm,fqk->fmk", wf, psi_f, phi_f) * inter[:, None, None]
            self.Qt[faces, side] = vol_q - face_q[:, None] * (sgn * nj)[:, :, None, None]
            self.Mdual[faces] += np.einsum("fq,fqk,fqm->fkm", ws, psi_s, psi_s)

    def _dual_material(self):
        m = self.mesh
        wl = m.sub_vol[m.face_l]
        wr = np.where(m.interior, m.sub_vol[np.maximum(m.face_r, 0)], 0.0)
        rl = np.maximum(m.face_r, 0)
        self.lam_f = (wl * self.lam_e[m.face_l] + wr * self.lam_e[rl]) / (wl + wr)
        self.mu_f = (wl * self.mu_e[m.face_l] + wr * self.mu_e[rl]) / (wl + wr)
        self.E = stiffness_tensor(self.lam_f, self.mu_f, self.dim)     # (nf, d, d, d, d)

    # ---- space-time blocks ----------------------------------------------------------
    def spacetime(self, dt, inverse="inv"):
        """Space-time blocks for step dt.  inverse="solve" forms (M^st_j)^{-1} by LU solves
        instead of explicit inversion: the same matrix up to rounding, used to measure the
        oracle's own rounding spread on ill-conditioned dual mass matrices."""
        tm = self.tm
        W, T, g0 = tm["W"], tm["T"], tm["g0"]
        self.dt = dt
        self.Dst = np.einsum("ab,fslkm->fslakbm", dt * W, self.D).reshape(
            self.D.shape[:3] + (self.Ng * self.Nphi, self.Ng * self.Npsi))
        self.Qst = np.einsum("ab,fslmk->fslambk", dt * W, self.Qt).reshape(
            self.Qt.shape[:3] + (self.Ng * self.Npsi, self.Ng * self.Nphi))
        Mst = np.einsum("ab,fkm->fakbm", T, self.Mdual).reshape(-1, self.Ng * self.Npsi, self.Ng * self.Npsi)
        if inverse == "solve":
            self.Mst_inv = np.linalg.solve(Mst, np.broadcast_to(np.eye(Mst.shape[1]), Mst.shape).copy())
        else:
            self.Mst_inv = np.linalg.inv(Mst)
        self.Mminus = np.einsum("a,fkm->fakm", g0, self.Mdual).reshape(-1, self.Ng * self.Npsi, self.Npsi)
        self.Mbar_st = np.einsum("ab,ekm->eakbm", T, self.Mbar).reshape(-1, self.Ng * self.Nphi, self.Ng * self.Nphi)
        self.Mbar_minus = np.einsum("a,ekm->eakm", g0, self.Mbar).reshape(-1, self.Ng * self.Nphi, self.Nphi)

    # ---- the Schur velocity system ---------------------------------------------------
    def vel_size(self):
        return self.mesh.n_elem * self.dim * self.Ng * self.Nphi

    def assemble(self, dt, scheme, inverse="inv"):
        """Sparse A of Eq. velocity.sys (scheme 'stdg') or Eq. velocity.sys.cn ('cn')."""
        self.spacetime(dt, inverse)
        c = 0.25 if scheme == "cn" else 1.0
        m, d = self.mesh, self.dim
        nb = self.Ng * self.Nphi
        rows, cols, vals = [], [], []
        # mass part rho_i Mbar^st_i for every component
        e, k, x, w = np.meshgrid(np.arange(m.n_elem), np.arange(d), np.arange(nb), np.arange(nb), indexing="ij")
        rows.append(((e * d + k) * nb + x).ravel())
        cols.append(((e * d + k) * nb + w).ravel())
        vals.append(np.broadcast_to((self.rho[:, None, None] * self.Mbar_st)[:, None], e.shape).ravel())
        # Schur part, chunked over faces
        nf = m.n_face
        chunk = max(1, 4000000 // (4 * d * d * nb * nb))
        for f0 in range(0, nf, chunk):
            f = np.arange(f0, min(nf, f0 + chunk))
            Dm = np.einsum("fslxy,fyz->fslxz", self.Dst[f], self.Mst_inv[f])
            DmQ = np.einsum("fslxz,ftnzw->fstlnxw", Dm, self.Qst[f])
            blk = -c * np.einsum("fklmn,fstlnxw->fskxtmw", self.E[f], DmQ)
            el = np.stack([m.face_l[f], m.face_r[f]], axis=1)
            for s in (0, 1):
                for t in (0, 1):
                    ok = (el[:, s] >= 0) & (el[:, t] >= 0)
                    if not ok.any():
                        continue
                    ff = np.where(ok)[0]
                    ei, ej = el[ff, s], el[ff, t]
                    _, kk, xx, mm, ww = np.meshgrid(ff, np.arange(d), np.arange(nb), np.arange(d), np.arange(nb),
                                                    indexing="ij")
                    rows.append(((ei[:, None, None, None, None] * d + kk) * nb + xx).ravel())
                    cols.append(((ej[:, None, None, None, None] * d + mm) * nb + ww).ravel())
                    vals.append(blk[ff, s, :, :, t, :, :].ravel())
        n = self.vel_size()
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
        return A.tocsr()

    # ---- pieces used by the stepper ------------------------------------------------
    def D_dot_sigma(self, sig_full_st):
        """sum_{j in S_i} sum_l D^st_{i,j}[l] sigma_j[k,l]  (sigma as (nf, d, d, Ng*Npsi))."""
        m, d = self.mesh, self.dim
        out = np.zeros((m.n_elem, d, self.Ng * self.Nphi))
        for s in (0, 1):
            el = m.face_l if s == 0 else m.face_r
            ok = el >= 0
            contrib = np.einsum("flxz,fklz->fkx", self.Dst[ok, s], sig_full_st[ok])
            np.add.at(out, el[ok], contrib)
        return out

    def E_dot_Q_v(self, v):
        """Per face: (E_j . sum_{i'} Q^st_{i',j} v_{i'})_{ab}, as full tensors (nf, d, d, Ng*Npsi)."""
        m = self.mesh
        nf = m.n_face
        G = np.zeros((nf, self.dim, self.dim, self.Ng * self.Npsi))   # G[k, l] = Q[l] v_k
        for s in (0, 1):
            el = m.face_l if s == 0 else m.face_r
            ok = el >= 0
            G[ok] += np.einsum("flzx,fkx->fklz", self.Qst[ok, s], v[el[ok]])
        return np.einsum("fabkl,fklz->fabz", self.E, G)

    def full_from_sym(self, sig):
        t = sym_index(self.dim)
        return sig[:, t, ...]

    def sym_from_full(self, full):
        return np.stack([full[:, a, b] for (a, b) in SYM[self.dim]], axis=1)
