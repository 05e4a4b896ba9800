"""Rows of the Schur velocity operator in extended precision (test infrastructure).

Why: with the Taylor dual basis, a dual cell next to a sliver element has a dual mass
matrix M_j of condition number ~5e8 at p = 3, and the FP64 oracle's (M^st_j)^{-1} then
carries rounding errors that move A x by ~1e-10 relative -- as much as the bar the GPU is
held to.  This module evaluates (A x)_i for chosen elements i with every step in
np.longdouble: on aarch64 Linux that is IEEE binary128 (113-bit significand, eps 1.9e-34),
on x86-64 Linux the x87 80-bit format (64-bit significand, eps 1.1e-19).  No LAPACK call is
involved (LAPACK has no extended type): Gauss-Legendre nodes by Newton's method on the
Legendre recurrence, inverses and solves by Gauss-Jordan elimination with partial pivoting.

What is computed is the oracle's definition of A (oracle/operators.py), restated term by
term for the faces of element i:
  (A x)_i = rho_i (T (x) Mbar_i) x_i
            - c sum_{j in S_i} sum_l D^st_{i,j}[l] (M^st_j)^{-1} sigma_j[k, l],
  sigma_j[k, l] = sum_{m,n} E_j[k,l,m,n] G_j[m,n],  G_j[m,n] = sum_{i' in {l(j), r(j)}} Q~^st_{i',j}[n] x_{i',m},
with D_{i,j} (Eq. MD_3), Q~_{i,j} from its own integrals (Eq. qtilde), M_j (Eq. MD_2), the time
factors W, T, the space-time blocks D^st = dt W (x) D, Q~^st = dt W (x) Q~, M^st = T (x) M_j
(Eqs. MD_2_1 - MD_2_3), c = 1 (Eq. velocity.sys) or 1/4 (Eq. velocity.sys.cn), and the same
readings as the FP64 oracle: l(j) the smaller element index, n_j from l(j) to r(j), sub-cells
T_{i,j} = simplex(face vertices, barycentre of T_i), the Taylor dual basis
((x - x_j)/h_j)^a with x_j the measure-weighted centroid of R_j and h_j its largest vertex
distance, E_j the sub-cell-weighted mean of the two elements' isotropic tensors, free
surface on boundary faces (no face integrals).  Meshes without periodic faces only.

Pins (tests/test_oracle_extended.py): Q~ = -D^T (Theorem 1 proof) to extended-precision
rounding; agreement with the FP64 oracle's assembled A on well-conditioned meshes; two exact
quadrature orders agreeing to ~1e-15 on the sliver construction where the FP64 oracle's two
orders differ by ~1e-10; the Crank-Nicolson matrix built from these rows symmetric to
extended-precision rounding (Theorem 1).

Test infrastructure: only tests/ import this module; the library never calls it.
"""
import numpy as np

from .basis import monomial_exponents

LD = np.longdouble


def eps():
    return float(np.finfo(LD).eps)


# ---- dense linear algebra in extended precision ---------------------------------------------
def solve(A, B):
    """A^{-1} B by Gauss-Jordan elimination with partial pivoting (A square, B matrix)."""
    A = np.array(A, dtype=LD)
    B = np.array(B, dtype=LD)
    vec = B.ndim == 1
    if vec:
        B = B[:, None]
    n = A.shape[0]
    M = np.concatenate([A, B], axis=1)
    for c in range(n):
        p = c + int(np.argmax(np.abs(M[c:, c])))
        if M[p, c] == 0:
            raise ValueError("singular matrix")
        if p != c:
            M[[c, p]] = M[[p, c]]
        M[c] = M[c] / M[c, c]
        f = M[:, c].copy()
        f[c] = 0
        M -= f[:, None] * M[c][None, :]
    X = M[:, n:]
    return X[:, 0] if vec else X


def inv(A):
    return solve(A, np.eye(np.asarray(A).shape[0], dtype=LD))


# ---- quadrature ---------------------------------------------------------------------------
def gauss_legendre01(n):
    """n-point Gauss-Legendre rule on [0, 1] in extended precision: Newton's method on the
    three-term Legendre recurrence, started from the FP64 nodes."""
    x = np.polynomial.legendre.leggauss(n)[0].astype(LD)

    def legendre(x):
        p0, p1 = np.ones_like(x), x.copy()
        for k in range(2, n + 1):
            p0, p1 = p1, ((2 * k - 1) * x * p1 - (k - 1) * p0) / k
        if n == 1:
            p0 = np.ones_like(x)
        dp = n * (x * p1 - p0) / (x * x - 1)
        return p1, dp

    for _ in range(8):
        pn, dp = legendre(x)
        x = x - pn / dp
    _, dp = legendre(x)
    w = 2 / ((1 - x * x) * dp * dp)
    return (x + 1) / 2, w / 2


def simplex_rule(dim, n):
    """Collapsed-coordinate rule on the unit reference simplex (weights sum to 1/dim!)."""
    x, w = gauss_legendre01(n)
    if dim == 1:
        return x[:, None], w
    if dim == 2:
        u, v = np.meshgrid(x, x, indexing="ij")
        wu, wv = np.meshgrid(w, w, indexing="ij")
        pts = np.stack([u.ravel(), (v * (1 - u)).ravel()], axis=1)
        return pts, (wu * wv * (1 - u)).ravel()
    u, v, s = np.meshgrid(x, x, x, indexing="ij")
    wu, wv, ws = np.meshgrid(w, w, w, indexing="ij")
    pts = np.stack([u.ravel(), (v * (1 - u)).ravel(), (s * (1 - u) * (1 - v)).ravel()], axis=1)
    return pts, (wu * wv * ws * (1 - u) ** 2 * (1 - v)).ravel()


def _det(E):
    if E.shape[0] == 1:
        return E[0, 0]
    if E.shape[0] == 2:
        return E[0, 0] * E[1, 1] - E[0, 1] * E[1, 0]
    return (E[0, 0] * (E[1, 1] * E[2, 2] - E[1, 2] * E[2, 1]) - E[0, 1] * (E[1, 0] * E[2, 2] - E[1, 2] * E[2, 0])
            + E[0, 2] * (E[1, 0] * E[2, 1] - E[1, 1] * E[2, 0]))


def map_rule(V, rule):
    """Rule on the simplex with vertices V (k+1, D): physical points (Q, D), weights (Q,)."""
    rp, rw = rule
    E = V[1:] - V[:1]                                  # (k, D)
    k = E.shape[0]
    pts = V[0][None, :] + rp @ E
    G = E @ E.T
    meas = np.sqrt(abs(_det(G)))                       # k! times the k-measure
    return pts, rw * meas


# ---- bases ------------------------------------------------------------------------------
def monomials(y, exps):
    out = np.ones(y.shape[:-1] + (exps.shape[0],), dtype=LD)
    for a in range(exps.shape[1]):
        out = out * y[..., a:a + 1] ** exps[:, a]
    return out


def monomial_grads(y, exps):
    g = np.zeros(y.shape[:-1] + exps.shape, dtype=LD)
    for r in range(exps.shape[1]):
        term = np.ones(y.shape[:-1] + (exps.shape[0],), dtype=LD)
        for a in range(exps.shape[1]):
            e = exps[:, a]
            term = term * (e * y[..., a:a + 1] ** np.maximum(e - 1, 0) if a == r else y[..., a:a + 1] ** e)
        g[..., r] = term
    return g


class Basis:
    """Nodal P_p on the reference simplex (equispaced nodes, z outer, y, x fastest), the
    Lagrange time basis on the Gauss-Legendre points of [0, 1], and its time matrices."""

    def __init__(self, dim, p, p_gamma):
        self.dim, self.p = dim, p
        self.exps = monomial_exponents(dim, p)
        nodes = []
        rng = range(p + 1)
        if dim == 2:
            nodes = [(LD(i) / p, LD(j) / p) for j in rng for i in range(p + 1 - j)]
        else:
            nodes = [(LD(i) / p, LD(j) / p, LD(k) / p) for k in rng for j in range(p + 1 - k) for i in range(p + 1 - j - k)]
        self.coef = inv(monomials(np.array(nodes, dtype=LD), self.exps))    # phi_k = sum_a coef[a, k] xi^a
        self.N = len(nodes)
        self.Ng = p_gamma + 1
        self.tn, _ = gauss_legendre01(self.Ng)
        xq, wq = gauss_legendre01(self.Ng + 2)
        G, dG = self.gamma(xq), self.dgamma(xq)
        self.W = np.einsum("q,qk,qm->km", wq, G, G)
        self.K = np.einsum("q,qk,qm->km", wq, dG, G)
        g1 = self.gamma(np.array([LD(1)]))[0]
        self.T = np.outer(g1, g1) - self.K

    def gamma(self, t):
        out = np.ones((t.size, self.Ng), dtype=LD)
        for k in range(self.Ng):
            for m in range(self.Ng):
                if m != k:
                    out[:, k] *= (t - self.tn[m]) / (self.tn[k] - self.tn[m])
        return out

    def dgamma(self, t):
        out = np.zeros((t.size, self.Ng), dtype=LD)
        for k in range(self.Ng):
            for q in range(self.Ng):
                if q == k:
                    continue
                term = np.full(t.size, 1 / (self.tn[k] - self.tn[q]), dtype=LD)
                for m in range(self.Ng):
                    if m != k and m != q:
                        term = term * (t - self.tn[m]) / (self.tn[k] - self.tn[m])
                out[:, k] += term
        return out

    def phi(self, X, x):
        """Values (Q, N) and physical gradients (Q, N, d) of the element with vertices X."""
        J = (X[1:] - X[:1]).T
        Jinv = inv(J)
        xi = (x - X[0][None, :]) @ Jinv.T
        val = monomials(xi, self.exps) @ self.coef
        g = np.einsum("qar,ak->qkr", monomial_grads(xi, self.exps), self.coef)
        return val, np.einsum("qkr,rl->qkl", g, Jinv)


def stiffness(lam, mu, d):
    I = np.eye(d, dtype=LD)
    return (lam * np.einsum("ab,kl->abkl", I, I)
            + mu * (np.einsum("ak,bl->abkl", I, I) + np.einsum("al,bk->abkl", I, I)))


class PatchOperator:
    """(A x)_i for chosen elements of a mesh without periodic faces, in extended precision."""

    def __init__(self, xyz, elem_vert, lam, mu, rho, p, p_gamma, scheme, dt, quad_n=None):
        self.xyz = np.asarray(xyz, dtype=np.float64).astype(LD)
        self.ev = np.asarray(elem_vert, dtype=np.int64)
        self.d = d = self.ev.shape[1] - 1
        self.lam = np.asarray(lam, dtype=np.float64).astype(LD)
        self.mu = np.asarray(mu, dtype=np.float64).astype(LD)
        self.rho = np.asarray(rho, dtype=np.float64).astype(LD)
        self.b = Basis(d, p, p_gamma)
        self.Npsi = self.b.N
        self.c = LD(0.25) if scheme == "cn" else LD(1)
        self.dt = LD(dt)
        n = quad_n or p + 3
        self.vol_rule = simplex_rule(d, n)
        self.face_rule = simplex_rule(d - 1, n)
        # faces by sorted vertex tuple: (element, local face) pairs
        table = {}
        for i in range(self.ev.shape[0]):
            for f in range(d + 1):
                table.setdefault(tuple(sorted(int(v) for k, v in enumerate(self.ev[i]) if k != f)), []).append((i, f))
        self.face_of = {}
        for key, ent in table.items():
            ent = sorted(ent)
            for (i, f) in ent:
                self.face_of[(i, f)] = ent

    def X(self, e):
        return self.xyz[self.ev[e]]

    def _face(self, ent):
        """Blocks of one face: sides [(element, D[l], Q~[l])], M_j, E_j."""
        d, b = self.d, self.b
        (el, fl) = ent[0]
        Xl = self.X(el)
        F = Xl[[k for k in range(d + 1) if k != fl]]
        if d == 2:
            t = F[1] - F[0]
            nrm = np.array([t[1], -t[0]], dtype=LD)
        else:
            nrm = np.cross(F[1] - F[0], F[2] - F[0]).astype(LD)
        nrm = nrm / np.sqrt(np.sum(nrm * nrm))
        if np.dot(nrm, F[0] - Xl[fl]) < 0:
            nrm = -nrm
        elems = [e for (e, _) in ent]
        interior = len(elems) == 2
        bary = [self.X(e).mean(axis=0) for e in elems]
        subs = [np.concatenate([F, bc[None, :]], axis=0) for bc in bary]
        vols = [abs(_det((S[1:] - S[:1]).T)) for S in subs]          # d! |T_{i,j}|
        cens = [S.mean(axis=0) for S in subs]
        xc = sum(v * cc for v, cc in zip(vols, cens)) / sum(vols)
        verts = list(F) + bary
        hj = max(np.sqrt(np.sum((q - xc) ** 2)) for q in verts)
        psi = lambda x: monomials((x - xc[None, :]) / hj, b.exps)
        pf, wf = map_rule(F, self.face_rule)
        M = np.zeros((self.Npsi, self.Npsi), dtype=LD)
        sides = []
        for s, (e, S) in enumerate(zip(elems, subs)):
            sgn = LD(1) if s == 0 else LD(-1)
            ps, ws = map_rule(S, self.vol_rule)
            phs, gphs = b.phi(self.X(e), ps)
            pss = psi(ps)
            vol = np.einsum("q,qkl,qm->lkm", ws, gphs, pss)            # int d_l phi_k psi_m
            volq = np.einsum("q,qm,qkl->lmk", ws, pss, gphs)           # int psi_m d_l phi_k
            if interior:
                phf, _ = b.phi(self.X(e), pf)
                fint = np.einsum("q,qk,qm->km", wf, phf, psi(pf))       # int_Gamma phi_k psi_m
                fintq = np.einsum("q,qm,qk->mk", wf, psi(pf), phf)      # int_Gamma psi_m phi_k
            else:
                fint = np.zeros((b.N, self.Npsi), dtype=LD)
                fintq = np.zeros((self.Npsi, b.N), dtype=LD)
            D = np.stack([fint * (sgn * nrm[l]) - vol[l] for l in range(d)])
            Q = np.stack([volq[l] - fintq * (sgn * nrm[l]) for l in range(d)])
            M += np.einsum("q,qk,qm->km", ws, pss, pss)
            sides.append((e, D, Q))
        w = [v / LD(1) for v in vols]
        lam = sum(wi * self.lam[e] for wi, e in zip(w, elems)) / sum(w)
        mu = sum(wi * self.mu[e] for wi, e in zip(w, elems)) / sum(w)
        return sides, M, stiffness(lam, mu, d)

    def face_blocks(self, i, f):
        return self._face(self.face_of[(i, f)])

    def row(self, i, x):
        """(A x)_i, shape (d, Ng * N_phi), for x in the canonical layout (any float type)."""
        d, b = self.d, self.b
        Ng, N = b.Ng, b.N
        xe = lambda e: np.asarray(x, dtype=np.float64).reshape(-1, d, Ng * N)[e].astype(LD)
        dtW = self.dt * b.W
        Xi = self.X(i)
        pe, we = map_rule(Xi, self.vol_rule)
        ph, _ = b.phi(Xi, pe)
        Mbar = np.einsum("q,qk,qm->km", we, ph, ph)
        y = self.rho[i] * np.einsum("xw,kw->kx", np.kron(b.T, Mbar), xe(i))
        for f in range(d + 1):
            sides, M, E = self.face_blocks(i, f)
            Mst = np.kron(b.T, M)
            G = np.zeros((d, d, Ng * self.Npsi), dtype=LD)             # G[m, n] = sum Q~st[n] x_m
            for (e, D, Q) in sides:
                xs = xe(e)
                for n_ in range(d):
                    Qst = np.kron(dtW, Q[n_])
                    for m in range(d):
                        G[m, n_] += Qst @ xs[m]
            sig = np.einsum("klmn,mnz->klz", E, G)
            h = solve(Mst, sig.reshape(d * d, -1).T).T.reshape(d, d, -1)
            me = [k for k, (e, _, _) in enumerate(sides) if e == i][0]
            D = sides[me][1]
            for k in range(d):
                for l in range(d):
                    y[k] -= self.c * (np.kron(dtW, D[l]) @ h[k, l])
        return y

    def rows(self, elems, x):
        return np.array([self.row(i, x) for i in elems])
