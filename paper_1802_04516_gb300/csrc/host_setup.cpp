// Host-side set-up: reference-element tables, time basis, quadrature rules and
// mesh connectivity (Sec. 3 "Staggered unstructured grid and basis functions").
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

#include "stdg_internal.h"

namespace stdg {

// In-place Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix.
static bool invert(int n, double* a) {
    std::vector<double> inv(n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(a[r * n + c]) > std::fabs(a[piv * n + c])) piv = r;
        if (a[piv * n + c] == 0.0) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) { std::swap(a[c * n + k], a[piv * n + k]); std::swap(inv[c * n + k], inv[piv * n + k]); }
        double d = 1.0 / a[c * n + c];
        for (int k = 0; k < n; ++k) { a[c * n + k] *= d; inv[c * n + k] *= d; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = a[r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) { a[r * n + k] -= f * a[c * n + k]; inv[r * n + k] -= f * inv[c * n + k]; }
        }
    }
    std::memcpy(a, inv.data(), sizeof(double) * n * n);
    return true;
}

// Gauss-Legendre points and weights on [0,1], ascending (Newton on P_n).
void gauss_legendre01(int n, double* x, double* w) {
    for (int k = 0; k < n; ++k) {
        double z = std::cos(M_PI * (n - k - 0.25) / (n + 0.5));   // ascending order
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int m = 2; m <= n; ++m) { double p2 = ((2 * m - 1) * z * p1 - (m - 1) * p0) / m; p0 = p1; p1 = p2; }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        {   // recompute derivative at the converged root
            double p0 = 1.0, p1 = z;
            for (int m = 2; m <= n; ++m) { double p2 = ((2 * m - 1) * z * p1 - (m - 1) * p0) / m; p0 = p1; p1 = p2; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[k] = 0.5 * (z + 1.0);
        w[k] = 1.0 / ((1.0 - z * z) * dp * dp);   // = (2/((1-z^2) P'^2)) / 2
    }
}

void lagrange_time(const RefTables& rt, double tau, double* val) {
    for (int a = 0; a < rt.Ng; ++a) {
        double v = 1.0;
        for (int b = 0; b < rt.Ng; ++b)
            if (b != a) v *= (tau - rt.tnodes[b]) / (rt.tnodes[a] - rt.tnodes[b]);
        val[a] = v;
    }
}

Rule simplex_rule(int dim, int n) {
    std::vector<double> x(n), w(n);
    gauss_legendre01(n, x.data(), w.data());
    Rule r;
    r.dim = dim;
    if (dim == 1) {
        for (int i = 0; i < n; ++i) { r.pts.push_back(x[i]); r.wts.push_back(w[i]); }
    } else if (dim == 2) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double u = x[i], v = x[j];
                r.pts.push_back(u);
                r.pts.push_back(v * (1.0 - u));
                r.wts.push_back(w[i] * w[j] * (1.0 - u));
            }
    } else {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    double u = x[i], v = x[j], s = x[k];
                    r.pts.push_back(u);
                    r.pts.push_back(v * (1.0 - u));
                    r.pts.push_back(s * (1.0 - u) * (1.0 - v));
                    r.wts.push_back(w[i] * w[j] * w[k] * (1.0 - u) * (1.0 - u) * (1.0 - v));
                }
    }
    return r;
}

static double mono(const int* e, const double* xi, int dim) {
    double v = 1.0;
    for (int r = 0; r < dim; ++r)
        for (int q = 0; q < e[r]; ++q) v *= xi[r];
    return v;
}

void build_ref_tables(int dim, int p, int pg, RefTables* rt) {
    std::memset(rt, 0, sizeof(RefTables));
    rt->dim = dim; rt->p = p; rt->pg = pg; rt->Ng = pg + 1; rt->s = dim == 2 ? 3 : 6;
    // graded-lex exponents: degree ascending, then x-exponent descending, then y descending
    int n = 0;
    for (int g = 0; g <= p; ++g) {
        if (dim == 2) {
            for (int a = g; a >= 0; --a) { rt->exps[n][0] = a; rt->exps[n][1] = g - a; rt->exps[n][2] = 0; ++n; }
        } else {
            for (int a = g; a >= 0; --a)
                for (int b = g - a; b >= 0; --b) { rt->exps[n][0] = a; rt->exps[n][1] = b; rt->exps[n][2] = g - a - b; ++n; }
        }
    }
    rt->Nphi = rt->Npsi = n;
    for (int i = 0; i < n; ++i)
        for (int r = 0; r < 3; ++r) {
            int want[3] = {rt->exps[i][0], rt->exps[i][1], rt->exps[i][2]};
            ++want[r];
            rt->succ[i][r] = -1;
            if (r < dim)
                for (int j = 0; j < n; ++j)
                    if (rt->exps[j][0] == want[0] && rt->exps[j][1] == want[1] && rt->exps[j][2] == want[2]) rt->succ[i][r] = j;
        }
    // equispaced nodes, z outer, y, x fastest
    std::vector<std::array<double, 3>> nodes;
    if (dim == 2) {
        for (int j = 0; j <= p; ++j)
            for (int i = 0; i <= p - j; ++i) nodes.push_back({(double)i / p, (double)j / p, 0.0});
    } else {
        for (int k = 0; k <= p; ++k)
            for (int j = 0; j <= p - k; ++j)
                for (int i = 0; i <= p - j - k; ++i) nodes.push_back({(double)i / p, (double)j / p, (double)k / p});
    }
    std::vector<double> V(n * n);
    for (int r = 0; r < n; ++r)
        for (int a = 0; a < n; ++a) V[r * n + a] = mono(rt->exps[a], nodes[r].data(), dim);
    invert(n, V.data());                       // V^{-1}[a][k]
    std::memcpy(rt->coef, V.data(), sizeof(double) * n * n);
    // reference mass matrix
    Rule q = simplex_rule(dim, p + 2);
    std::vector<double> phi(n), m(n);
    for (int iq = 0; iq < q.n(); ++iq) {
        const double* xi = &q.pts[iq * dim];
        for (int a = 0; a < n; ++a) m[a] = mono(rt->exps[a], xi, dim);
        for (int k = 0; k < n; ++k) { double v = 0; for (int a = 0; a < n; ++a) v += rt->coef[a * n + k] * m[a]; phi[k] = v; }
        for (int k = 0; k < n; ++k)
            for (int l = 0; l < n; ++l) rt->Mref[k * n + l] += q.wts[iq] * phi[k] * phi[l];
    }
    std::memcpy(rt->MrefInv, rt->Mref, sizeof(double) * n * n);
    invert(n, rt->MrefInv);
    {   // Cholesky factor R of M_ref and its inverse (lower triangular)
        std::vector<double> R(n * n, 0.0);
        for (int i = 0; i < n; ++i)
            for (int j = 0; j <= i; ++j) {
                double s = rt->Mref[i * n + j];
                for (int k = 0; k < j; ++k) s -= R[i * n + k] * R[j * n + k];
                R[i * n + j] = i == j ? std::sqrt(s) : s / R[j * n + j];
            }
        invert(n, R.data());
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) rt->MrefLinv[i * n + j] = j <= i ? R[i * n + j] : 0.0;
    }
    // time basis on the Gauss-Legendre points of [0,1]
    int G = rt->Ng;
    gauss_legendre01(G, rt->tnodes, rt->W);
    lagrange_time(*rt, 0.0, rt->g0);
    lagrange_time(*rt, 1.0, rt->g1);
    // K[a][b] = int gamma_a' gamma_b = w_b gamma_a'(tau_b) (Gauss rule exact for degree 2G-3)
    double K[kMaxNG * kMaxNG];
    for (int a = 0; a < G; ++a)
        for (int b = 0; b < G; ++b) {
            double d = 0.0;
            if (a == b) {
                for (int c = 0; c < G; ++c) if (c != a) d += 1.0 / (rt->tnodes[a] - rt->tnodes[c]);
            } else {
                d = 1.0 / (rt->tnodes[a] - rt->tnodes[b]);
                for (int c = 0; c < G; ++c)
                    if (c != a && c != b) d *= (rt->tnodes[b] - rt->tnodes[c]) / (rt->tnodes[a] - rt->tnodes[c]);
            }
            K[a * G + b] = rt->W[b] * d;
        }
    for (int a = 0; a < G; ++a)
        for (int b = 0; b < G; ++b) rt->T[a * G + b] = rt->g1[a] * rt->g1[b] - K[a * G + b];
    std::memcpy(rt->Tinv, rt->T, sizeof(double) * G * G);
    invert(G, rt->Tinv);
    for (int a = 0; a < G; ++a) {
        double s = 0.0;
        for (int b = 0; b < G; ++b) {
            rt->S[a * G + b] = rt->W[a] * rt->Tinv[a * G + b] * rt->W[b];
            s += rt->Tinv[a * G + b] * rt->g0[b];
        }
        rt->Tinv_g0[a] = s;
    }
    rt->kappa = 0.0;
    for (int b = 0; b < G; ++b) {
        double s = 0.0;
        for (int a = 0; a < G; ++a) s += rt->g1[a] * rt->Tinv[a * G + b];
        rt->u_tr[b] = s * rt->W[b];
        rt->kappa += s * rt->g0[b];
    }
}

// ------------------------------------------------------------------------------------
struct FaceRec {
    int32_t v[3];
    int32_t elem;
    int8_t f;
};

int build_host_mesh(int dim, int64_t n_vert, const double* xyz, int64_t n_elem, const int32_t* ev,
                    const double* period, HostMesh* m, std::string* err) {
    const int nv = dim + 1;
    m->dim = dim;
    m->n_elem = n_elem;
    m->period.clear();
    if (period) m->period.assign(period, period + dim);
    m->X.assign(n_elem * nv * dim, 0.0);
    m->Jinv.assign(n_elem * dim * dim, 0.0);
    m->detJ.assign(n_elem, 0.0);
    for (int64_t e = 0; e < n_elem; ++e) {
        for (int k = 0; k < nv; ++k) {
            int32_t g = ev[e * nv + k];
            if (g < 0 || g >= n_vert) { *err = "vertex index out of range"; return STDG_EINVAL; }
            for (int a = 0; a < dim; ++a) {
                double x = xyz[(int64_t)g * dim + a];
                if (!std::isfinite(x)) { *err = "non-finite vertex coordinate"; return STDG_EINVAL; }
                if (period && period[a] > 0 && k > 0) {
                    double x0 = m->X[(e * nv) * dim + a];
                    x -= period[a] * std::nearbyint((x - x0) / period[a]);
                }
                m->X[(e * nv + k) * dim + a] = x;
            }
        }
        double J[9];
        for (int a = 0; a < dim; ++a)
            for (int c = 0; c < dim; ++c)
                J[a * dim + c] = m->X[(e * nv + c + 1) * dim + a] - m->X[(e * nv) * dim + a];
        double det = dim == 2 ? J[0] * J[3] - J[1] * J[2]
                              : J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                                    J[2] * (J[3] * J[7] - J[4] * J[6]);
        if (!(det > 0.0)) { *err = "inverted or degenerate element " + std::to_string(e); return STDG_EMESH; }
        m->detJ[e] = det;
        invert(dim, J);
        std::memcpy(&m->Jinv[e * dim * dim], J, sizeof(double) * dim * dim);
    }
    // faces by sorted vertex tuple
    std::vector<FaceRec> recs(n_elem * nv);
    for (int64_t e = 0; e < n_elem; ++e)
        for (int f = 0; f < nv; ++f) {
            FaceRec& r = recs[e * nv + f];
            int q = 0;
            for (int k = 0; k < nv; ++k) if (k != f) r.v[q++] = ev[e * nv + k];
            if (dim == 2) r.v[2] = -1;
            std::sort(r.v, r.v + dim);
            r.elem = (int32_t)e;
            r.f = (int8_t)f;
        }
    std::sort(recs.begin(), recs.end(), [](const FaceRec& a, const FaceRec& b) {
        if (a.v[0] != b.v[0]) return a.v[0] < b.v[0];
        if (a.v[1] != b.v[1]) return a.v[1] < b.v[1];
        if (a.v[2] != b.v[2]) return a.v[2] < b.v[2];
        return a.elem < b.elem;
    });
    m->face_l.clear(); m->face_r.clear(); m->face_fl.clear(); m->face_fr.clear();
    m->elem_face.assign(n_elem * nv, -1);
    size_t i = 0;
    m->n_bnd = 0;
    while (i < recs.size()) {
        size_t j = i + 1;
        while (j < recs.size() && recs[j].v[0] == recs[i].v[0] && recs[j].v[1] == recs[i].v[1] && recs[j].v[2] == recs[i].v[2]) ++j;
        if (j - i > 2) { *err = "non-manifold face"; return STDG_EMESH; }
        int32_t fid = (int32_t)m->face_l.size();
        m->face_l.push_back(recs[i].elem);
        m->face_fl.push_back(recs[i].f);
        m->elem_face[(int64_t)recs[i].elem * nv + recs[i].f] = fid;
        if (j - i == 2) {
            if (recs[i + 1].elem == recs[i].elem) { *err = "element is its own neighbour"; return STDG_EMESH; }
            m->face_r.push_back(recs[i + 1].elem);
            m->face_fr.push_back(recs[i + 1].f);
            m->elem_face[(int64_t)recs[i + 1].elem * nv + recs[i + 1].f] = fid;
        } else {
            m->face_r.push_back(-1);
            m->face_fr.push_back(-1);
            ++m->n_bnd;
        }
        i = j;
    }
    const int64_t nf = (int64_t)m->face_l.size();
    m->n_face = nf;
    m->face_X.assign(nf * dim * dim, 0.0);
    m->shift.assign(nf * dim, 0.0);
    m->normal.assign(nf * dim, 0.0);
    m->xc.assign(nf * dim, 0.0);
    m->hj.assign(nf, 0.0);
    m->frame.assign(nf * dim * dim, 0.0);
    for (int64_t f = 0; f < nf; ++f) {
        const int64_t el = m->face_l[f];
        const int fl = m->face_fl[f];
        int q = 0;
        int32_t g0 = -1;
        for (int k = 0; k < nv; ++k) {
            if (k == fl) continue;
            if (q == 0) g0 = ev[el * nv + k];
            for (int a = 0; a < dim; ++a) m->face_X[(f * dim + q) * dim + a] = m->X[(el * nv + k) * dim + a];
            ++q;
        }
        const double* F = &m->face_X[f * dim * dim];
        const int64_t er = m->face_r[f];
        if (er >= 0) {
            int kr = 0;
            while (ev[er * nv + kr] != g0) ++kr;
            for (int a = 0; a < dim; ++a) m->shift[f * dim + a] = F[a] - m->X[(er * nv + kr) * dim + a];
        }
        double n[3] = {0, 0, 0};
        if (dim == 2) {
            n[0] = F[3] - F[1];
            n[1] = -(F[2] - F[0]);
        } else {
            double u[3], w[3];
            for (int a = 0; a < 3; ++a) { u[a] = F[3 + a] - F[a]; w[a] = F[6 + a] - F[a]; }
            n[0] = u[1] * w[2] - u[2] * w[1];
            n[1] = u[2] * w[0] - u[0] * w[2];
            n[2] = u[0] * w[1] - u[1] * w[0];
        }
        double nn = 0, dot = 0;
        for (int a = 0; a < dim; ++a) nn += n[a] * n[a];
        nn = std::sqrt(nn);
        for (int a = 0; a < dim; ++a) {
            n[a] /= nn;
            dot += n[a] * (F[a] - m->X[(el * nv + fl) * dim + a]);
        }
        for (int a = 0; a < dim; ++a) m->normal[f * dim + a] = dot < 0 ? -n[a] : n[a];
        // dual cell R_j: measure-weighted centroid of its sub-cells and scale h_j
        double bl[3] = {0, 0, 0}, br[3] = {0, 0, 0}, fs[3] = {0, 0, 0};
        for (int k = 0; k < nv; ++k)
            for (int a = 0; a < dim; ++a) bl[a] += m->X[(el * nv + k) * dim + a] / nv;
        for (int q2 = 0; q2 < dim; ++q2)
            for (int a = 0; a < dim; ++a) fs[a] += F[q2 * dim + a];
        double wl = m->detJ[el], wr = 0.0;
        double c[3];
        for (int a = 0; a < dim; ++a) c[a] = wl * (fs[a] + bl[a]) / nv;
        if (er >= 0) {
            wr = m->detJ[er];
            for (int k = 0; k < nv; ++k)
                for (int a = 0; a < dim; ++a) br[a] += m->X[(er * nv + k) * dim + a] / nv;
            for (int a = 0; a < dim; ++a) {
                br[a] += m->shift[f * dim + a];
                c[a] += wr * (fs[a] + br[a]) / nv;
            }
        }
        for (int a = 0; a < dim; ++a) m->xc[f * dim + a] = c[a] / (wl + wr);
        double h = 0.0;
        auto upd = [&](const double* p) {
            double d2 = 0;
            for (int a = 0; a < dim; ++a) d2 += (p[a] - m->xc[f * dim + a]) * (p[a] - m->xc[f * dim + a]);
            h = std::max(h, std::sqrt(d2));
        };
        for (int q2 = 0; q2 < dim; ++q2) upd(F + q2 * dim);
        upd(bl);
        if (er >= 0) upd(br);
        m->hj[f] = h;
        // principal-axis frame of R_j: covariance of the dual cell about x_j (a simplex S has
        // int_S v v^T = |S| / ((d+1)(d+2)) (sum_i v_i v_i^T + (sum_i v_i)(sum_i v_i)^T), v = x - x_j),
        // B_j = Cov^{-1/2}.  Monomials of y' = B_j (x - x_j) span the same P_p(R_j) as the Taylor
        // monomials but stay well conditioned on thin dual cells (slivers).
        double cov[3][3] = {{0}}, meas = 0.0;
        auto add_sub = [&](const double* bc, double detJ) {
            const double sub = detJ / (dim == 2 ? 2.0 : 6.0) / nv;   // |T_{i,j}| = |T_i| / (d+1)
            double v[4][3], sv[3] = {0, 0, 0};
            for (int q2 = 0; q2 < nv; ++q2)
                for (int a = 0; a < dim; ++a) {
                    v[q2][a] = (q2 < dim ? F[q2 * dim + a] : bc[a]) - m->xc[f * dim + a];
                    sv[a] += v[q2][a];
                }
            const double k = sub / ((dim + 1) * (dim + 2));
            for (int a = 0; a < dim; ++a)
                for (int b2 = 0; b2 < dim; ++b2) {
                    double t = sv[a] * sv[b2];
                    for (int q2 = 0; q2 < nv; ++q2) t += v[q2][a] * v[q2][b2];
                    cov[a][b2] += k * t;
                }
            meas += sub;
        };
        add_sub(bl, m->detJ[el]);
        if (er >= 0) add_sub(br, m->detJ[er]);
        double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, A[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b2 = 0; b2 < 3; ++b2) A[a][b2] = a < dim && b2 < dim ? cov[a][b2] / meas : (a == b2 ? 1.0 : 0.0);
        for (int sweep = 0; sweep < 30; ++sweep) {   // cyclic Jacobi on the symmetric covariance
            double off = 0;
            for (int a = 0; a < dim; ++a)
                for (int b2 = a + 1; b2 < dim; ++b2) off += A[a][b2] * A[a][b2];
            if (off <= 1e-30 * (A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2])) break;
            for (int pp = 0; pp < dim; ++pp)
                for (int qq = pp + 1; qq < dim; ++qq) {
                    if (A[pp][qq] == 0.0) continue;
                    const double th = 0.5 * (A[qq][qq] - A[pp][pp]) / A[pp][qq];
                    const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                    const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                    for (int k2 = 0; k2 < 3; ++k2) {   // A <- A J
                        const double x1 = A[k2][pp], x2 = A[k2][qq];
                        A[k2][pp] = cs * x1 - sn * x2;
                        A[k2][qq] = sn * x1 + cs * x2;
                    }
                    for (int k2 = 0; k2 < 3; ++k2) {   // A <- J^T A
                        const double x1 = A[pp][k2], x2 = A[qq][k2];
                        A[pp][k2] = cs * x1 - sn * x2;
                        A[qq][k2] = sn * x1 + cs * x2;
                    }
                    for (int k2 = 0; k2 < 3; ++k2) {   // V <- V J
                        const double x1 = V[k2][pp], x2 = V[k2][qq];
                        V[k2][pp] = cs * x1 - sn * x2;
                        V[k2][qq] = sn * x1 + cs * x2;
                    }
                }
        }
        for (int r = 0; r < dim; ++r) {   // B = Lambda^{-1/2} V^T
            const double sc = 1.0 / std::sqrt(A[r][r]);
            for (int a = 0; a < dim; ++a) m->frame[(f * dim + r) * dim + a] = sc * V[a][r];
        }
    }
    return STDG_OK;
}

int64_t locate_point(const HostMesh& m, const double* x, double* x_local) {
    const int dim = m.dim, nv = dim + 1;
    for (int64_t e = 0; e < m.n_elem; ++e) {
        double y[3];
        for (int a = 0; a < dim; ++a) {
            y[a] = x[a];
            if (!m.period.empty() && m.period[a] > 0)
                y[a] -= m.period[a] * std::nearbyint((y[a] - m.X[(e * nv) * dim + a]) / m.period[a]);
        }
        double lam0 = 1.0;
        bool inside = true;
        for (int r = 0; r < dim; ++r) {
            double xi = 0;
            for (int a = 0; a < dim; ++a) xi += m.Jinv[(e * dim + r) * dim + a] * (y[a] - m.X[(e * nv) * dim + a]);
            if (xi < -1e-12) inside = false;
            lam0 -= xi;
        }
        if (lam0 < -1e-12) inside = false;
        if (inside) {
            for (int a = 0; a < dim; ++a) x_local[a] = y[a];
            return e;
        }
    }
    return -1;
}

}  // namespace stdg
