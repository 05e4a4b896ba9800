// Receiver misfit and its gradient with respect to per-element lambda, mu, rho and the point
// sources (amplitude, force direction, position; Sec. 6.3) by the discrete adjoint of the space-time DG slab map (the paper has no adjoint; the forward
// map is Eq. velocity.sys followed by the stress update of Eq. NM26 and the traces).
//
// Forward slab n -> n+1 of one shot, as the library computes it (orthonormal dual basis):
//   b      = rho|J| g0 (x) M_ref v^n  +  coef (x) D~ . sigma^n  +  s^n,   coef = dt W T^{-1} g0
//   A x    = b,                        A = rho|J| T (x) M_ref + c dt^2 D~ (S (x) E_j :) D~^T
//   sigma^{n+1} = kappa sigma^n - dt sum_b u_b E_j : (D~^T x)_b,     v^{n+1} = g1^T x
//   L      = 1/2 sum_shots sum_{n=1..N} sum_r |v_h(x_r, t^n) - d_r^n|^2
// Backward slab (a_v, a_s: adjoints of v^{n+1}, sigma^{n+1}):
//   a_x    = g1 (x) a_v  +  D~ (-dt u (x) E' : a_s)           (E' = transpose of E_j : on the
//            symmetric components: lam delta tr + mu (2 a_c on the diagonal, a_c off it))
//   A^T lam = a_x
//   a_v    <- rho|J| g0^T (x) M_ref lam  +  R^T (rec^n - d^n)
//   a_s    <- kappa a_s + sum_a coef_a sym(D~^T lam_a)         (mirror entries summed)
//   dL/drho_i   += |J_i| [lam_i . (g0 (x) M_ref v^n_i) - lam_i . (T (x) M_ref x_i)]
//   dL/dlam_j   += -c dt^2 <tr D~^T lam, S tr D~^T x> - dt sum_b u_b <diag-sum a_s, tr (D~^T x)_b>
//   dL/dmu_j    += -c dt^2 <D~^T lam, S (G + G^T)> - dt sum_b u_b <a_s, sym(G + G^T)_b>,  G = D~^T x
// and the dual-cell values feed the elements with the sub-cell weights |T_i| / |R_j|.
//   dL/dtheta_src += lam . ds^n/dtheta_src,  s^n = a1 dir (x) (dt int gamma S_1) (x) phi(x_s):
//   linear in a1 and dir, through phi(x_s) in the position (the source's element held fixed).
//
// The transposed solve needs no operator of its own: with the Lagrange time basis on the
// symmetric Gauss-Legendre points, T^T = J T J and S^T = J S J for the reversal J of the
// time nodes, so A^T = J A J and A^T lam = a_x is A (J lam) = J a_x -- the forward solver
// (and its preconditioner) on time-reversed vectors.
//
// Memory: uniform checkpointing.  The forward run stores the traces of all shots every K
// slabs; the backward sweep recomputes each segment of K slabs from its checkpoint,
// keeping v^n and x^{n+1} of the segment, and runs the adjoint slabs through it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "stdg_internal.h"

namespace stdg {

namespace {

__device__ __forceinline__ int symc(int dim, int a, int b) {
    if (a == b) return a;
    if (dim == 2) return 2;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return (lo == 0 && hi == 1) ? 3 : (lo == 1 ? 4 : 5);
}
__device__ __forceinline__ void symab(int dim, int c, int& a, int& b) {
    if (c < dim) { a = b = c; return; }
    if (dim == 2) { a = 0; b = 1; return; }
    if (c == 3) { a = 0; b = 1; } else if (c == 4) { a = 1; b = 2; } else { a = 0; b = 2; }
}

// b[s][e][k][J(a)][n] = g1[a] a_v[s][e][k][n]   (J a = NG - 1 - a: the time reversal)
__global__ void adj_gamma_kernel(int64_t nrows, int NP, int NG, const RefTables* __restrict__ rtp,
                                 const double* __restrict__ av, double* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows * NG * NP; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / (NG * NP);
        const int a = (int)((i / NP) % NG), n = (int)(i % NP);
        b[(row * NG + (NG - 1 - a)) * NP + n] = rtp->g1[a] * av[row * NP + n];
    }
}

// a_v[s][e_r][k][n] += phi_r[n] (rec - d)[s][r][k]
__global__ void adj_receivers_kernel(int n_shots, int n_rec, int dim, int NP, int64_t ntr, const int32_t* __restrict__ elem,
                                     const double* __restrict__ phi, const double* __restrict__ rec, int64_t rec_stride,
                                     const double* __restrict__ data, int64_t data_stride, double* __restrict__ av) {
    const int64_t total = (int64_t)n_shots * n_rec * dim * NP;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(i % NP);
        const int k = (int)((i / NP) % dim);
        const int r = (int)((i / (NP * dim)) % n_rec);
        const int s = (int)(i / ((int64_t)NP * dim * n_rec));
        const double res = rec[s * rec_stride + r * dim + k] - data[s * data_stride + r * dim + k];
        atomicAdd(&av[s * ntr + ((int64_t)elem[r] * dim + k) * NP + n], phi[r * NP + n] * res);
    }
}

// Per (shot, element, component) row: rho gradient and the new a_v = rho|J| g0^T (x) M_ref lam.
// lam is read time-reversed from the solve's y = J lam.
__global__ void adj_element_kernel(int64_t n_elem, int n_shots, int dim, int NP, int NG, const RefTables* __restrict__ rtp,
                                   const double* __restrict__ rhoJ, const double* __restrict__ detJ,
                                   const double* __restrict__ y, const double* __restrict__ vtr, const double* __restrict__ x,
                                   double* __restrict__ av, double* __restrict__ g_rho) {
    const int64_t nvel = n_elem * dim * NG * NP, ntr = n_elem * dim * NP;
    const int64_t rows = (int64_t)n_shots * n_elem * dim;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < rows; row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = row / (n_elem * dim);
        const int64_t ek = row % (n_elem * dim);
        const int64_t e = ek / dim;
        const double* ys = y + s * nvel + ek * NG * NP;
        const double* xs = x + s * nvel + ek * NG * NP;
        const double* vs = vtr + s * ntr + ek * NP;
        double gm = 0.0;     // lam . (g0 (x) M v^n) - lam . (T (x) M x)
        double* ao = av + s * ntr + ek * NP;
        for (int n = 0; n < NP; ++n) {
            double mv = 0.0, lg = 0.0;
            for (int q = 0; q < NP; ++q) mv += rtp->Mref[n * NP + q] * vs[q];
            for (int a = 0; a < NG; ++a) {
                const double la = ys[(NG - 1 - a) * NP + n];
                lg += rtp->g0[a] * la;
                double tmx = 0.0;
                for (int b = 0; b < NG; ++b) {
                    double mx = 0.0;
                    for (int q = 0; q < NP; ++q) mx += rtp->Mref[n * NP + q] * xs[b * NP + q];
                    tmx += rtp->T[a * NG + b] * mx;
                }
                gm -= la * tmx;
            }
            gm += lg * mv;
        }
        // a_v[n] = rho|J| sum_q M_ref[n][q] (g0 . lam)[q]
        for (int n = 0; n < NP; ++n) {
            double acc = 0.0;
            for (int q = 0; q < NP; ++q) {
                double lg = 0.0;
                for (int a = 0; a < NG; ++a) lg += rtp->g0[a] * ys[(NG - 1 - a) * NP + q];
                acc += rtp->Mref[n * NP + q] * lg;
            }
            ao[n] = rhoJ[e] * acc;
        }
        atomicAdd(&g_rho[e], detJ[e] * gm);
    }
}

// One warp per face, shots in sequence: the lambda_j / mu_j gradients (with the adjoint
// stress a_s of sigma^{n+1}), then a_s <- a_s of sigma^n.  lam is read time-reversed.
template <int DIM>
__global__ void __launch_bounds__(128) adj_face_kernel(int64_t n_face, int n_shots, int NP, int NG,
                                                       const int32_t* __restrict__ fl, const int32_t* __restrict__ fr,
                                                       const double* __restrict__ D, const RefTables* __restrict__ rtp,
                                                       double dt, double scale, const double* __restrict__ y,
                                                       const double* __restrict__ x, double* __restrict__ as,
                                                       int64_t nvel, int64_t nsig, double* __restrict__ g_lf,
                                                       double* __restrict__ g_mf) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int nD = 2 * DIM * NP * NP;
    const int nvs = DIM * NG * NP;
    const int ng = DIM * DIM * NG * NP;
    double* sD = sm + (size_t)warp * (nD + 4 * nvs + 2 * ng + NS * NP);
    double* sl = sD + nD;            // lam, both sides [side][k][a][n]
    double* sx = sl + 2 * nvs;       // x^{n+1}, both sides
    double* gL = sx + 2 * nvs;       // [k][l][a][m]  D~^T lam
    double* gX = gL + ng;            // [k][l][b][m]  D~^T x
    double* sa = gX + ng;            // a_s [c][m]
    const double kap = rtp->kappa;
    for (int64_t f = blockIdx.x * (int64_t)wpb + warp; f < n_face; f += (int64_t)gridDim.x * wpb) {
        const int el = fl[f], er = fr[f];
        for (int t = lane; t < nD; t += 32) sD[t] = D[f * nD + t];
        double acc_l = 0.0, acc_m = 0.0;
        for (int s = 0; s < n_shots; ++s) {
            const double* ys = y + s * nvel;
            const double* xs = x + s * nvel;
            for (int t = lane; t < nvs; t += 32) {
                const int k = t / (NG * NP), a = (t / NP) % NG, n = t % NP;
                const int tr = (k * NG + (NG - 1 - a)) * NP + n;
                sl[t] = ys[(int64_t)el * nvs + tr];
                sl[nvs + t] = er >= 0 ? ys[(int64_t)er * nvs + tr] : 0.0;
                sx[t] = xs[(int64_t)el * nvs + t];
                sx[nvs + t] = er >= 0 ? xs[(int64_t)er * nvs + t] : 0.0;
            }
            for (int t = lane; t < NS * NP; t += 32) sa[t] = as[s * nsig + f * NS * NP + t];
            __syncwarp();
            // g[k][l][a][m] = sum_side sum_n D~_side[l][n][m] v_side[k][a][n]
            for (int ent = lane; ent < 2 * ng; ent += 32) {
                const int which = ent / ng, r = ent % ng;
                const int k = r / (DIM * NG * NP), l = (r / (NG * NP)) % DIM, a = (r / NP) % NG, m = r % NP;
                const double* src = which == 0 ? sl : sx;
                double acc = 0.0;
                for (int side = 0; side < 2; ++side) {
                    const double* Dp = sD + (side * DIM + l) * NP * NP + m;
                    const double* vp = src + side * nvs + (k * NG + a) * NP;
                    for (int n = 0; n < NP; ++n) acc += Dp[n * NP] * vp[n];
                }
                (which == 0 ? gL : gX)[r] = acc;
            }
            __syncwarp();
            for (int ent = lane; ent < NG * NP; ent += 32) {
                const int a = ent / NP, m = ent % NP;
                // -lam^T (dA/dtheta_j) x:  -c dt^2 sum <gL[k][l]_a, S_ab (dE/dtheta : gX)_b>
                double trL = 0.0;
                for (int q = 0; q < DIM; ++q) trL += gL[((q * DIM + q) * NG + a) * NP + m];
                double trSX = 0.0, muSX = 0.0;
                for (int b2 = 0; b2 < NG; ++b2) {
                    const double sab = rtp->S[a * NG + b2];
                    double trX = 0.0;
                    for (int q = 0; q < DIM; ++q) trX += gX[((q * DIM + q) * NG + b2) * NP + m];
                    trSX += sab * trX;
                    for (int k = 0; k < DIM; ++k)
                        for (int l = 0; l < DIM; ++l)
                            muSX += gL[((k * DIM + l) * NG + a) * NP + m] * sab *
                                    (gX[((k * DIM + l) * NG + b2) * NP + m] + gX[((l * DIM + k) * NG + b2) * NP + m]);
                }
                acc_l -= scale * trL * trSX;
                acc_m -= scale * muSX;
                // a_s^T (dSx/dtheta_j) x, time node a:  -dt u_a sum_c a_s[c] (dE/dtheta : gX_a)[c]
                double trX = 0.0;
                for (int q = 0; q < DIM; ++q) trX += gX[((q * DIM + q) * NG + a) * NP + m];
                double dg = 0.0, mg = 0.0;
                for (int c = 0; c < NS; ++c) {
                    int p, q;
                    symab(DIM, c, p, q);
                    const double ac = sa[c * NP + m];
                    if (p == q) dg += ac;
                    mg += ac * (gX[((p * DIM + q) * NG + a) * NP + m] + gX[((q * DIM + p) * NG + a) * NP + m]);
                }
                acc_l -= dt * rtp->u_tr[a] * dg * trX;
                acc_m -= dt * rtp->u_tr[a] * mg;
            }
            // a_s <- kappa a_s + sum_a coef_a (gL[p][q] + [p != q] gL[q][p])_a,  coef_a = dt W_a (T^{-1} g0)_a
            for (int ent = lane; ent < NS * NP; ent += 32) {
                const int c = ent / NP, m = ent % NP;
                int p, q;
                symab(DIM, c, p, q);
                double v = kap * sa[ent];
                for (int a = 0; a < NG; ++a) {
                    double g = gL[((p * DIM + q) * NG + a) * NP + m];
                    if (p != q) g += gL[((q * DIM + p) * NG + a) * NP + m];
                    v += dt * rtp->W[a] * rtp->Tinv_g0[a] * g;
                }
                as[s * nsig + f * NS * NP + ent] = v;
            }
            __syncwarp();
        }
        for (int o = 16; o > 0; o >>= 1) {
            acc_l += __shfl_xor_sync(0xffffffffu, acc_l, o);
            acc_m += __shfl_xor_sync(0xffffffffu, acc_m, o);
        }
        if (lane == 0) {
            g_lf[f] += acc_l;
            g_mf[f] += acc_m;
        }
        __syncwarp();
    }
}

// Stress part of the adjoint right-hand side, time-reversed: b_side[k][J b][n] +=
// sum_l sum_m D~_side[l][n][m] h[sym(k,l)][b][m],  h[c][b] = -dt u_b E'(a_s)[c]  (Sx^T a_s)
template <int DIM>
__global__ void __launch_bounds__(128) adj_rhs_kernel(int64_t n_face, int n_shots, int NP, int NG,
                                                      const int32_t* __restrict__ fl, const int32_t* __restrict__ fr,
                                                      const double* __restrict__ D, const double* __restrict__ lamf,
                                                      const double* __restrict__ muf, const RefTables* __restrict__ rtp,
                                                      double dt, const double* __restrict__ as, double* __restrict__ b,
                                                      int64_t nvel, int64_t nsig) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    const int nD = 2 * DIM * NP * NP;
    const int nvs = DIM * NG * NP;
    double* sD = sm + (size_t)warp * (nD + NS * NP + NS * NG * NP);
    double* sa = sD + nD;
    double* sh = sa + NS * NP;
    for (int64_t f = blockIdx.x * (int64_t)wpb + warp; f < n_face; f += (int64_t)gridDim.x * wpb) {
        const int el = fl[f], er = fr[f];
        const double lam = lamf[f], mu = muf[f];
        for (int t = lane; t < nD; t += 32) sD[t] = D[f * nD + t];
        for (int s = 0; s < n_shots; ++s) {
            for (int t = lane; t < NS * NP; t += 32) sa[t] = as[s * nsig + f * NS * NP + t];
            __syncwarp();
            for (int ent = lane; ent < NS * NG * NP; ent += 32) {
                const int c = ent / (NG * NP), bb = (ent / NP) % NG, m = ent % NP;
                int p, q;
                symab(DIM, c, p, q);
                double e;
                if (p == q) {
                    double trn = 0.0;
                    for (int d2 = 0; d2 < DIM; ++d2) trn += sa[d2 * NP + m];
                    e = lam * trn + 2.0 * mu * sa[c * NP + m];
                } else {
                    e = mu * sa[c * NP + m];
                }
                sh[ent] = -dt * rtp->u_tr[bb] * e;
            }
            __syncwarp();
            const int nside = er >= 0 ? 2 : 1;
            for (int ent = lane; ent < nside * nvs; ent += 32) {
                const int side = ent / nvs, r = ent % nvs;
                const int k = r / (NG * NP), bb = (r / NP) % NG, n = r % NP;
                double acc = 0.0;
                for (int l = 0; l < DIM; ++l) {
                    const double* Dp = sD + ((side * DIM + l) * NP + n) * NP;
                    const double* hp = sh + (symc(DIM, k, l) * NG + bb) * NP;
                    for (int m = 0; m < NP; ++m) acc += Dp[m] * hp[m];
                }
                const int e = side == 0 ? el : er;
                atomicAdd(&b[s * nvel + (int64_t)e * nvs + (k * NG + (NG - 1 - bb)) * NP + n], acc);
            }
            __syncwarp();
        }
    }
}

// Point-source term of the gradient, per slab: for every source q (shot k = q / per) and
// component l, G[q][l][n] += sum_a lam[k][e_q][l][a][n] tint_a with tint_a = dt int gamma_a S at
// unit amplitude for this slab (lam read time-reversed from J lam).  The source vector of the
// slab is s = a1 dir (x) tint (x) phi(x_s), so lam^T ds/dtheta for the amplitude, the direction
// and the position are contractions of G with phi(x_s), grad phi(x_s) and dir (on the host).
struct TimeInt { double v[kMaxNG]; };
__global__ void adj_source_kernel(int nsrc, int per, int dim, int NP, int NG, const int32_t* __restrict__ elem,
                                  const double* __restrict__ lamJ, int64_t nvel, TimeInt tint, double* __restrict__ G) {
    const int64_t total = (int64_t)nsrc * dim * NP;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(i % NP), l = (int)((i / NP) % dim);
        const int64_t q = i / ((int64_t)NP * dim);
        const int64_t k = q / per;
        const double* lam = lamJ + k * nvel + ((int64_t)elem[q] * dim + l) * NG * NP;
        double acc = 0.0;
        for (int a = 0; a < NG; ++a) acc += lam[(NG - 1 - a) * NP + n] * tint.v[a];
        G[i] += acc;
    }
}

}  // namespace

// The misfit (and with gradients requested, the adjoint sweep) of n_steps slabs from the
// current state of every shot.  data: [shot][step][receiver][component].
int misfit_grad_impl(stdg_ctx* c, double dt, int N, const double* data, int K, double* loss, double* g_lam,
                     double* g_mu, double* g_rho, double* g_src, stdg_stats* stats) {
    const bool grads = g_lam || g_mu || g_rho || g_src;
    const bool src_grad = g_src && c->have_sources;
    const int nsrc = src_grad ? (int)c->src_elem.size() : 0;
    const int ns = c->n_shots, d = c->dim, NP = c->Nphi, NG = c->Ng, NR = c->n_rec;
    const int64_t ntr = c->ntr, nsig = c->nsig, nvel = c->nvel;
    const int64_t per_rec = (int64_t)NR * d;
    const int64_t rec0 = c->rec_steps;
    const double t0 = c->t;
    const int nseg = (N + K - 1) / K;
    std::vector<void*> tmp;
    auto alloc = [&](void** p, size_t bytes) {
        const int rc = dev_alloc(c, p, bytes);
        if (rc == STDG_OK) tmp.push_back(*p);
        return rc;
    };
    auto cleanup = [&]() {
        cudaStreamSynchronize(c->stream);
        for (void* p : tmp) dev_release(c, p);
        tmp.clear();
    };
    int rc = STDG_OK;
    double *ck = nullptr, *d_data = nullptr;
    const int64_t state = ns * (ntr + nsig);
    auto save = [&](double* dst) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, c->d_vtr, sizeof(double) * ns * ntr, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(dst + ns * ntr, c->d_sigtr, sizeof(double) * ns * nsig, cudaMemcpyDeviceToDevice, c->stream);
    };
    auto restore = [&](const double* src) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(c->d_vtr, src, sizeof(double) * ns * ntr, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(c->d_sigtr, src + ns * ntr, sizeof(double) * ns * nsig, cudaMemcpyDeviceToDevice, c->stream);
    };
#define ADJ_TRY(expr) do { rc = (expr); if (rc != STDG_OK) { cleanup(); return rc; } } while (0)
#define ADJ_CUDA(expr) do { cudaError_t e_ = (expr); if (e_ != cudaSuccess) { c->err = std::string(#expr) + ": " + \
                                cudaGetErrorString(e_); cleanup(); return STDG_ECUDA; } } while (0)
    std::memset(stats, 0, sizeof(*stats));
    auto add_stats = [&](const stdg_stats& s) {
        stats->iters_total += s.iters_total;
        stats->iters_max = std::max(stats->iters_max, s.iters_max);
        stats->refinements += s.refinements;
        stats->final_rel_res = std::max(stats->final_rel_res, s.final_rel_res);
    };
    // ---- forward with checkpoints
    if (grads) ADJ_TRY(alloc((void**)&ck, sizeof(double) * state * (nseg + 1)));
    for (int seg = 0; seg < nseg; ++seg) {
        const int n0 = seg * K, n1 = std::min(N, n0 + K);
        if (grads) ADJ_CUDA(save(ck + seg * state));
        stdg_stats st;
        ADJ_TRY(solver_step(c, dt, n1 - n0, &st));
        add_stats(st);
    }
    if (grads) ADJ_CUDA(save(ck + nseg * state));   // final state, restored at the end
    // ---- misfit on the host
    std::vector<double> rec((size_t)ns * N * per_rec);
    for (int s = 0; s < ns; ++s)
        ADJ_CUDA(cudaMemcpy(rec.data() + (size_t)s * N * per_rec, c->d_records + (s * c->rec_cap_steps + rec0) * per_rec,
                            sizeof(double) * N * per_rec, cudaMemcpyDeviceToHost));
    double L = 0.0;
    for (size_t i = 0; i < rec.size(); ++i) {
        const double r = rec[i] - data[i];
        L += 0.5 * r * r;
    }
    *loss = L;
    if (!grads) { cleanup(); return STDG_OK; }
    // ---- backward sweep
    double *Vb = nullptr, *Xb = nullptr, *av = nullptr, *as = nullptr, *lamJ = nullptr;
    double *glf = nullptr, *gmf = nullptr, *grho = nullptr, *dJ = nullptr;
    ADJ_TRY(alloc((void**)&d_data, sizeof(double) * ns * N * per_rec));
    ADJ_TRY(alloc((void**)&Vb, sizeof(double) * (size_t)K * ns * ntr));
    ADJ_TRY(alloc((void**)&Xb, sizeof(double) * (size_t)K * ns * nvel));
    ADJ_TRY(alloc((void**)&av, sizeof(double) * ns * ntr));
    ADJ_TRY(alloc((void**)&as, sizeof(double) * ns * nsig));
    ADJ_TRY(alloc((void**)&lamJ, sizeof(double) * ns * nvel));
    ADJ_TRY(alloc((void**)&glf, sizeof(double) * c->n_face));
    ADJ_TRY(alloc((void**)&gmf, sizeof(double) * c->n_face));
    ADJ_TRY(alloc((void**)&grho, sizeof(double) * c->n_elem));
    ADJ_TRY(alloc((void**)&dJ, sizeof(double) * c->n_elem));
    ADJ_CUDA(cudaMemcpyAsync(d_data, data, sizeof(double) * ns * N * per_rec, cudaMemcpyHostToDevice, c->stream));
    ADJ_CUDA(cudaMemcpyAsync(dJ, c->hm.detJ.data(), sizeof(double) * c->n_elem, cudaMemcpyHostToDevice, c->stream));
    ADJ_CUDA(cudaMemsetAsync(av, 0, sizeof(double) * ns * ntr, c->stream));
    ADJ_CUDA(cudaMemsetAsync(as, 0, sizeof(double) * ns * nsig, c->stream));
    ADJ_CUDA(cudaMemsetAsync(lamJ, 0, sizeof(double) * ns * nvel, c->stream));
    ADJ_CUDA(cudaMemsetAsync(glf, 0, sizeof(double) * c->n_face, c->stream));
    ADJ_CUDA(cudaMemsetAsync(gmf, 0, sizeof(double) * c->n_face, c->stream));
    ADJ_CUDA(cudaMemsetAsync(grho, 0, sizeof(double) * c->n_elem, c->stream));
    double* gsrc = nullptr;
    int32_t* selem = nullptr;
    std::vector<double> gl8(16);
    gauss_legendre01(8, gl8.data(), gl8.data() + 8);
    if (src_grad) {
        ADJ_TRY(alloc((void**)&gsrc, sizeof(double) * nsrc * d * NP));
        ADJ_TRY(alloc((void**)&selem, sizeof(int32_t) * nsrc));
        std::vector<int32_t> se(c->src_elem.begin(), c->src_elem.end());
        ADJ_CUDA(cudaMemcpyAsync(selem, se.data(), sizeof(int32_t) * nsrc, cudaMemcpyHostToDevice, c->stream));
        ADJ_CUDA(cudaMemsetAsync(gsrc, 0, sizeof(double) * nsrc * d * NP, c->stream));
        ADJ_CUDA(cudaStreamSynchronize(c->stream));   // the host vector se goes out of scope
    }
    // dt int_0^1 gamma_a(tau) S(t + tau dt) dtau at unit amplitude, 8-point Gauss-Legendre (as the forward RHS)
    auto time_integral = [&](double tn) {
        TimeInt ti{};
        const double a2 = -(M_PI * c->src_f0) * (M_PI * c->src_f0);
        for (int q = 0; q < 8; ++q) {
            double g[kMaxNG];
            lagrange_time(c->rt, gl8[q], g);
            const double u = tn + gl8[q] * dt - c->src_td;
            const double S = (0.5 + a2 * u * u) * std::exp(a2 * u * u);
            for (int a = 0; a < NG; ++a) ti.v[a] += dt * gl8[8 + q] * g[a] * S;
        }
        return ti;
    };
    const unsigned egrid = (unsigned)std::min<int64_t>((ns * nvel + 255) / 256, c->n_sm * 32);
    auto residual_into_av = [&](int n) {   // a_v += R^T (rec^n - d^n), n = 1..N
        const int64_t tot = (int64_t)ns * NR * d * NP;
        adj_receivers_kernel<<<(unsigned)std::min<int64_t>((tot + 255) / 256, c->n_sm * 8), 256, 0, c->stream>>>(
            ns, NR, d, NP, ntr, c->d_rec_elem, c->d_rec_phi, c->d_records + (rec0 + n - 1) * per_rec,
            c->rec_cap_steps * per_rec, d_data + (int64_t)(n - 1) * per_rec, (int64_t)N * per_rec, av);
        note_launch(c);
    };
    const double scale = dt * dt;   // c dt^2 with c = 1 (space-time DG)
    const int nsh = d == 2 ? 3 : 6;
    const size_t fsmem = sizeof(double) * 4 *
                         ((size_t)2 * d * NP * NP + 4 * (size_t)d * NG * NP + 2 * (size_t)d * d * NG * NP + nsh * NP);
    const size_t rsmem = sizeof(double) * 4 * ((size_t)2 * d * NP * NP + nsh * NP + (size_t)nsh * NG * NP);
    if (d == 2) {
        cudaFuncSetAttribute(adj_face_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
        cudaFuncSetAttribute(adj_rhs_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
    } else {
        cudaFuncSetAttribute(adj_face_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
        cudaFuncSetAttribute(adj_rhs_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
    }
    const unsigned fgrid = (unsigned)std::min<int64_t>((c->n_face + 3) / 4, c->n_sm * 16);
    // seed: a_v^N = R^T (rec^N - d^N), a_s^N = 0
    residual_into_av(N);
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int n0 = seg * K, n1 = std::min(N, n0 + K);
        // recompute the segment from its checkpoint, keeping v^n and x^{n+1}
        ADJ_CUDA(restore(ck + seg * state));
        for (int n = n0; n < n1; ++n) {
            ADJ_CUDA(cudaMemcpyAsync(Vb + (size_t)(n - n0) * ns * ntr, c->d_vtr, sizeof(double) * ns * ntr,
                                     cudaMemcpyDeviceToDevice, c->stream));
            c->t = t0 + n * dt;
            c->rec_steps = rec0 + n;
            stdg_stats st;
            ADJ_TRY(solver_step(c, dt, 1, &st));
            add_stats(st);
            ADJ_CUDA(cudaMemcpyAsync(Xb + (size_t)(n - n0) * ns * nvel, c->d_x, sizeof(double) * ns * nvel,
                                     cudaMemcpyDeviceToDevice, c->stream));
        }
        for (int n = n1 - 1; n >= n0; --n) {
            // right-hand side J a_x, a_x = g1 (x) a_v + Sx^T a_s (the adjoints of v^{n+1}, sigma^{n+1})
            adj_gamma_kernel<<<egrid, 256, 0, c->stream>>>(ns * c->n_elem * d, NP, NG, c->d_rt, av, c->d_b); note_launch(c);
            if (d == 2)
                adj_rhs_kernel<2><<<fgrid, 128, rsmem, c->stream>>>(c->n_face, ns, NP, NG, c->d_face_l, c->d_face_r, c->d_D,
                                                                    c->d_lamf, c->d_muf, c->d_rt, dt, as, c->d_b, nvel, nsig);
            else
                adj_rhs_kernel<3><<<fgrid, 128, rsmem, c->stream>>>(c->n_face, ns, NP, NG, c->d_face_l, c->d_face_r, c->d_D,
                                                                    c->d_lamf, c->d_muf, c->d_rt, dt, as, c->d_b, nvel, nsig);
            note_launch(c);
            // A (J lam) = J a_x, initial guess the previous slab's J lam
            ADJ_CUDA(cudaMemcpyAsync(c->d_x, lamJ, sizeof(double) * ns * nvel, cudaMemcpyDeviceToDevice, c->stream));
            stdg_stats st;
            ADJ_TRY(solver_solve(c, dt, &st));
            add_stats(st);
            ADJ_CUDA(cudaMemcpyAsync(lamJ, c->d_x, sizeof(double) * ns * nvel, cudaMemcpyDeviceToDevice, c->stream));
            const double* xn = Xb + (size_t)(n - n0) * ns * nvel;
            const double* vn = Vb + (size_t)(n - n0) * ns * ntr;
            adj_element_kernel<<<egrid, 256, 0, c->stream>>>(c->n_elem, ns, d, NP, NG, c->d_rt, c->d_rhoJ, dJ, lamJ, vn, xn,
                                                             av, grho); note_launch(c);
            if (src_grad) {   // lam^T ds^n/dtheta: the source enters b^n only
                const int64_t tot = (int64_t)nsrc * d * NP;
                adj_source_kernel<<<(unsigned)std::min<int64_t>((tot + 127) / 128, c->n_sm * 4), 128, 0, c->stream>>>(
                    nsrc, c->src_per_shot, d, NP, NG, selem, lamJ, nvel, time_integral(t0 + n * dt), gsrc);
                note_launch(c);
            }
            if (n >= 1) residual_into_av(n);
            if (d == 2)
                adj_face_kernel<2><<<fgrid, 128, fsmem, c->stream>>>(c->n_face, ns, NP, NG, c->d_face_l, c->d_face_r, c->d_D,
                                                                     c->d_rt, dt, scale, lamJ, xn, as, nvel, nsig, glf, gmf);
            else
                adj_face_kernel<3><<<fgrid, 128, fsmem, c->stream>>>(c->n_face, ns, NP, NG, c->d_face_l, c->d_face_r, c->d_D,
                                                                     c->d_rt, dt, scale, lamJ, xn, as, nvel, nsig, glf, gmf);
            note_launch(c);
            ADJ_CUDA(cudaGetLastError());
        }
    }
    // ---- dual-cell values to elements (sub-cell weights), rho directly
    std::vector<double> hl(c->n_face), hm_(c->n_face), hr(c->n_elem);
    ADJ_CUDA(cudaMemcpyAsync(hl.data(), glf, sizeof(double) * c->n_face, cudaMemcpyDeviceToHost, c->stream));
    ADJ_CUDA(cudaMemcpyAsync(hm_.data(), gmf, sizeof(double) * c->n_face, cudaMemcpyDeviceToHost, c->stream));
    ADJ_CUDA(cudaMemcpyAsync(hr.data(), grho, sizeof(double) * c->n_elem, cudaMemcpyDeviceToHost, c->stream));
    ADJ_CUDA(cudaStreamSynchronize(c->stream));
    if (g_lam) std::fill(g_lam, g_lam + c->n_elem, 0.0);
    if (g_mu) std::fill(g_mu, g_mu + c->n_elem, 0.0);
    for (int64_t f = 0; f < c->n_face; ++f) {
        const int64_t l = c->hm.face_l[f], r = c->hm.face_r[f];
        const double wl = c->hm.detJ[l], wr = r >= 0 ? c->hm.detJ[r] : 0.0;
        if (g_lam) { g_lam[l] += wl / (wl + wr) * hl[f]; if (r >= 0) g_lam[r] += wr / (wl + wr) * hl[f]; }
        if (g_mu) { g_mu[l] += wl / (wl + wr) * hm_[f]; if (r >= 0) g_mu[r] += wr / (wl + wr) * hm_[f]; }
    }
    if (g_rho) std::copy(hr.begin(), hr.end(), g_rho);
    if (g_src) {   // per source: [d/d amplitude, d/d direction (dim), d/d position (dim)]
        const int64_t nall = (int64_t)ns * c->src_per_shot;
        std::fill(g_src, g_src + nall * (1 + 2 * d), 0.0);
        if (src_grad) {
            std::vector<double> G((size_t)nsrc * d * NP), phi(NP), dphi((size_t)NP * d);
            ADJ_CUDA(cudaMemcpy(G.data(), gsrc, sizeof(double) * G.size(), cudaMemcpyDeviceToHost));
            for (int64_t q = 0; q < nsrc; ++q) {
                source_basis_host(c, q, phi.data(), dphi.data());
                const double* dir = c->src_dir.data() + q * d;
                const double* Gq = G.data() + q * d * NP;
                double* out = g_src + q * (1 + 2 * d);
                for (int l = 0; l < d; ++l) {
                    double gp = 0.0;
                    for (int n = 0; n < NP; ++n) gp += Gq[l * NP + n] * phi[n];
                    out[0] += dir[l] * gp;
                    out[1 + l] = c->src_a1 * gp;
                    for (int m = 0; m < d; ++m) {
                        double gd = 0.0;
                        for (int n = 0; n < NP; ++n) gd += Gq[l * NP + n] * dphi[n * d + m];
                        out[1 + d + m] += c->src_a1 * dir[l] * gd;
                    }
                }
            }
        }
    }
    // the context ends at the final time, as after a forward run
    ADJ_CUDA(restore(ck + nseg * state));
    c->t = t0 + N * dt;
    c->rec_steps = rec0 + N;
    cleanup();
    return STDG_OK;
#undef ADJ_TRY
#undef ADJ_CUDA
}

}  // namespace stdg
