// Device kernels of the staggered space-time DG scheme (arXiv:1802.04516, Sec. 4).
//
// Notation (per face j with neighbours l(j), r(j); per element i):
//   D_{i,j}[l][n][m]  spatial block of Eq. MD_3 (n: velocity node, m: dual mode)
//   M_j^{-1}          inverse dual mass matrix (Eq. MD_2)
//   time factors      W = diag(w_GL), T = gamma(1)gamma(1)^T - K, S = W T^{-1} W
// The Schur velocity operator of Eq. velocity.sys (Crank-Nicolson: Eq. velocity.sys.cn)
// is, with Q~ = -D^T (proof of Theorem 1) and constant E_j per dual cell,
//   (A v)_i = rho_i |J_i| (T (x) M_ref) v_i
//           + c dt^2 sum_{j in S_i} (D_{i,j} (x) I) S [ M_j^{-1} E_j : sum_{i'} (D_{i',j}^T v_{i'}) ]
// with c = 1 (space-time DG) or 1/4 (Crank-Nicolson).  The face kernel evaluates the
// bracket once per face and scatters to both neighbours; the mass kernel writes the
// element term first.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "stdg_internal.h"

namespace stdg {

// symmetric stress component c -> (a, b)
__constant__ int c_sym2[3][2] = {{0, 0}, {1, 1}, {0, 1}};
__constant__ int c_sym3[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {1, 2}, {0, 2}};

template <int DIM>
__device__ __forceinline__ void sym_ab(int c, int& a, int& b) {
    if (DIM == 2) { a = c_sym2[c][0]; b = c_sym2[c][1]; }
    else { a = c_sym3[c][0]; b = c_sym3[c][1]; }
}
template <int DIM>
__device__ __forceinline__ int sym_c(int a, int b) {
    if (a == b) return a;
    if (DIM == 2) return 2;
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return (lo == 0 && hi == 1) ? 3 : (lo == 1 ? 4 : 5);
}

// ---------------------------------------------------------------------------------
// Set-up: per (face, side) blocks D_{i,j} and sub-cell dual mass contributions
// (Eq. MD_3, Eq. MD_2), by a collapsed Gauss-Legendre rule on the sub-cell T_{i,j}
// and on Gamma_j.  One CTA per pair.
// ---------------------------------------------------------------------------------
template <int DIM>
__device__ void eval_monomials(const RefTables& rt, const double* xi, double* mono, double* grad /*[NP][DIM] or null*/) {
    double pw[3][8];
    for (int r = 0; r < DIM; ++r) {
        pw[r][0] = 1.0;
        for (int q = 1; q <= rt.p; ++q) pw[r][q] = pw[r][q - 1] * xi[r];
    }
    for (int a = 0; a < rt.Nphi; ++a) {
        double v = 1.0;
        for (int r = 0; r < DIM; ++r) v *= pw[r][rt.exps[a][r]];
        mono[a] = v;
        if (grad) {
            for (int r = 0; r < DIM; ++r) {
                int e = rt.exps[a][r];
                double g = e == 0 ? 0.0 : e * pw[r][e - 1];
                for (int s = 0; s < DIM; ++s) if (s != r) g *= pw[s][rt.exps[a][s]];
                grad[a * DIM + r] = g;
            }
        }
    }
}

constexpr int kChunk = 32;

template <int DIM>
__global__ void pair_blocks_kernel(const RefTables* __restrict__ rtp, int64_t n_face,
                                   const int32_t* __restrict__ face_l, const int32_t* __restrict__ face_r,
                                   const double* __restrict__ X, const double* __restrict__ Jinv,
                                   const double* __restrict__ faceX, const double* __restrict__ shift,
                                   const double* __restrict__ normal, const double* __restrict__ xc,
                                   const double* __restrict__ frame, const double* __restrict__ rule_v, int nq_v,
                                   const double* __restrict__ rule_f, int nq_f,
                                   double* __restrict__ D, double* __restrict__ Mdual) {
    extern __shared__ double sm[];
    const RefTables& rt = *rtp;
    const int NP = rt.Nphi;
    const int64_t f = blockIdx.x;
    const int side = blockIdx.y;
    if (f >= n_face) return;
    const int64_t nblk = (int64_t)DIM * NP * NP;
    double* Dout = D + (f * 2 + side) * nblk;
    const int e = side == 0 ? face_l[f] : face_r[f];
    if (e < 0) {
        for (int64_t t = threadIdx.x; t < nblk; t += blockDim.x) Dout[t] = 0.0;
        return;
    }
    const bool interior = face_r[f] >= 0;
    double* sD = sm;                          // DIM*NP*NP
    double* sM = sD + nblk;                   // NP*NP
    double* sW = sM + NP * NP;                // kChunk
    double* sPhi = sW + kChunk;               // kChunk*NP
    double* sGphi = sPhi + kChunk * NP;       // kChunk*NP*DIM
    double* sPsi = sGphi + kChunk * NP * DIM; // kChunk*NP
    for (int t = threadIdx.x; t < nblk; t += blockDim.x) sD[t] = 0.0;
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sM[t] = 0.0;

    // geometry of the sub-cell T_{e,j} in the frame of e
    constexpr int NV = DIM + 1;
    double V[NV][DIM], X0[DIM], Ji[DIM][DIM], off[DIM], nrm[DIM], cen[DIM];
    const double sgn = side == 0 ? 1.0 : -1.0;
    for (int a = 0; a < DIM; ++a) {
        off[a] = side == 0 ? 0.0 : shift[f * DIM + a];
        nrm[a] = sgn * normal[f * DIM + a];
        cen[a] = xc[f * DIM + a];
        X0[a] = X[((int64_t)e * NV) * DIM + a];
        double b = 0.0;
        for (int k = 0; k < NV; ++k) b += X[((int64_t)e * NV + k) * DIM + a];
        V[DIM][a] = b / NV;
        for (int q = 0; q < DIM; ++q) V[q][a] = faceX[(f * DIM + q) * DIM + a] - off[a];
        for (int r = 0; r < DIM; ++r) Ji[a][r] = Jinv[((int64_t)e * DIM + a) * DIM + r];
    }
    double Bf[DIM][DIM];   // dual basis: monomials of y = B_j (x - x_j), the principal axes of R_j
    for (int r = 0; r < DIM; ++r)
        for (int a = 0; a < DIM; ++a) Bf[r][a] = frame[(f * DIM + r) * DIM + a];
    // |det| of the sub-simplex edge matrix (the reference rule's weights sum to 1/DIM!)
    // vertices ordered (V0..V_{DIM-1} face, V_DIM barycentre): edges V1-V0 .. V_DIM - V0
    double E[DIM][DIM];
    for (int q = 0; q < DIM; ++q)
        for (int a = 0; a < DIM; ++a) E[q][a] = V[q + 1][a] - V[0][a];
    double detv = DIM == 2 ? E[0][0] * E[1][1] - E[0][1] * E[1][0]
                           : E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) - E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                                 E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
    detv = fabs(detv);
    // face measure factor: (DIM-1)! * measure = |F1-F0| (2D) or |(F1-F0)x(F2-F0)| (3D)
    double detf;
    if (DIM == 2) {
        double a0 = V[1][0] - V[0][0], a1 = V[1][1] - V[0][1];
        detf = sqrt(a0 * a0 + a1 * a1);
    } else {
        double u[3], w[3];
        for (int a = 0; a < 3; ++a) { u[a] = V[1][a] - V[0][a]; w[a] = V[2][a] - V[0][a]; }
        double c0 = u[1] * w[2] - u[2] * w[1], c1 = u[2] * w[0] - u[0] * w[2], c2 = u[0] * w[1] - u[1] * w[0];
        detf = sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    }
    __syncthreads();

    for (int pass = 0; pass < 2; ++pass) {
        const int nq = pass == 0 ? nq_v : (interior ? nq_f : 0);
        for (int q0 = 0; q0 < nq; q0 += kChunk) {
            const int nc = min(kChunk, nq - q0);
            for (int t = threadIdx.x; t < nc; t += blockDim.x) {
                double x[DIM];
                double w;
                if (pass == 0) {
                    const double* rp = rule_v + (int64_t)(q0 + t) * (DIM + 1);
                    for (int a = 0; a < DIM; ++a) {
                        x[a] = V[0][a];
                        for (int q = 0; q < DIM; ++q) x[a] += rp[q] * (V[q + 1][a] - V[0][a]);
                    }
                    w = rp[DIM] * detv;
                } else {
                    const double* rp = rule_f + (int64_t)(q0 + t) * DIM;
                    for (int a = 0; a < DIM; ++a) {
                        x[a] = V[0][a];
                        for (int q = 0; q < DIM - 1; ++q) x[a] += rp[q] * (V[q + 1][a] - V[0][a]);
                    }
                    w = rp[DIM - 1] * detf;
                }
                double xi[DIM], y[DIM];
                for (int r = 0; r < DIM; ++r) {
                    double s = 0.0, t = 0.0;
                    for (int a = 0; a < DIM; ++a) {
                        s += Ji[r][a] * (x[a] - X0[a]);
                        t += Bf[r][a] * (x[a] + off[a] - cen[a]);
                    }
                    xi[r] = s;
                    y[r] = t;
                }
                double mono[kMaxNP], gm[kMaxNP * DIM], ps[kMaxNP];
                eval_monomials<DIM>(rt, xi, mono, gm);
                eval_monomials<DIM>(rt, y, ps, nullptr);
                sW[t] = w;
                for (int k = 0; k < NP; ++k) {
                    double v = 0.0, g[DIM];
                    for (int r = 0; r < DIM; ++r) g[r] = 0.0;
                    for (int a = 0; a < NP; ++a) {
                        const double ck = rt.coef[a * NP + k];
                        v += ck * mono[a];
                        for (int r = 0; r < DIM; ++r) g[r] += ck * gm[a * DIM + r];
                    }
                    sPhi[t * NP + k] = v;
                    for (int l = 0; l < DIM; ++l) {
                        double s = 0.0;
                        for (int r = 0; r < DIM; ++r) s += g[r] * Ji[r][l];
                        sGphi[(t * NP + k) * DIM + l] = s;
                    }
                    sPsi[t * NP + k] = ps[k];
                }
            }
            __syncthreads();
            if (pass == 0) {
                for (int64_t ent = threadIdx.x; ent < nblk; ent += blockDim.x) {
                    const int l = (int)(ent / (NP * NP)), k = (int)((ent / NP) % NP), m = (int)(ent % NP);
                    double s = 0.0;
                    for (int t = 0; t < nc; ++t) s += sW[t] * sGphi[(t * NP + k) * DIM + l] * sPsi[t * NP + m];
                    sD[ent] -= s;
                }
                for (int ent = threadIdx.x; ent < NP * NP; ent += blockDim.x) {
                    const int k = ent / NP, m = ent % NP;
                    double s = 0.0;
                    for (int t = 0; t < nc; ++t) s += sW[t] * sPsi[t * NP + k] * sPsi[t * NP + m];
                    sM[ent] += s;
                }
            } else {
                for (int64_t ent = threadIdx.x; ent < nblk; ent += blockDim.x) {
                    const int l = (int)(ent / (NP * NP)), k = (int)((ent / NP) % NP), m = (int)(ent % NP);
                    double s = 0.0;
                    for (int t = 0; t < nc; ++t) s += sW[t] * sPhi[t * NP + k] * sPsi[t * NP + m];
                    sD[ent] += s * nrm[l];
                }
            }
            __syncthreads();
        }
    }
    for (int64_t t = threadIdx.x; t < nblk; t += blockDim.x) Dout[t] = sD[t];
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) atomicAdd(&Mdual[f * NP * NP + t], sM[t]);
}

cudaError_t launch_precompute(stdg_ctx* c, const double* d_rule_v, const double* d_rule_f, int nq_v, int nq_f) {
    const int NP = c->Nphi, DIM = c->dim;
    size_t smem = sizeof(double) * ((size_t)DIM * NP * NP + NP * NP + kChunk * (1 + NP + NP * DIM + NP));
    cudaMemsetAsync(c->d_Mdual, 0, sizeof(double) * c->n_face * NP * NP, c->stream);
    dim3 grid((unsigned)c->n_face, 2);
    if (DIM == 2) {
        cudaFuncSetAttribute(pair_blocks_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        pair_blocks_kernel<2><<<grid, 128, smem, c->stream>>>(c->d_rt, c->n_face, c->d_face_l, c->d_face_r, c->d_X, c->d_Jinv,
                                                              c->d_faceX, c->d_shift, c->d_normal, c->d_xc, c->d_frame,
                                                              d_rule_v, nq_v, d_rule_f, nq_f, c->d_D, c->d_Mdual); note_launch(c);
    } else {
        cudaFuncSetAttribute(pair_blocks_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        pair_blocks_kernel<3><<<grid, 128, smem, c->stream>>>(c->d_rt, c->n_face, c->d_face_l, c->d_face_r, c->d_X, c->d_Jinv,
                                                              c->d_faceX, c->d_shift, c->d_normal, c->d_xc, c->d_frame,
                                                              d_rule_v, nq_v, d_rule_f, nq_f, c->d_D, c->d_Mdual); note_launch(c);
    }
    return cudaGetLastError();
}

// Orthonormal dual basis per face: M_j = L_j L_j^T (Cholesky) and the blocks become
// D~_{i,j} = D_{i,j} L_j^{-T}, so that the dual mass matrix in the new basis is the identity.
// The Schur term D M^{-1} D^T = D~ D~^T is unchanged (it does not depend on the dual
// basis), but no M_j^{-1} is formed: its FP64 rounding grows like cond(M_j), which for
// Taylor monomials on sliver sub-cells exceeds 1e8, whereas D~ carries only
// ~sqrt(cond(M_j)) and is well scaled for an FP32 copy.  Stress states are kept as
// sigma~ = L_j^T sigma and converted at the API boundary.  One thread per face.
__global__ void orthonormalize_kernel(int64_t n_face, int NP, int DIM, const double* __restrict__ M,
                                      double* __restrict__ Lout, double* __restrict__ D, int* __restrict__ bad) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= n_face) return;
    double L[kMaxNP * kMaxNP];
    const double* A = M + f * NP * NP;
    for (int i = 0; i < NP; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = 0.5 * (A[i * NP + j] + A[j * NP + i]);
            for (int k = 0; k < j; ++k) s -= L[i * NP + k] * L[j * NP + k];
            if (i == j) {
                if (!(s > 0.0)) { atomicExch(bad, 1); s = 1.0; }
                L[i * NP + i] = sqrt(s);
            } else {
                L[i * NP + j] = s / L[j * NP + j];
            }
        }
    double* Lg = Lout + f * NP * NP;
    for (int i = 0; i < NP; ++i)
        for (int j = 0; j < NP; ++j) Lg[i * NP + j] = j <= i ? L[i * NP + j] : 0.0;
    // every row r = D[side][l][n][:] becomes L^{-1} r (forward substitution)
    double* Df = D + f * 2 * DIM * NP * NP;
    for (int row = 0; row < 2 * DIM * NP; ++row) {
        double* r = Df + row * NP;
        for (int i = 0; i < NP; ++i) {
            double s = r[i];
            for (int k = 0; k < i; ++k) s -= L[i * NP + k] * r[k];
            r[i] = s / L[i * NP + i];
        }
    }
}

cudaError_t launch_orthonormalize(stdg_ctx* c) {
    int* d_bad = nullptr;
    cudaError_t e = cudaMallocAsync(&d_bad, sizeof(int), c->stream);
    if (e != cudaSuccess) return e;
    cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream);
    orthonormalize_kernel<<<(unsigned)((c->n_face + 127) / 128), 128, 0, c->stream>>>(c->n_face, c->Nphi, c->dim, c->d_Mdual,
                                                                                    c->d_L, c->d_D, d_bad); note_launch(c);
    int bad = 0;
    cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    cudaFreeAsync(d_bad, c->stream);
    e = cudaGetLastError();
    if (e == cudaSuccess && bad) return cudaErrorInvalidValue;
    return e;
}

// Stress DOF conversion at the API boundary.  The caller's dual basis is the Taylor
// monomials psi_a = ((x - x_j)/h_j)^a; the library's internal one is psi'_b = (B_j (x - x_j))^b,
// the monomials in the principal-axis coordinates of R_j (same space P_p(R_j), well conditioned
// on thin dual cells), orthonormalised by L_j (dual mass matrix in psi', M'_j = L_j L_j^T).
// With y = G y' (G = B_j^{-1} / h_j), psi_a = sum_b E(G)[b][a] psi'_b, E(G)[b][a] the coefficient
// of y'^b in (G y')^a; the reverse substitution gives E(G^{-1}) = E(G)^{-1}.
//   dir 0 (Taylor -> orthonormal): sigma~ = L^T E(G) sigma_T
//   dir 1 (orthonormal -> Taylor): sigma_T = E(G^{-1}) L^{-T} sigma~
template <int DIM>
__device__ void substitution_matrix(const RefTables& rt, const double (&G)[DIM][DIM], double* E) {
    const int NP = rt.Npsi;
    for (int a = 0; a < NP; ++a) {
        double poly[kMaxNP], nw[kMaxNP];
        for (int b = 0; b < NP; ++b) poly[b] = 0.0;
        poly[0] = 1.0;                       // exps[0] is the constant monomial
        for (int r = 0; r < DIM; ++r)
            for (int t = 0; t < rt.exps[a][r]; ++t) {   // multiply by the linear form y_r = sum_s G[r][s] y'_s
                for (int b = 0; b < NP; ++b) nw[b] = 0.0;
                for (int b = 0; b < NP; ++b) {
                    if (poly[b] == 0.0) continue;
                    for (int s2 = 0; s2 < DIM; ++s2) {
                        const int k = rt.succ[b][s2];
                        if (k >= 0) nw[k] += G[r][s2] * poly[b];
                    }
                }
                for (int b = 0; b < NP; ++b) poly[b] = nw[b];
            }
        for (int b = 0; b < NP; ++b) E[b * NP + a] = poly[b];
    }
}

template <int DIM>
__global__ void sig_convert_kernel(int64_t n_face, const RefTables* __restrict__ rtp, const double* __restrict__ frame,
                                   const double* __restrict__ hj, const double* __restrict__ L,
                                   const double* __restrict__ in, double* __restrict__ out, int dir) {
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= n_face) return;
    const RefTables& rt = *rtp;
    const int NP = rt.Npsi, NS = rt.s;
    double B[DIM][DIM], G[DIM][DIM];
    for (int r = 0; r < DIM; ++r)
        for (int a = 0; a < DIM; ++a) B[r][a] = frame[(f * DIM + r) * DIM + a];
    const double h = hj[f];
    if (dir == 0) {   // G = B^{-1} / h by cofactors
        if (DIM == 2) {
            const double det = B[0][0] * B[1][1] - B[0][1] * B[1][0];
            G[0][0] = B[1][1] / (det * h); G[0][1] = -B[0][1] / (det * h);
            G[1][0] = -B[1][0] / (det * h); G[1][1] = B[0][0] / (det * h);
        } else {
            double cof[3][3];
            for (int r = 0; r < 3; ++r)
                for (int a = 0; a < 3; ++a) {
                    const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
                    cof[r][a] = B[r1][a1] * B[r2][a2] - B[r1][a2] * B[r2][a1];
                }
            const double det = B[0][0] * cof[0][0] + B[0][1] * cof[0][1] + B[0][2] * cof[0][2];
            for (int r = 0; r < 3; ++r)
                for (int a = 0; a < 3; ++a) G[r][a] = cof[a][r] / (det * h);
        }
    } else {
        for (int r = 0; r < DIM; ++r)
            for (int a = 0; a < DIM; ++a) G[r][a] = h * B[r][a];
    }
    double E[kMaxNP * kMaxNP];
    substitution_matrix<DIM>(rt, G, E);
    const double* Lf = L + f * NP * NP;
    for (int c2 = 0; c2 < NS; ++c2) {
        const double* a = in + (f * NS + c2) * NP;
        double* b = out + (f * NS + c2) * NP;
        double t[kMaxNP];
        if (dir == 0) {
            for (int m = 0; m < NP; ++m) {
                double s = 0;
                for (int k = 0; k < NP; ++k) s += E[m * NP + k] * a[k];
                t[m] = s;
            }
            for (int m = 0; m < NP; ++m) {
                double s = 0;
                for (int k = m; k < NP; ++k) s += Lf[k * NP + m] * t[k];
                b[m] = s;
            }
        } else {
            for (int m = NP - 1; m >= 0; --m) {
                double s = a[m];
                for (int k = m + 1; k < NP; ++k) s -= Lf[k * NP + m] * t[k];
                t[m] = s / Lf[m * NP + m];
            }
            for (int m = 0; m < NP; ++m) {
                double s = 0;
                for (int k = 0; k < NP; ++k) s += E[m * NP + k] * t[k];
                b[m] = s;
            }
        }
    }
}

cudaError_t launch_sig_convert(stdg_ctx* c, const double* in, double* out, int dir) {
    const unsigned g = (unsigned)((c->n_face + 127) / 128);
    if (c->dim == 2)
        sig_convert_kernel<2><<<g, 128, 0, c->stream>>>(c->n_face, c->d_rt, c->d_frame, c->d_hj, c->d_L, in, out, dir);
    else
        sig_convert_kernel<3><<<g, 128, 0, c->stream>>>(c->n_face, c->d_rt, c->d_frame, c->d_hj, c->d_L, in, out, dir);
    note_launch(c);
    return cudaGetLastError();
}

__global__ void to_fp32_kernel(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = (float)a[i];
}

cudaError_t launch_cast32(stdg_ctx* c, const double* a, float* b, int64_t n) {
    to_fp32_kernel<<<4096, 256, 0, c->stream>>>(n, a, b); note_launch(c);
    return cudaGetLastError();
}

cudaError_t launch_to_fp32(stdg_ctx* c) {
    const int64_t nD = c->n_face * 2 * c->dim * c->Nphi * c->Nphi;
    to_fp32_kernel<<<4096, 256, 0, c->stream>>>(nD, c->d_D, c->d_D32); note_launch(c);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Operator: element mass term and face (Schur) term.
// ---------------------------------------------------------------------------------
// y[e][k][a][n] = rho_i |J_i| sum_b T[a][b] sum_n' Mref[n][n'] v[e][k][b][n']
// n_elem = elements x shots of the (shot-major) vectors, n_elem_base = elements of the mesh.
// A block takes EB = blockDim / (d N_gamma) consecutive elements at a time: their values are
// loaded into shared memory with consecutive (coalesced) reads, each thread forms one row
// (k, a) of one element, the rows go back to the same shared buffer and out with consecutive
// writes.
template <int NP, typename R>
__global__ void __launch_bounds__(128) mass_kernel(int64_t n_elem, int64_t n_elem_base, int dim, int NG,
                                                   const RefTables* __restrict__ rtp, const R* __restrict__ rhoJ,
                                                   const R* __restrict__ v, const int* __restrict__ vidx, int64_t ld,
                                                   R* __restrict__ y) {
    if (vidx) v += (int64_t)(*vidx) * ld;
    extern __shared__ __align__(16) unsigned char mass_smem[];
    R* sV = reinterpret_cast<R*>(mass_smem);
    __shared__ R sM[NP * NP];
    __shared__ R sT[kMaxNG * kMaxNG];
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sM[t] = (R)rtp->Mref[t];
    for (int t = threadIdx.x; t < NG * NG; t += blockDim.x) sT[t] = (R)rtp->T[t];
    const int rows_e = dim * NG, per_e = rows_e * NP;
    const int EB = blockDim.x / rows_e;
    const int r = threadIdx.x, le = r / rows_e, ka = r % rows_e, k = ka / NG, a = ka % NG;
    for (int64_t e0 = blockIdx.x * (int64_t)EB; e0 < n_elem; e0 += (int64_t)gridDim.x * EB) {
        const int ne = (int)min((int64_t)EB, n_elem - e0);
        const int64_t base = e0 * per_e;
        __syncthreads();   // the previous elements' values have been written out
        for (int t = threadIdx.x; t < ne * per_e; t += blockDim.x) sV[t] = v[base + t];
        __syncthreads();
        const bool act = le < ne;
        R out[NP];
        if (act) {
            const R* ve = sV + (le * dim + k) * NG * NP;
            R tv[NP];
#pragma unroll
            for (int n = 0; n < NP; ++n) tv[n] = 0;
            for (int b = 0; b < NG; ++b) {
                const R tab = sT[a * NG + b];
#pragma unroll
                for (int n = 0; n < NP; ++n) tv[n] += tab * ve[b * NP + n];
            }
            const R sc = rhoJ[(e0 + le) % n_elem_base];
#pragma unroll
            for (int n = 0; n < NP; ++n) {
                R acc = 0;
#pragma unroll
                for (int q = 0; q < NP; ++q) acc += sM[n * NP + q] * tv[q];
                out[n] = sc * acc;
            }
        }
        __syncthreads();   // every row has read the element's values
        if (act) {
#pragma unroll
            for (int n = 0; n < NP; ++n) sV[r * NP + n] = out[n];   // row (e, k, a) of y
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne * per_e; t += blockDim.x) y[base + t] = sV[t];
    }
}

// Row-per-thread variant for stacked shots: thread (element, k, a) reads the element's rows
// directly; with many shots the grid streams long contiguous vectors and this form measured
// faster than the staged one (1.17 -> 0.91 ms per launch for 64 shots on 200,704 triangles).
template <int NP, typename R>
__global__ void mass_rows_kernel(int64_t n_elem, int64_t n_elem_base, int dim, int NG, const RefTables* __restrict__ rtp,
                                 const R* __restrict__ rhoJ, const R* __restrict__ v, const int* __restrict__ vidx,
                                 int64_t ld, R* __restrict__ y) {
    if (vidx) v += (int64_t)(*vidx) * ld;
    __shared__ R sM[NP * NP];
    __shared__ R sT[kMaxNG * kMaxNG];
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sM[t] = (R)rtp->Mref[t];
    for (int t = threadIdx.x; t < NG * NG; t += blockDim.x) sT[t] = (R)rtp->T[t];
    __syncthreads();
    const int per_e = dim * NG;          // rows of NP values per element
    const int64_t nrow = n_elem * per_e;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < nrow; row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = row / per_e;
        const int ka = (int)(row % per_e);
        const int k = ka / NG, a = ka % NG;
        const R* ve = v + (e * dim + k) * NG * NP;
        R tv[NP];
#pragma unroll
        for (int n = 0; n < NP; ++n) tv[n] = 0;
        for (int b = 0; b < NG; ++b) {
            const R tab = sT[a * NG + b];
#pragma unroll
            for (int n = 0; n < NP; ++n) tv[n] += tab * ve[b * NP + n];
        }
        const R s = rhoJ[e % n_elem_base];
        R* ye = y + row * NP;
#pragma unroll
        for (int n = 0; n < NP; ++n) {
            R acc = 0;
#pragma unroll
            for (int q = 0; q < NP; ++q) acc += sM[n * NP + q] * tv[q];
            ye[n] = s * acc;
        }
    }
}

// Shared-memory layout of one warp's face workspace (element counts).
struct FaceSmem {
    int D, v, g, t, h;
    int total;
};
__host__ __device__ inline FaceSmem face_smem(int dim, int NP, int NG) {
    FaceSmem s;
    const int ns = dim == 2 ? 3 : 6;
    s.D = 2 * dim * NP * NP;
    s.v = 2 * dim * NG * NP;
    s.g = dim * dim * NG * NP;
    s.t = ns * NG * NP;
    s.h = ns * NG * NP;
    s.total = s.D + s.v + s.g + s.t + s.h;
    return s;
}

// The per-face Schur bracket shared by the operator, the right-hand side and the
// stress update: from the two neighbours' velocities (in the warp's smem `v`) compute,
// with the orthonormalised blocks D~ (dual mass = identity),
//   g[k][l][b][m] = sum_side sum_n D~_side[l][n][m] v_side[k][b][n]     (D~^T v)
//   t[c][b][m]    = (E_j : g)_c = lam delta_ab tr g + mu (g_ab + g_ba)
template <int DIM, int NP, typename R>
__device__ __forceinline__ void face_bracket(int NG, int lane, const R* sD, const R* sv, R* sg, R* st, R lam, R mu) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    const int ng_np = NG * NP;
    const int nvs = DIM * ng_np;   // values per element
    for (int ent = lane; ent < DIM * DIM * ng_np; ent += 32) {
        const int k = ent / (DIM * ng_np);
        const int l = (ent / ng_np) % DIM;
        const int b = (ent / NP) % NG;
        const int m = ent % NP;
        R acc = 0;
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const R* Dp = sD + (side * DIM + l) * NP * NP + m;
            const R* vp = sv + side * nvs + (k * NG + b) * NP;
#pragma unroll
            for (int n = 0; n < NP; ++n) acc += Dp[n * NP] * vp[n];
        }
        sg[ent] = acc;
    }
    __syncwarp();
    for (int ent = lane; ent < NS * ng_np; ent += 32) {
        const int c = ent / ng_np;
        const int bm = ent % ng_np;
        int a, b;
        sym_ab<DIM>(c, a, b);
        R val = mu * (sg[(a * DIM + b) * ng_np + bm] + sg[(b * DIM + a) * ng_np + bm]);
        if (a == b) {
            R tr = 0;
#pragma unroll
            for (int q = 0; q < DIM; ++q) tr += sg[(q * DIM + q) * ng_np + bm];
            val += lam * tr;
        }
        st[ent] = val;
    }
    __syncwarp();
}

// Load the D~ blocks of face f into the warp's smem.
template <int DIM, int NP, typename R>
__device__ __forceinline__ void face_load_D(int64_t f, int lane, const R* __restrict__ D, R* sD) {
    const int nD = 2 * DIM * NP * NP;
    const R* Dg = D + f * nD;
    for (int t = lane; t < nD; t += 32) sD[t] = Dg[t];
}

// Load the neighbours' values of face f (midpoint average with x2 for Crank-Nicolson).
template <int DIM, int NP, typename R>
__device__ __forceinline__ void face_load_v(int NG, int lane, int el, int er, const R* __restrict__ x, R* sv,
                                            const R* __restrict__ x2 = nullptr) {
    const int nvs = DIM * NG * NP;
    for (int t = lane; t < nvs; t += 32) {
        R a = x[(int64_t)el * nvs + t];
        R b = er >= 0 ? x[(int64_t)er * nvs + t] : (R)0;
        if (x2) {
            a = (R)0.5 * (a + x2[(int64_t)el * nvs + t]);
            b = er >= 0 ? (R)0.5 * (b + x2[(int64_t)er * nvs + t]) : (R)0;
        }
        sv[t] = a;
        sv[nvs + t] = b;
    }
}

template <int DIM, int NP, typename R>
__device__ __forceinline__ void face_load(int64_t f, int NG, int lane, int el, int er, const R* __restrict__ D,
                                          const R* __restrict__ x, R* sD, R* sv, const R* __restrict__ x2 = nullptr) {
    face_load_D<DIM, NP, R>(f, lane, D, sD);
    face_load_v<DIM, NP, R>(NG, lane, el, er, x, sv, x2);
    __syncwarp();
}

// y_side += scale * sum_l sum_m D~_side[l][n][m] (S t)[(k,l)][b][m]
template <int DIM, int NP, typename R>
__global__ void __launch_bounds__(128) face_apply_kernel(int64_t n_face, int NG, const int32_t* __restrict__ fl,
                                                         const int32_t* __restrict__ fr, const R* __restrict__ D,
                                                         const R* __restrict__ lamf,
                                                         const R* __restrict__ muf, const RefTables* __restrict__ rtp,
                                                         const R* __restrict__ x, const int* __restrict__ xidx, int64_t ld,
                                                         R* __restrict__ y, R scale, int nshots, int64_t nvec) {
    if (xidx) x += (int64_t)(*xidx) * ld;
    extern __shared__ unsigned char smraw[];
    R* sm = reinterpret_cast<R*>(smraw);
    const FaceSmem L = face_smem(DIM, NP, NG);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    R* sS = sm;                                     // NG*NG
    R* base = sm + kMaxNG * kMaxNG + warp * L.total;
    R *sD = base, *sv = sD + L.D, *sg = sv + L.v, *st = sg + L.g, *sh = st + L.t;
    for (int t = threadIdx.x; t < NG * NG; t += blockDim.x) sS[t] = (R)rtp->S[t];
    __syncthreads();
    constexpr int NS = DIM == 2 ? 3 : 6;
    const int ng_np = NG * NP;
    const int nvs = DIM * ng_np;
    for (int64_t f = blockIdx.x * (int64_t)wpb + warp; f < n_face; f += (int64_t)gridDim.x * wpb) {
        const int el = fl[f], er = fr[f];
        const R lam = lamf[f], mu = muf[f];
        face_load_D<DIM, NP, R>(f, lane, D, sD);   // once per face, reused by every shot
        for (int s = 0; s < nshots; ++s) {
            const R* xs = x + (int64_t)s * nvec;
            R* ys = y + (int64_t)s * nvec;
            face_load_v<DIM, NP, R>(NG, lane, el, er, xs, sv);
            __syncwarp();
            face_bracket<DIM, NP, R>(NG, lane, sD, sv, sg, st, lam, mu);
            // time factor S and scale: h = scale * S t
            for (int ent = lane; ent < NS * ng_np; ent += 32) {
                const int c = ent / ng_np, b = (ent / NP) % NG, m = ent % NP;
                R acc = 0;
                for (int b2 = 0; b2 < NG; ++b2) acc += sS[b * NG + b2] * st[(c * NG + b2) * NP + m];
                sh[ent] = scale * acc;
            }
            __syncwarp();
            const int nside = er >= 0 ? 2 : 1;
            for (int ent = lane; ent < nside * nvs; ent += 32) {
                const int side = ent / nvs;
                const int r = ent % nvs;
                const int k = r / ng_np, b = (r / NP) % NG, n = r % NP;
                R acc = 0;
#pragma unroll
                for (int l = 0; l < DIM; ++l) {
                    const R* Dp = sD + ((side * DIM + l) * NP + n) * NP;
                    const R* hp = sh + (sym_c<DIM>(k, l) * NG + b) * NP;
#pragma unroll
                    for (int m = 0; m < NP; ++m) acc += Dp[m] * hp[m];
                }
                const int e = side == 0 ? el : er;
                atomicAdd(&ys[(int64_t)e * nvs + r], acc);
            }
            __syncwarp();
        }
    }
}

template <int DIM, int NP, typename R>
static cudaError_t apply_tmpl(stdg_ctx* c, const R* D, const R* lamf, const R* muf, const R* rhoJ,
                              const R* x, R* y, double scale, bool mass, bool face = true,
                              const int* xidx = nullptr, int64_t ld = 0, int nshots = 1) {
    const int NG = c->Ng;
    if (mass) {
        const int64_t rows = c->n_elem * nshots * c->dim * NG;
        const int64_t ne = c->n_elem * nshots;
        if (nshots > 1) {
            mass_rows_kernel<NP, R><<<(unsigned)std::min<int64_t>((rows + 127) / 128, c->n_sm * 64), 128, 0, c->stream>>>(
                ne, c->n_elem, c->dim, NG, c->d_rt, rhoJ, x, xidx, ld, y); note_launch(c);
        } else {
            const int EB = 128 / (c->dim * NG);   // elements per block and pass (d N_gamma <= 15)
            const size_t smem = sizeof(R) * (size_t)EB * c->dim * NG * NP;
            mass_kernel<NP, R><<<(unsigned)std::min<int64_t>((ne + EB - 1) / EB, (int64_t)c->n_sm * 16), 128, smem,
                                 c->stream>>>(ne, c->n_elem, c->dim, NG, c->d_rt, rhoJ, x, xidx, ld, y); note_launch(c);
        }
    }
    if (!face) return cudaGetLastError();
    cudaError_t fe;
    if (launch_face_fast<R>(c, D, lamf, muf, x, xidx, ld, y, scale, &fe, nshots)) return fe;
    const FaceSmem L = face_smem(DIM, NP, NG);
    const int wpb = 4;
    size_t smem = sizeof(R) * (kMaxNG * kMaxNG + (size_t)wpb * L.total);
    cudaFuncSetAttribute(face_apply_kernel<DIM, NP, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int64_t blocks = (c->n_face + wpb - 1) / wpb;
    face_apply_kernel<DIM, NP, R><<<(unsigned)std::min<int64_t>(blocks, 1 << 30), 32 * wpb, smem, c->stream>>>(
        c->n_face, NG, c->d_face_l, c->d_face_r, D, lamf, muf, c->d_rt, x, xidx, ld, y, (R)scale, nshots, c->nvel);
    note_launch(c);
    return cudaGetLastError();
}

#define STDG_DISPATCH(DIMV, NPV, ...)                                             \
    do {                                                                         \
        if (DIMV == 2) {                                                         \
            switch (NPV) {                                                       \
                case 3: { constexpr int D_ = 2, N_ = 3; __VA_ARGS__; } break;          \
                case 6: { constexpr int D_ = 2, N_ = 6; __VA_ARGS__; } break;          \
                case 10: { constexpr int D_ = 2, N_ = 10; __VA_ARGS__; } break;        \
                case 15: { constexpr int D_ = 2, N_ = 15; __VA_ARGS__; } break;        \
                default: return cudaErrorInvalidValue;                           \
            }                                                                    \
        } else {                                                                 \
            switch (NPV) {                                                       \
                case 4: { constexpr int D_ = 3, N_ = 4; __VA_ARGS__; } break;          \
                case 10: { constexpr int D_ = 3, N_ = 10; __VA_ARGS__; } break;        \
                case 20: { constexpr int D_ = 3, N_ = 20; __VA_ARGS__; } break;        \
                default: return cudaErrorInvalidValue;                           \
            }                                                                    \
        }                                                                        \
    } while (0)

static double schur_c(const stdg_ctx* c) { return c->opt.scheme == STDG_SCHEME_CN ? 0.25 : 1.0; }

cudaError_t launch_apply(stdg_ctx* c, double dt, const double* x, double* y, double cfac, const int* xidx, int64_t ld,
                         int nshots) {
    const double scale = cfac * schur_c(c) * dt * dt;
    STDG_DISPATCH(c->dim, c->Nphi, return (apply_tmpl<D_, N_, double>(c, c->d_D, c->d_lamf, c->d_muf, c->d_rhoJ, x, y, scale, true, true, xidx, ld, nshots)));
    return cudaSuccess;
}

cudaError_t launch_apply32(stdg_ctx* c, double dt, const float* x, float* y, double cfac, const int* xidx, int64_t ld,
                           int nshots) {
    const double scale = cfac * schur_c(c) * dt * dt;
    STDG_DISPATCH(c->dim, c->Nphi, return (apply_tmpl<D_, N_, float>(c, c->d_D32, c->d_lamf32, c->d_muf32, c->d_rhoJ32, x, y, scale, true, true, xidx, ld, nshots)));
    return cudaSuccess;
}

cudaError_t launch_face_only(stdg_ctx* c, double dt, const void* x, void* y, double cfac, int fp32) {
    const double scale = cfac * schur_c(c) * dt * dt;
    if (fp32) {
        STDG_DISPATCH(c->dim, c->Nphi, return (apply_tmpl<D_, N_, float>(c, c->d_D32, c->d_lamf32, c->d_muf32, c->d_rhoJ32, (const float*)x, (float*)y, scale, false)));
    } else {
        STDG_DISPATCH(c->dim, c->Nphi, return (apply_tmpl<D_, N_, double>(c, c->d_D, c->d_lamf, c->d_muf, c->d_rhoJ, (const double*)x, (double*)y, scale, false)));
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------------------------
// Right-hand side (Eq. velocity.sys / velocity.sys.cn), per shot.
// dparams (device): [0] = t^n, [1] = dt, [2] = step index
// ---------------------------------------------------------------------------------
// Element part.  Space-time DG: b[e][k][a][n] = rho|J| g0[a] (Mref vtr[e][k])[n].
template <int NP>
__global__ void rhs_mass_stdg_kernel(int64_t n_elem, int dim, int NG, const RefTables* __restrict__ rtp,
                                     const double* __restrict__ rhoJ, const double* __restrict__ vtr, double* __restrict__ b) {
    __shared__ double sM[NP * NP];
    for (int t = threadIdx.x; t < NP * NP; t += blockDim.x) sM[t] = rtp->Mref[t];
    __syncthreads();
    const int64_t nrow = n_elem * dim;
    for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < nrow; row += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = row / dim;
        const double* vp = vtr + row * NP;
        double tv[NP];
#pragma unroll
        for (int n = 0; n < NP; ++n) {
            double acc = 0;
#pragma unroll
            for (int q = 0; q < NP; ++q) acc += sM[n * NP + q] * vp[q];
            tv[n] = rhoJ[e] * acc;
        }
        for (int a = 0; a < NG; ++a) {
            const double g = rtp->g0[a];
            double* bp = b + (row * NG + a) * NP;
#pragma unroll
            for (int n = 0; n < NP; ++n) bp[n] = g * tv[n];
        }
    }
}

// Face part: b_side[k][a][n] += coef[a] sum_l sum_m D_side[l][n][m] sigma_tr[(k,l)][m],
// coef[a] = dt W[a] (T^{-1} g0)[a]  (space-time DG)  or dt  (Crank-Nicolson).
template <int DIM, int NP>
__global__ void __launch_bounds__(128) rhs_face_kernel(int64_t n_face, int NG, const int32_t* __restrict__ fl,
                                                       const int32_t* __restrict__ fr, const double* __restrict__ D,
                                                       const RefTables* __restrict__ rtp, double dt,
                                                       const double* __restrict__ sigtr, double* __restrict__ b) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    constexpr int PER = 2 * DIM * NP * NP + NS * NP;
    extern __shared__ unsigned char smraw[];
    double* sm = reinterpret_cast<double*>(smraw);
    __shared__ double sCoef[kMaxNG];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double* sD = sm + warp * PER;
    double* sSig = sD + 2 * DIM * NP * NP;
    if (threadIdx.x < NG) sCoef[threadIdx.x] = rtp->pg == 0 ? dt : dt * rtp->W[threadIdx.x] * rtp->Tinv_g0[threadIdx.x];
    __syncthreads();
    const int nvs = DIM * NG * NP;
    for (int64_t f = blockIdx.x * 4LL + warp; f < n_face; f += (int64_t)gridDim.x * 4) {
        const int el = fl[f], er = fr[f];
        for (int t = lane; t < 2 * DIM * NP * NP; t += 32) sD[t] = D[f * 2 * DIM * NP * NP + t];
        for (int t = lane; t < NS * NP; t += 32) sSig[t] = sigtr[f * NS * NP + t];
        __syncwarp();
        const int nside = er >= 0 ? 2 : 1;
        for (int ent = lane; ent < nside * DIM * NP; ent += 32) {
            const int side = ent / (DIM * NP), k = (ent / NP) % DIM, n = ent % NP;
            double acc = 0;
#pragma unroll
            for (int l = 0; l < DIM; ++l) {
                const double* Dp = sD + ((side * DIM + l) * NP + n) * NP;
                const double* sp = sSig + sym_c<DIM>(k, l) * NP;
#pragma unroll
                for (int m = 0; m < NP; ++m) acc += Dp[m] * sp[m];
            }
            const int e = side == 0 ? el : er;
            for (int a = 0; a < NG; ++a) atomicAdd(&b[(int64_t)e * nvs + (k * NG + a) * NP + n], sCoef[a] * acc);
        }
        __syncwarp();
    }
}

// Point source (Sec. 6.3): b[e_s][k][a][n] += dir_k phi_n(x_s) dt int_0^1 gamma_a(tau) S(t^n + tau dt) dtau.
__global__ void rhs_source_kernel(int dim, int NP, int NG, const RefTables* __restrict__ rtp, const double* __restrict__ dparams,
                                  int32_t elem, const double* __restrict__ src /*dir[dim], phi[NP]*/, double f0, double td,
                                  double a1, const double* __restrict__ gl /*8 nodes, 8 weights*/, double* __restrict__ b) {
    const double t0 = dparams[0], dt = dparams[1];
    __shared__ double tint[kMaxNG];
    if (threadIdx.x < NG) {
        const int a = threadIdx.x;
        const double a2 = -(M_PI * f0) * (M_PI * f0);
        double s = 0.0;
        for (int q = 0; q < 8; ++q) {
            const double tau = gl[q];
            double g = 1.0;
            for (int c = 0; c < NG; ++c)
                if (c != a) g *= (tau - rtp->tnodes[c]) / (rtp->tnodes[a] - rtp->tnodes[c]);
            const double u = t0 + tau * dt - td;
            s += gl[8 + q] * g * a1 * (0.5 + a2 * u * u) * exp(a2 * u * u);
        }
        tint[a] = dt * s;
    }
    __syncthreads();
    const int nvs = dim * NG * NP;
    for (int t = threadIdx.x; t < nvs; t += blockDim.x) {
        const int k = t / (NG * NP), a = (t / NP) % NG, n = t % NP;
        b[(int64_t)elem * nvs + t] += src[k] * src[dim + n] * tint[a];
    }
}

template <int NP>
static void rhs_mass_stdg(stdg_ctx* c, const double* vtr, double* b) {
    const int64_t rows = c->n_elem * c->dim;
    rhs_mass_stdg_kernel<NP><<<(unsigned)std::min<int64_t>((rows + 127) / 128, c->n_sm * 64), 128, 0, c->stream>>>(
        c->n_elem, c->dim, c->Ng, c->d_rt, c->d_rhoJ, vtr, b); note_launch(c);
}

cudaError_t launch_rhs(stdg_ctx* c, double dt, const double* dparams, int shot, double* b) {
    const int NP = c->Nphi, NG = c->Ng;
    const double* vtr = c->d_vtr + shot * c->ntr;
    const double* sig = c->d_sigtr + shot * c->nsig;
    if (c->opt.scheme == STDG_SCHEME_CN) {
        // b = 2 rho Mbar v^n - A v^n + dt sum D sigma^n + src = mass(v^n) - face(v^n) + ...
        // (N_gamma = 1, so the trace layout equals the slab layout)
        const double scale = -0.25 * dt * dt;
        STDG_DISPATCH(c->dim, NP, {
            cudaError_t e = apply_tmpl<D_, N_, double>(c, c->d_D, c->d_lamf, c->d_muf, c->d_rhoJ, vtr, b, scale, true);
            if (e != cudaSuccess) return e;
        });
    } else {
        switch (NP) {
            case 3: rhs_mass_stdg<3>(c, vtr, b); break;
            case 4: rhs_mass_stdg<4>(c, vtr, b); break;
            case 6: rhs_mass_stdg<6>(c, vtr, b); break;
            case 10: rhs_mass_stdg<10>(c, vtr, b); break;
            case 15: rhs_mass_stdg<15>(c, vtr, b); break;
            case 20: rhs_mass_stdg<20>(c, vtr, b); break;
            default: return cudaErrorInvalidValue;
        }
    }
    STDG_DISPATCH(c->dim, NP, ({
        const int ns = D_ == 2 ? 3 : 6;
        size_t smem = sizeof(double) * 4 * (size_t)(2 * D_ * N_ * N_ + ns * N_);
        cudaFuncSetAttribute(rhs_face_kernel<D_, N_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        rhs_face_kernel<D_, N_><<<(unsigned)std::min<int64_t>((c->n_face + 3) / 4, 1 << 30), 128, smem, c->stream>>>(
            c->n_face, NG, c->d_face_l, c->d_face_r, c->d_D, c->d_rt, dt, sig, b); note_launch(c);
    }));
    for (int q = 0; c->have_sources && q < c->src_per_shot; ++q) {   // sequential: sources may share an element
        const int64_t sq = (int64_t)shot * c->src_per_shot + q;
        // a source in a part with time scale alpha sees its wavelet in that part's scaled time
        const double al = c->src_alpha.empty() ? 1.0 : c->src_alpha[sq];
        rhs_source_kernel<<<1, 128, 0, c->stream>>>(c->dim, NP, NG, c->d_rt, dparams, (int32_t)c->src_elem[sq],
                                                     c->d_src + sq * (c->dim + NP), c->src_f0 * al, c->src_td / al,
                                                     c->src_a1, c->d_gl8, b); note_launch(c);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Stress back-substitution (Eq. NM26 / NM26.cn) written directly as the new trace:
//   sigma_tr <- kappa sigma_tr - dt sum_b u_tr[b] (M_j^{-1} E_j : g)[c][b]
// with kappa = gamma(1)^T T^{-1} gamma(0), u_tr = gamma(1)^T T^{-1} W (both 1 for CN,
// where the velocity is the midpoint (v^n + v^{n+1})/2).
// ---------------------------------------------------------------------------------
template <int DIM, int NP>
__global__ void __launch_bounds__(128) stress_kernel(int64_t n_face, int NG, const int32_t* __restrict__ fl,
                                                     const int32_t* __restrict__ fr, const double* __restrict__ D,
                                                     const double* __restrict__ lamf,
                                                     const double* __restrict__ muf, const RefTables* __restrict__ rtp,
                                                     double dt, const double* __restrict__ x,
                                                     const double* __restrict__ x_old, double* __restrict__ sigtr) {
    extern __shared__ unsigned char smraw[];
    double* sm = reinterpret_cast<double*>(smraw);
    const FaceSmem L = face_smem(DIM, NP, NG);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpb = blockDim.x >> 5;
    double* base = sm + warp * L.total;
    double *sD = base, *sv = sD + L.D, *sg = sv + L.v, *st = sg + L.g;
    constexpr int NS = DIM == 2 ? 3 : 6;
    for (int64_t f = blockIdx.x * (int64_t)wpb + warp; f < n_face; f += (int64_t)gridDim.x * wpb) {
        const int el = fl[f], er = fr[f];
        face_load<DIM, NP, double>(f, NG, lane, el, er, D, x, sD, sv, x_old);
        face_bracket<DIM, NP, double>(NG, lane, sD, sv, sg, st, lamf[f], muf[f]);
        for (int ent = lane; ent < NS * NP; ent += 32) {
            const int cc = ent / NP, m = ent % NP;
            double acc = 0;
            for (int b = 0; b < NG; ++b) acc += rtp->u_tr[b] * st[(cc * NG + b) * NP + m];
            double* sp = sigtr + f * NS * NP + ent;
            *sp = rtp->kappa * (*sp) - dt * acc;
        }
        __syncwarp();
    }
}

cudaError_t launch_stress_update(stdg_ctx* c, double dt, int shot, const double* x) {
    const int NG = c->Ng;
    const double* x_old = c->opt.scheme == STDG_SCHEME_CN ? c->d_vtr + shot * c->ntr : nullptr;
    double* sig = c->d_sigtr + shot * c->nsig;
    STDG_DISPATCH(c->dim, c->Nphi, ({
        const FaceSmem L = face_smem(D_, N_, NG);
        const int wpb = 4;
        size_t smem = sizeof(double) * (size_t)wpb * L.total;
        cudaFuncSetAttribute(stress_kernel<D_, N_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        stress_kernel<D_, N_><<<(unsigned)std::min<int64_t>((c->n_face + wpb - 1) / wpb, 1 << 30), 32 * wpb, smem, c->stream>>>(
            c->n_face, NG, c->d_face_l, c->d_face_r, c->d_D, c->d_lamf, c->d_muf, c->d_rt, dt, x, x_old, sig); note_launch(c);
    }));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Traces, initial guess, receivers, energy
// ---------------------------------------------------------------------------------
__global__ void traces_kernel(int64_t nrows, int NP, int NG, const RefTables* __restrict__ rtp, const double* __restrict__ x,
                              double* __restrict__ vtr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows * NP; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / NP;
        const int n = (int)(i % NP);
        double s = 0;
        for (int a = 0; a < NG; ++a) s += rtp->g1[a] * x[(row * NG + a) * NP + n];
        vtr[i] = s;
    }
}

cudaError_t launch_traces(stdg_ctx* c, int shot, const double* x) {
    const int64_t rows = c->n_elem * c->dim;
    traces_kernel<<<(unsigned)std::min<int64_t>((rows * c->Nphi + 255) / 256, c->n_sm * 32), 256, 0, c->stream>>>(
        rows, c->Nphi, c->Ng, c->d_rt, x, c->d_vtr + shot * c->ntr); note_launch(c);
    return cudaGetLastError();
}

__global__ void initial_guess_kernel(int64_t nrows, int NP, int NG, const double* __restrict__ vtr, double* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nrows * NG * NP; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / (NG * NP);
        const int n = (int)(i % NP);
        x[i] = vtr[row * NP + n];
    }
}

cudaError_t launch_initial_guess(stdg_ctx* c, int shot, double* x) {
    const int64_t rows = c->n_elem * c->dim;
    initial_guess_kernel<<<(unsigned)std::min<int64_t>((rows * c->Ng * c->Nphi + 255) / 256, c->n_sm * 32), 256, 0, c->stream>>>(
        rows, c->Nphi, c->Ng, c->d_vtr + shot * c->ntr, x); note_launch(c);
    return cudaGetLastError();
}

__global__ void receivers_kernel(int n_rec, int dim, int NP, const int32_t* __restrict__ elem, const double* __restrict__ phi,
                                 const double* __restrict__ vtr, const double* __restrict__ dparams, int64_t cap_steps,
                                 double* __restrict__ out) {
    const int64_t step = (int64_t)dparams[2];
    if (step >= cap_steps) return;
    for (int i = threadIdx.x; i < n_rec * dim; i += blockDim.x) {
        const int r = i / dim, k = i % dim;
        const double* vp = vtr + ((int64_t)elem[r] * dim + k) * NP;
        double s = 0;
        for (int n = 0; n < NP; ++n) s += phi[r * NP + n] * vp[n];
        out[(step * n_rec + r) * dim + k] = s;
    }
}

cudaError_t launch_receivers(stdg_ctx* c, const double* dparams, int shot) {
    if (c->n_rec == 0) return cudaSuccess;
    receivers_kernel<<<1, 256, 0, c->stream>>>(c->n_rec, c->dim, c->Nphi, c->d_rec_elem, c->d_rec_phi, c->d_vtr + shot * c->ntr,
                                                dparams, c->rec_cap_steps,
                                                c->d_records + (int64_t)shot * c->rec_cap_steps * c->n_rec * c->dim); note_launch(c);
    return cudaGetLastError();
}

// Energy (Eq. SP3F): 1/2 sum_i rho_i |J_i| v^T Mref v + 1/2 sum_j int_{R_j} sigma : E_j^{-1} sigma.
// With the orthonormal dual basis the dual mass matrix is the identity, so the elastic
// part is a plain sum over modes of sigma~ : E_j^{-1} sigma~.
template <int DIM>
__global__ void energy_kernel(int64_t n_elem, int64_t n_face, int NP, const RefTables* __restrict__ rtp,
                              const double* __restrict__ rhoJ, const double* __restrict__ vtr,
                              const double* __restrict__ lamf, const double* __restrict__ muf, const double* __restrict__ sigtr,
                              double* __restrict__ out) {
    constexpr int NS = DIM == 2 ? 3 : 6;
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_elem * DIM; i += (int64_t)gridDim.x * blockDim.x) {
        const double* vp = vtr + i * NP;
        double s = 0;
        for (int n = 0; n < NP; ++n) {
            double t = 0;
            for (int q = 0; q < NP; ++q) t += rtp->Mref[n * NP + q] * vp[q];
            s += vp[n] * t;
        }
        acc += 0.5 * rhoJ[i / DIM] * s;
    }
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n_face; f += (int64_t)gridDim.x * blockDim.x) {
        const double* sp = sigtr + f * NS * NP;
        const double lam = lamf[f], mu = muf[f];
        const double coef = lam / (DIM * lam + 2.0 * mu);
        // E^{-1} sigma = (sigma - coef tr(sigma) I) / (2 mu); off-diagonal components count twice
        double s = 0;
        for (int m = 0; m < NP; ++m) {
            double tr = 0;
            for (int a = 0; a < DIM; ++a) tr += sp[a * NP + m];
            for (int c2 = 0; c2 < NS; ++c2) s += (c2 < DIM ? 1.0 : 2.0) * sp[c2 * NP + m] * sp[c2 * NP + m];
            s -= coef * tr * tr;
        }
        acc += 0.5 * s / (2.0 * mu);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        atomicAdd(out, s);
    }
}

cudaError_t launch_energy(stdg_ctx* c, int shot, double* d_out) {
    cudaMemsetAsync(d_out, 0, sizeof(double), c->stream);
    // physical material when a time scale is set (the operator's copies are scaled)
    const double* rhoJ = c->d_rhoJ_ph ? c->d_rhoJ_ph : c->d_rhoJ;
    const double* lamf = c->d_lamf_ph ? c->d_lamf_ph : c->d_lamf;
    const double* muf = c->d_muf_ph ? c->d_muf_ph : c->d_muf;
    if (c->dim == 2) {
        energy_kernel<2><<<c->n_sm * 4, 256, 0, c->stream>>>(c->n_elem, c->n_face, c->Nphi, c->d_rt, rhoJ, c->d_vtr + shot * c->ntr,
                                                         lamf, muf, c->d_sigtr + shot * c->nsig, d_out);
    } else {
        energy_kernel<3><<<c->n_sm * 4, 256, 0, c->stream>>>(c->n_elem, c->n_face, c->Nphi, c->d_rt, rhoJ, c->d_vtr + shot * c->ntr,
                                                         lamf, muf, c->d_sigtr + shot * c->nsig, d_out);
    }
    note_launch(c);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// Plane-wave initial data (Eqs. NT2.1, NT2.2): L2 projections onto both bases.
// ---------------------------------------------------------------------------------
struct PlaneWave {
    double k[3], rv[3], rs[3][3], omega, amp, t;
};

template <int DIM>
__device__ void pw_eval(const PlaneWave& pw, const double* x, double* v, double s[3][3]) {
    double ph = -pw.omega * pw.t;
    for (int a = 0; a < DIM; ++a) ph += pw.k[a] * x[a];
    const double sn = pw.amp * sin(ph);
    for (int a = 0; a < DIM; ++a) {
        v[a] = sn * pw.rv[a];
        for (int b = 0; b < DIM; ++b) s[a][b] = sn * pw.rs[a][b];
    }
}

template <int DIM>
__global__ void project_vel_kernel(int64_t n_elem, const RefTables* __restrict__ rtp, const double* __restrict__ X,
                                   const double* __restrict__ detJ, PlaneWave pw, const double* __restrict__ rule, int nq,
                                   double* __restrict__ vtr) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_elem) return;
    const RefTables& rt = *rtp;
    const int NP = rt.Nphi;
    constexpr int NV = DIM + 1;
    double acc[3][kMaxNP];
    for (int k = 0; k < DIM; ++k)
        for (int n = 0; n < NP; ++n) acc[k][n] = 0;
    for (int q = 0; q < nq; ++q) {
        const double* rp = rule + q * (DIM + 1);
        double x[DIM];
        for (int a = 0; a < DIM; ++a) {
            x[a] = X[(e * NV) * DIM + a];
            for (int r = 0; r < DIM; ++r) x[a] += rp[r] * (X[(e * NV + r + 1) * DIM + a] - X[(e * NV) * DIM + a]);
        }
        double mono[kMaxNP];
        eval_monomials<DIM>(rt, rp, mono, nullptr);
        double v[3], s[3][3];
        pw_eval<DIM>(pw, x, v, s);
        for (int n = 0; n < NP; ++n) {
            double phi = 0;
            for (int a = 0; a < NP; ++a) phi += rt.coef[a * NP + n] * mono[a];
            for (int k = 0; k < DIM; ++k) acc[k][n] += rp[DIM] * phi * v[k];
        }
    }
    for (int k = 0; k < DIM; ++k)
        for (int n = 0; n < NP; ++n) {
            double s = 0;
            for (int q = 0; q < NP; ++q) s += rt.MrefInv[n * NP + q] * acc[k][q];
            vtr[(e * DIM + k) * NP + n] = s;   // (|J| Mref)^{-1} |J| int_ref phi v
        }
}

template <int DIM>
__global__ void project_sig_kernel(int64_t n_face, const RefTables* __restrict__ rtp, const int32_t* __restrict__ fl,
                                   const int32_t* __restrict__ fr, const double* __restrict__ X,
                                   const double* __restrict__ faceX, const double* __restrict__ shift,
                                   const double* __restrict__ xc, const double* __restrict__ frame,
                                   const double* __restrict__ Lc, PlaneWave pw, const double* __restrict__ rule, int nq,
                                   double* __restrict__ sigtr) {
    int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= n_face) return;
    const RefTables& rt = *rtp;
    const int NP = rt.Nphi;
    constexpr int NV = DIM + 1;
    constexpr int NS = DIM == 2 ? 3 : 6;
    double acc[NS][kMaxNP];
    for (int c2 = 0; c2 < NS; ++c2)
        for (int m = 0; m < NP; ++m) acc[c2][m] = 0;
    for (int side = 0; side < 2; ++side) {
        const int e = side == 0 ? fl[f] : fr[f];
        if (e < 0) continue;
        double V[NV][DIM], off[DIM];
        for (int a = 0; a < DIM; ++a) {
            off[a] = side == 0 ? 0.0 : shift[f * DIM + a];
            double b = 0;
            for (int k = 0; k < NV; ++k) b += X[((int64_t)e * NV + k) * DIM + a];
            V[DIM][a] = b / NV;
            for (int q = 0; q < DIM; ++q) V[q][a] = faceX[(f * DIM + q) * DIM + a] - off[a];
        }
        double E[DIM][DIM];
        for (int q = 0; q < DIM; ++q)
            for (int a = 0; a < DIM; ++a) E[q][a] = V[q + 1][a] - V[0][a];
        double det = DIM == 2 ? E[0][0] * E[1][1] - E[0][1] * E[1][0]
                              : E[0][0] * (E[1][1] * E[2][2] - E[1][2] * E[2][1]) - E[0][1] * (E[1][0] * E[2][2] - E[1][2] * E[2][0]) +
                                    E[0][2] * (E[1][0] * E[2][1] - E[1][1] * E[2][0]);
        det = fabs(det);
        for (int q = 0; q < nq; ++q) {
            const double* rp = rule + q * (DIM + 1);
            double x[DIM], y[DIM];
            for (int a = 0; a < DIM; ++a) {
                x[a] = V[0][a];
                for (int r = 0; r < DIM; ++r) x[a] += rp[r] * E[r][a];
            }
            for (int r = 0; r < DIM; ++r) {   // principal-axis coordinates of R_j (the internal dual basis)
                double t = 0.0;
                for (int a = 0; a < DIM; ++a) t += frame[(f * DIM + r) * DIM + a] * (x[a] + off[a] - xc[f * DIM + a]);
                y[r] = t;
            }
            double ps[kMaxNP];
            eval_monomials<DIM>(rt, y, ps, nullptr);
            double v[3], s[3][3];
            pw_eval<DIM>(pw, x, v, s);
            const double w = rp[DIM] * det;
            for (int c2 = 0; c2 < NS; ++c2) {
                int a, b;
                sym_ab<DIM>(c2, a, b);
                for (int m = 0; m < NP; ++m) acc[c2][m] += w * ps[m] * s[a][b];
            }
        }
    }
    // orthonormal coordinates: sigma~ = L^T M^{-1} rhs = L^{-1} rhs (forward substitution)
    const double* Lf = Lc + f * NP * NP;
    for (int c2 = 0; c2 < NS; ++c2)
        for (int m = 0; m < NP; ++m) {
            double s = acc[c2][m];
            for (int q = 0; q < m; ++q) s -= Lf[m * NP + q] * sigtr[(f * NS + c2) * NP + q];
            sigtr[(f * NS + c2) * NP + m] = s / Lf[m * NP + m];
        }
}

cudaError_t launch_project_plane_wave(stdg_ctx* c, int shot, int kind, const double* n, const double* pol, double amp,
                                      double t, const double* d_rule, int nq) {
    PlaneWave pw{};
    const int d = c->dim;
    double nn = 0;
    for (int a = 0; a < d; ++a) nn += n[a] * n[a];
    nn = std::sqrt(nn);
    double nh[3] = {0, 0, 0}, e[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) { nh[a] = n[a] / nn; pw.k[a] = 2 * M_PI * n[a]; }
    const double l0 = c->lam_e[0], m0 = c->mu_e[0], r0 = c->rho_e[0];
    double cw;
    if (kind == 0) {
        cw = std::sqrt((l0 + 2 * m0) / r0);
        for (int a = 0; a < d; ++a) {
            pw.rv[a] = -cw * nh[a];
            for (int b = 0; b < d; ++b) pw.rs[a][b] = (a == b ? l0 : 0.0) + 2 * m0 * nh[a] * nh[b];
        }
    } else {
        cw = std::sqrt(m0 / r0);
        if (pol) { for (int a = 0; a < d; ++a) e[a] = pol[a]; }
        else { e[0] = -nh[1]; e[1] = nh[0]; }
        double ne = 0;
        for (int a = 0; a < d; ++a) ne += e[a] * e[a];
        ne = std::sqrt(ne);
        for (int a = 0; a < d; ++a) e[a] /= ne;
        for (int a = 0; a < d; ++a) {
            pw.rv[a] = -cw * e[a];
            for (int b = 0; b < d; ++b) pw.rs[a][b] = m0 * (nh[a] * e[b] + e[a] * nh[b]);
        }
    }
    pw.omega = cw * 2 * M_PI * nn;
    pw.amp = amp;
    pw.t = t;
    double* vtr = c->d_vtr + shot * c->ntr;
    double* sig = c->d_sigtr + shot * c->nsig;
    const unsigned ge = (unsigned)((c->n_elem + 127) / 128), gf = (unsigned)((c->n_face + 127) / 128);
    if (d == 2) {
        project_vel_kernel<2><<<ge, 128, 0, c->stream>>>(c->n_elem, c->d_rt, c->d_X, c->d_detJ, pw, d_rule, nq, vtr); note_launch(c);
        project_sig_kernel<2><<<gf, 128, 0, c->stream>>>(c->n_face, c->d_rt, c->d_face_l, c->d_face_r, c->d_X, c->d_faceX,
                                                         c->d_shift, c->d_xc, c->d_frame, c->d_L, pw, d_rule, nq, sig); note_launch(c);
    } else {
        project_vel_kernel<3><<<ge, 128, 0, c->stream>>>(c->n_elem, c->d_rt, c->d_X, c->d_detJ, pw, d_rule, nq, vtr); note_launch(c);
        project_sig_kernel<3><<<gf, 128, 0, c->stream>>>(c->n_face, c->d_rt, c->d_face_l, c->d_face_r, c->d_X, c->d_faceX,
                                                         c->d_shift, c->d_xc, c->d_frame, c->d_L, pw, d_rule, nq, sig); note_launch(c);
    }
    return cudaGetLastError();
}

}  // namespace stdg
