// Block-Jacobi preconditioner "Pre1" (Appendix A, Eq. pre1): the exact inverse of each
// element's diagonal block of the velocity system.
//
// The diagonal block has Kronecker form (space (x) time):
//   A_ii = M_i (x) T + c dt^2 K_i (x) S,   M_i = rho_i |J_i| (I_d (x) M_ref),
//   K_i[(k,n),(k',n')] = sum_{j in S_i} sum_{l,l'} E_j[k,l,k',l'] (D~_{i,j}[l] D~_{i,j}[l']^T)[n,n'],
// (T, S time factors as in the operator; c = 1 or 1/4 for Crank-Nicolson).  With the
// generalised eigen-decomposition K_i V = M_i V Lambda, V^T M_i V = I:
//   A_ii^{-1} = (V (x) I) blockdiag_q (T + c dt^2 lambda_q S)^{-1} (V^T (x) I).
// V and Lambda do not depend on dt; only the small N_gamma x N_gamma blocks do.  The
// symmetric eigenproblem R^{-1} K R^{-T} / (rho|J|) = Q Lambda Q^T (M_ref = R R^T) is
// solved per element by a cyclic two-sided Jacobi method with round-robin pair ordering
// (all pairs of a round rotate concurrently), in FP64.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "stdg_internal.h"
#include "tma.h"

namespace stdg {

constexpr int kPreThreads = 128;
constexpr int kMaxN = 3 * kMaxNP;   // d * N_phi <= 60

// smem: C (n x n, stride n+1), Q (n x n, stride n+1), D~ one side (d*NP*NP), pairs, angles
__global__ void __launch_bounds__(kPreThreads) pre1_setup_kernel(
    int64_t n_elem, int dim, const RefTables* __restrict__ rtp, const int32_t* __restrict__ elem_face,
    const int32_t* __restrict__ face_l, const double* __restrict__ D, const double* __restrict__ lamf,
    const double* __restrict__ muf, const double* __restrict__ rhoJ, const double* __restrict__ Rinv,
    double* __restrict__ Vout, double* __restrict__ Lout, int* __restrict__ status) {
    extern __shared__ double sm[];
    const int NP = rtp->Nphi;
    const int n = dim * NP;
    const int ld = n + 1;
    double* C = sm;                       // n * ld
    double* Q = C + n * ld;               // n * ld
    double* Ds = Q + n * ld;              // dim * NP * NP
    double* Ri = Ds + dim * NP * NP;      // NP * NP
    double* cs = Ri + NP * NP;            // n/2 + 1
    double* sn = cs + kMaxN / 2 + 1;
    int* top = reinterpret_cast<int*>(sn + kMaxN / 2 + 1);   // round-robin tables
    int* bot = top + kMaxN / 2 + 1;
    __shared__ double s_off, s_diag;
    const int tid = threadIdx.x;
    for (int t = tid; t < NP * NP; t += blockDim.x) Ri[t] = Rinv[t];
    for (int64_t e = blockIdx.x; e < n_elem; e += gridDim.x) {
        // ---- K_i
        for (int t = tid; t < n * ld; t += blockDim.x) C[t] = 0.0;
        __syncthreads();
        for (int f = 0; f <= dim; ++f) {
            const int j = elem_face[e * (dim + 1) + f];
            const int side = face_l[j] == (int)e ? 0 : 1;
            const double* Dg = D + ((int64_t)j * 2 + side) * dim * NP * NP;
            for (int t = tid; t < dim * NP * NP; t += blockDim.x) Ds[t] = Dg[t];
            const double lam = lamf[j], mu = muf[j];
            __syncthreads();
            for (int ent = tid; ent < n * n; ent += blockDim.x) {
                const int r = ent / n, c = ent % n;
                const int k = r / NP, nn = r % NP, k2 = c / NP, n2 = c % NP;
                // P[l][l'][n][n'] = sum_m D~[l][n][m] D~[l'][n'][m]
                auto P = [&](int l, int l2) {
                    const double* a = Ds + (l * NP + nn) * NP;
                    const double* b = Ds + (l2 * NP + n2) * NP;
                    double s = 0;
                    for (int m = 0; m < NP; ++m) s += a[m] * b[m];
                    return s;
                };
                double v = lam * P(k, k2) + mu * P(k2, k);
                if (k == k2)
                    for (int l = 0; l < dim; ++l) v += mu * P(l, l);
                C[r * ld + c] += v;
            }
            __syncthreads();
        }
        // ---- C <- R^{-1} K R^{-T} / (rho |J|), using Q as scratch
        const double inv = 1.0 / rhoJ[e];
        for (int ent = tid; ent < n * n; ent += blockDim.x) {
            const int r = ent / n, c = ent % n;
            const int k2 = c / NP, n2 = c % NP;
            double s = 0;
            for (int q = 0; q <= n2; ++q) s += C[r * ld + k2 * NP + q] * Ri[n2 * NP + q];
            Q[r * ld + c] = s;
        }
        __syncthreads();
        for (int ent = tid; ent < n * n; ent += blockDim.x) {
            const int r = ent / n, c = ent % n;
            const int k = r / NP, nn = r % NP;
            double s = 0;
            for (int q = 0; q <= nn; ++q) s += Ri[nn * NP + q] * Q[(k * NP + q) * ld + c];
            C[r * ld + c] = s * inv;
        }
        __syncthreads();
        // symmetrise and set Q = I
        for (int ent = tid; ent < n * n; ent += blockDim.x) {
            const int r = ent / n, c = ent % n;
            if (r < c) {
                const double a = 0.5 * (C[r * ld + c] + C[c * ld + r]);
                C[r * ld + c] = a;
                C[c * ld + r] = a;
            }
            Q[r * ld + c] = r == c ? 1.0 : 0.0;
        }
        // ---- cyclic Jacobi, round-robin ordering on an even number of slots
        const int m2 = (n + 1) / 2;          // pairs per round (a dummy slot when n is odd)
        const int slots = 2 * m2;
        if (tid < m2) { top[tid] = 2 * tid; bot[tid] = 2 * tid + 1; }
        __syncthreads();
        int sweep = 0;
        for (; sweep < 30; ++sweep) {
            if (tid == 0) { s_off = 0.0; s_diag = 0.0; }
            __syncthreads();
            double off = 0, dg = 0;
            for (int ent = tid; ent < n * n; ent += blockDim.x) {
                const int r = ent / n, c = ent % n;
                const double a = C[r * ld + c];
                if (r == c) dg += a * a; else off += a * a;
            }
            atomicAdd(&s_off, off);
            atomicAdd(&s_diag, dg);
            __syncthreads();
            if (s_off <= 1e-30 * s_diag || s_diag == 0.0) break;
            for (int round = 0; round < slots - 1; ++round) {
                // rotation angles for the pairs of this step of the pair schedule
                if (tid < m2) {
                    int p = top[tid], q = bot[tid];
                    if (p > q) { int t = p; p = q; q = t; }
                    double c = 1.0, s = 0.0;
                    if (q < n) {
                        const double apq = C[p * ld + q];
                        if (apq != 0.0) {
                            const double app = C[p * ld + p], aqq = C[q * ld + q];
                            const double theta = (aqq - app) / (2.0 * apq);
                            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                            c = 1.0 / sqrt(t * t + 1.0);
                            s = t * c;
                        }
                    }
                    cs[tid] = c;
                    sn[tid] = s;
                }
                __syncthreads();
                // columns: C <- C J, Q <- Q J
                for (int ent = tid; ent < n * m2; ent += blockDim.x) {
                    const int r = ent / m2, k = ent % m2;
                    int p = top[k], q = bot[k];
                    if (p > q) { int t = p; p = q; q = t; }
                    if (q >= n) continue;
                    const double c = cs[k], s = sn[k];
                    const double a = C[r * ld + p], b = C[r * ld + q];
                    C[r * ld + p] = c * a - s * b;
                    C[r * ld + q] = s * a + c * b;
                    const double qa = Q[r * ld + p], qb = Q[r * ld + q];
                    Q[r * ld + p] = c * qa - s * qb;
                    Q[r * ld + q] = s * qa + c * qb;
                }
                __syncthreads();
                // rows: C <- J^T C
                for (int ent = tid; ent < n * m2; ent += blockDim.x) {
                    const int col = ent / m2, k = ent % m2;
                    int p = top[k], q = bot[k];
                    if (p > q) { int t = p; p = q; q = t; }
                    if (q >= n) continue;
                    const double c = cs[k], s = sn[k];
                    const double a = C[p * ld + col], b = C[q * ld + col];
                    C[p * ld + col] = c * a - s * b;
                    C[q * ld + col] = s * a + c * b;
                }
                __syncthreads();
                // next round-robin arrangement (slot top[0] stays fixed)
                if (tid == 0) {
                    const int t_last = top[m2 - 1];
                    const int b0 = bot[0];
                    for (int k = m2 - 1; k > 1; --k) top[k] = top[k - 1];
                    if (m2 > 1) top[1] = b0;
                    for (int k = 0; k < m2 - 1; ++k) bot[k] = bot[k + 1];
                    bot[m2 - 1] = t_last;
                }
                __syncthreads();
            }
        }
        if (tid == 0 && sweep >= 30) atomicExch(status, 1);
        // ---- V = (I (x) R^{-T}) Q / sqrt(rho |J|), eigenvalues
        const double sc = sqrt(inv);
        double* Vg = Vout + e * (int64_t)n * n;
        for (int ent = tid; ent < n * n; ent += blockDim.x) {
            const int r = ent / n, c = ent % n;
            const int k = r / NP, nn = r % NP;
            double s = 0;
            for (int q = nn; q < NP; ++q) s += Ri[q * NP + nn] * Q[(k * NP + q) * ld + c];
            Vg[ent] = s * sc;
        }
        for (int q = tid; q < n; q += blockDim.x) Lout[e * n + q] = C[q * ld + q];
        __syncthreads();
    }
}

// B[e][q] = (T + cdt2 lambda_q S)^{-1}  (N_gamma x N_gamma, Gauss-Jordan)
template <typename R>
__global__ void pre1_time_kernel(int64_t nq, int NG, const RefTables* __restrict__ rtp, const double* __restrict__ lam,
                                 double cdt2, R* __restrict__ B) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nq) return;
    double A[kMaxNG][2 * kMaxNG];
    const double l = lam[i];
    for (int a = 0; a < NG; ++a)
        for (int b = 0; b < NG; ++b) {
            A[a][b] = rtp->T[a * NG + b] + cdt2 * l * rtp->S[a * NG + b];
            A[a][NG + b] = a == b ? 1.0 : 0.0;
        }
    for (int c = 0; c < NG; ++c) {
        int piv = c;
        for (int r = c + 1; r < NG; ++r) if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c)
            for (int k = 0; k < 2 * NG; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
        const double d = 1.0 / A[c][c];
        for (int k = 0; k < 2 * NG; ++k) A[c][k] *= d;
        for (int r = 0; r < NG; ++r) {
            if (r == c) continue;
            const double f = A[r][c];
            for (int k = 0; k < 2 * NG; ++k) A[r][k] -= f * A[c][k];
        }
    }
    for (int a = 0; a < NG; ++a)
        for (int b = 0; b < NG; ++b) B[i * NG * NG + a * NG + b] = (R)A[a][NG + b];
}

// z_e = V (blockdiag B) V^T r_e for every element; r, z layout [e][k][a][n].  One warp per
// element; V staged in shared memory with a padded row stride.
template <typename R>
__global__ void __launch_bounds__(128) pre1_apply_kernel(int64_t n_elem, int dim, int NP, int NG, const R* __restrict__ V,
                                                         const R* __restrict__ B, const R* __restrict__ r0,
                                                         const int* __restrict__ ridx, int64_t ld_vec, R* __restrict__ z0,
                                                         int nshots, int64_t nvec) {
    const R* r = r0;
    extern __shared__ unsigned char smraw[];
    R* sm = reinterpret_cast<R*>(smraw);
    if (ridx) r += (int64_t)(*ridx) * ld_vec;
    const int n = dim * NP;
    const int ldv = n + 1;
    const int per = n * ldv + 2 * n * NG;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    R* sV = sm + warp * per;
    R* sr = sV + n * ldv;        // [(k,n)][a]
    R* sw = sr + n * NG;         // [q][a]
    for (int64_t e = blockIdx.x * (int64_t)wpb + warp; e < n_elem; e += (int64_t)gridDim.x * wpb) {
        const R* Vg = V + e * (int64_t)n * n;
        for (int t = lane; t < n * n; t += 32) sV[(t / n) * ldv + t % n] = Vg[t];
        for (int shot = 0; shot < nshots; ++shot) {
        const R* re = r + (int64_t)shot * nvec + e * (int64_t)n * NG;
        R* z = z0 + (int64_t)shot * nvec;
        for (int t = lane; t < n * NG; t += 32) {
            const int k = t / (NG * NP), a = (t / NP) % NG, nn = t % NP;
            sr[(k * NP + nn) * NG + a] = re[t];
        }
        __syncwarp();
        for (int q = lane; q < n; q += 32) {
            R u[kMaxNG];
            for (int a = 0; a < NG; ++a) u[a] = 0;
            for (int row = 0; row < n; ++row) {
                const R v = sV[row * ldv + q];
                for (int a = 0; a < NG; ++a) u[a] += v * sr[row * NG + a];
            }
            const R* Bq = B + (e * n + q) * NG * NG;
            for (int a = 0; a < NG; ++a) {
                R s = 0;
                for (int b = 0; b < NG; ++b) s += Bq[a * NG + b] * u[b];
                sw[q * NG + a] = s;
            }
        }
        __syncwarp();
        R* ze = z + e * (int64_t)n * NG;
        for (int row = lane; row < n; row += 32) {
            R acc[kMaxNG];
            for (int a = 0; a < NG; ++a) acc[a] = 0;
            for (int q = 0; q < n; ++q) {
                const R v = sV[row * ldv + q];
                for (int a = 0; a < NG; ++a) acc[a] += v * sw[q * NG + a];
            }
            const int k = row / NP, nn = row % NP;
            for (int a = 0; a < NG; ++a) ze[(k * NG + a) * NP + nn] = acc[a];
        }
        __syncwarp();
        }   // shots
    }
}

// Register-blocked variant for d*N_phi <= 32: lane q holds column q of V (for u = V^T r),
// lane `row` holds row `row` of V (for z = V w); the rows of r and w are read from shared
// memory by all lanes at once (broadcast), so the inner loops are FMAs.
template <int DIM, int NP, int NG, typename R>
__global__ void __launch_bounds__(128) pre1_apply_reg_kernel(int64_t n_elem, const R* __restrict__ V, const R* __restrict__ B,
                                                             const R* __restrict__ r0, const int* __restrict__ ridx,
                                                             int64_t ld_vec, R* __restrict__ z0, int nshots, int64_t nvec) {
    const R* r = r0;
    constexpr int N = DIM * NP;
    static_assert(N <= 32, "register-blocked block-Jacobi apply needs d*N_phi <= 32");
    __shared__ __align__(16) R s_r[4][N * NG];
    __shared__ __align__(16) R s_w[4][N * NG];
    if (ridx) r += (int64_t)(*ridx) * ld_vec;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    R* sr = s_r[warp];
    R* sw = s_w[warp];
    const bool act = lane < N;
    const int q = act ? lane : 0;
    for (int64_t e = blockIdx.x * (int64_t)wpb + warp; e < n_elem; e += (int64_t)gridDim.x * wpb) {
        const R* Ve = V + e * (int64_t)(N * N);
        R Vc[N], Vr[N], Bq[NG * NG];
#pragma unroll
        for (int row = 0; row < N; ++row) Vc[row] = act ? Ve[row * N + q] : (R)0;
#pragma unroll
        for (int qq = 0; qq < N; ++qq) Vr[qq] = act ? Ve[q * N + qq] : (R)0;
#pragma unroll
        for (int t = 0; t < NG * NG; ++t) Bq[t] = act ? B[(e * N + q) * (int64_t)(NG * NG) + t] : (R)0;
        for (int shot = 0; shot < nshots; ++shot) {   // V and B stay in registers for every shot
        const R* re = r + (int64_t)shot * nvec + e * (int64_t)(N * NG);
        R* z = z0 + (int64_t)shot * nvec;
        // r rows (k,n) with the NG time values contiguous
#pragma unroll
        for (int t0 = 0; t0 < N * NG; t0 += 32) {
            const int t = t0 + lane;
            if (t < N * NG) {
                const int k = t / (NG * NP), a = (t / NP) % NG, n = t % NP;
                sr[(k * NP + n) * NG + a] = re[t];
            }
        }
        __syncwarp();
        // u[q][a] = sum_row V[row][q] r[row][a];  w[q] = B_q u[q]
        R u[NG];
#pragma unroll
        for (int a = 0; a < NG; ++a) u[a] = 0;
#pragma unroll
        for (int row = 0; row < N; ++row)
            if constexpr (std::is_same<R, float>::value && NG % 2 == 0) {   // time-node pairs, packed FMA
                const float2* s2 = reinterpret_cast<const float2*>(sr + row * NG);
#pragma unroll
                for (int a = 0; a < NG; a += 2) {
                    const float2 p = ffma2(make_float2(Vc[row], Vc[row]), s2[a / 2], make_float2(u[a], u[a + 1]));
                    u[a] = p.x;
                    u[a + 1] = p.y;
                }
            } else {
#pragma unroll
                for (int a = 0; a < NG; ++a) u[a] = fma(Vc[row], sr[row * NG + a], u[a]);
            }
        if (act) {
#pragma unroll
            for (int a = 0; a < NG; ++a) {
                R s = 0;
#pragma unroll
                for (int b = 0; b < NG; ++b) s = fma(Bq[a * NG + b], u[b], s);
                sw[q * NG + a] = s;
            }
        }
        __syncwarp();
        // z[row][a] = sum_q V[row][q] w[q][a], row = lane
        R acc[NG];
#pragma unroll
        for (int a = 0; a < NG; ++a) acc[a] = 0;
#pragma unroll
        for (int qq = 0; qq < N; ++qq)
            if constexpr (std::is_same<R, float>::value && NG % 2 == 0) {
                const float2* w2 = reinterpret_cast<const float2*>(sw + qq * NG);
#pragma unroll
                for (int a = 0; a < NG; a += 2) {
                    const float2 p = ffma2(make_float2(Vr[qq], Vr[qq]), w2[a / 2], make_float2(acc[a], acc[a + 1]));
                    acc[a] = p.x;
                    acc[a + 1] = p.y;
                }
            } else {
#pragma unroll
                for (int a = 0; a < NG; ++a) acc[a] = fma(Vr[qq], sw[qq * NG + a], acc[a]);
            }
        if (act) {
            const int k = q / NP, n = q % NP;
            R* ze = z + e * (int64_t)(N * NG);
#pragma unroll
            for (int a = 0; a < NG; ++a) ze[(k * NG + a) * NP + n] = acc[a];
        }
        __syncwarp();
        }   // shots
    }
}

// Multi-shot FP32 variant for 2D, p = 2 (d N_phi = 12, N_gamma = 3), batches of 16 shots or
// more: one lane per shot.  A warp takes an element and 32 shots at a time; the element's V
// (12 x 12) and B (12 blocks of 3 x 3) are copied to shared memory once and read by all lanes
// at once, and each lane computes u = V^T r, w = B u, z = V w for its shot in registers.  The
// rows of r of the next (element, 32 shots) item are copied by the warp in order (cp.async)
// while the current one is computed, and z goes back through the same shared rows to
// 16-byte stores along each shot's element row.
struct Pre1Shots {
    static constexpr int NP = 6, NG = 3, N = 2 * NP, NV = N * NG;   // 36 values per element
    static constexpr int ROW = 44;                                  // 11 x 16 bytes (odd)
    static constexpr int RBUF = 32 * ROW;
    static constexpr int VB = N * N + N * NG * NG;                  // V then B: 144 + 108
    static constexpr int PER_WARP = 2 * RBUF + 2 * VB;
    static_assert(NV <= ROW && (ROW / 4) % 2 == 1 && (VB * 4) % 16 == 0 && (N * N * 4) % 16 == 0, "layout");
};

__device__ __forceinline__ void pre_cp16(float* dst, const float* src, bool on) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(on ? 16u : 0u)
                 : "memory");
}

__global__ void __launch_bounds__(128) pre1_apply_shots_kernel(int64_t n_elem, const float* __restrict__ V,
                                                               const float* __restrict__ B, const float* __restrict__ r,
                                                               const int* __restrict__ ridx, int64_t ld_vec,
                                                               float* __restrict__ z0, int nshots, int64_t nvec) {
    using P = Pre1Shots;
    constexpr int NP = P::NP, NG = P::NG, N = P::N, NV = P::NV;
    extern __shared__ __align__(16) unsigned char smraw[];
    if (ridx) r += (int64_t)(*ridx) * ld_vec;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    float* rbuf = reinterpret_cast<float*>(smraw) + warp * P::PER_WARP;
    float* vbb = rbuf + 2 * P::RBUF;
    const int nc = (nshots + 31) >> 5;
    const int64_t gw = blockIdx.x * (int64_t)wpb + warp, W = (int64_t)gridDim.x * wpb;
    const int64_t n_mine = gw < n_elem ? (n_elem - 1 - gw) / W + 1 : 0;
    const int64_t n_items = n_mine * nc;
    constexpr int CPR = NV / 4;   // 16-byte chunks per shot row
    auto issue = [&](int64_t t) {
        if (t < n_items) {
            const int64_t e = gw + (t / nc) * W;
            const int c0 = (int)(t % nc) * 32;
            float* buf = rbuf + (t & 1) * P::RBUF;
#pragma unroll
            for (int u = 0; u < CPR; ++u) {
                const int ci = lane + 32 * u, sl = ci / CPR, j = ci % CPR;
                const bool ok = c0 + sl < nshots;
                pre_cp16(buf + sl * P::ROW + 4 * j, r + (ok ? (int64_t)(c0 + sl) * nvec + e * NV + 4 * j : 0), ok);
            }
            float* vb = vbb + (t & 1) * P::VB;
            for (int j = lane; j < N * N / 4; j += 32) pre_cp16(vb + 4 * j, V + e * (N * N) + 4 * j, true);
            for (int j = lane; j < N * NG * NG / 4; j += 32)
                pre_cp16(vb + N * N + 4 * j, B + e * (N * NG * NG) + 4 * j, true);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    issue(0);
    for (int64_t t = 0; t < n_items; ++t) {
        issue(t + 1);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncwarp();
        float* row = rbuf + (t & 1) * P::RBUF + lane * P::ROW;
        const float* sV = vbb + (t & 1) * P::VB;
        const float* sB = sV + N * N;
        // r[row][a], row = (k, n), from the element layout [k][a][n]
        float rv[N][NG];
#pragma unroll
        for (int j = 0; j < CPR; ++j) {
            const float4 q = reinterpret_cast<const float4*>(row)[j];
            const float e4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = 4 * j + u, k = i / (NG * NP), a = (i / NP) % NG, n = i % NP;
                rv[k * NP + n][a] = e4[u];
            }
        }
        // w[q] = B_q (V^T r)[q]
        float w[N][NG];
#pragma unroll
        for (int q = 0; q < N; ++q) {
            float u[NG];
#pragma unroll
            for (int a = 0; a < NG; ++a) u[a] = 0.f;
#pragma unroll
            for (int rr = 0; rr < N; ++rr) {
                const float vq = sV[rr * N + q];
#pragma unroll
                for (int a = 0; a < NG; ++a) u[a] = fmaf(vq, rv[rr][a], u[a]);
            }
#pragma unroll
            for (int a = 0; a < NG; ++a) {
                float s = 0.f;
#pragma unroll
                for (int b = 0; b < NG; ++b) s = fmaf(sB[(q * NG + a) * NG + b], u[b], s);
                w[q][a] = s;
            }
        }
        // z = V w, written back to the lane's row in the element layout
#pragma unroll
        for (int rr = 0; rr < N; ++rr) {
            float acc[NG];
#pragma unroll
            for (int a = 0; a < NG; ++a) acc[a] = 0.f;
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const float v = sV[rr * N + q];
#pragma unroll
                for (int a = 0; a < NG; ++a) acc[a] = fmaf(v, w[q][a], acc[a]);
            }
            const int k = rr / NP, n = rr % NP;
#pragma unroll
            for (int a = 0; a < NG; ++a) rv[rr][a] = acc[a];
            (void)k; (void)n;
        }
#pragma unroll
        for (int j = 0; j < CPR; ++j) {
            float e4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int i = 4 * j + u, k = i / (NG * NP), a = (i / NP) % NG, n = i % NP;
                e4[u] = rv[k * NP + n][a];
            }
            reinterpret_cast<float4*>(row)[j] = make_float4(e4[0], e4[1], e4[2], e4[3]);
        }
        __syncwarp();
        const int64_t e = gw + (t / nc) * W;
        const int c0 = (int)(t % nc) * 32;
        const float* rows = rbuf + (t & 1) * P::RBUF;
#pragma unroll
        for (int u = 0; u < CPR; ++u) {
            const int ci = lane + 32 * u, sl = ci / CPR, j = ci % CPR;
            if (c0 + sl < nshots)
                *reinterpret_cast<float4*>(z0 + (int64_t)(c0 + sl) * nvec + e * NV + 4 * j) =
                    reinterpret_cast<const float4*>(rows + sl * P::ROW)[j];
        }
        __syncwarp();   // the rows and the V, B blocks are free for the item after next
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Single-shot FP32 block-Jacobi apply for 2D, p = 3 (N = d N_phi = 20, N_gamma = 4).  Per
// element u = V^T r, w_q = B_q u_q, z = V w are 20 x 20 x 4 products.  Six consecutive
// elements per warp, five lanes each: lane g holds columns 4g..4g+3 for u and w (16
// accumulators: every V value read feeds four products, every r value four; B comes in the
// lane order [qi][a][g][b]) and rows g, g+5, g+10, g+15 for z (their V rows are 20 floats
// apart across lanes: distinct banks).  The six elements' V, B and r are three contiguous ranges, copied by
// cp.async.bulk one group ahead (per-warp double buffer, bounded mbarrier waits); w goes to
// the element's r slot, z to its B slot, and z leaves with consecutive 16-byte stores.
struct Pre1Tile {
    static constexpr int NP = 10, NG = 4, N = 20, NV = N * NG;     // 80 values per element
    static constexpr int EPW = 6;                                  // elements per warp and group
    static constexpr int VE = N * N, BE = N * NG * NG;             // 400, 320 floats
    static constexpr int SB = EPW * VE, SR = SB + EPW * BE;        // stage: V | B | r
    static constexpr int STAGE = SR + EPW * NV;                    // 4,800 floats
    static constexpr int PER_WARP = 2 * STAGE;
    static_assert((VE * 4) % 16 == 0 && (BE * 4) % 16 == 0 && (NV * 4) % 16 == 0, "bulk copies need 16-byte sizes");
};

// B of every element from [q][a][b] to the lane order of the apply below, [qi][a][g][b] with
// q = 4g + qi: the five lanes of an element then read consecutive 16-byte pieces
__global__ void pre1_b_lane_order_kernel(int64_t n_elem, const float* __restrict__ B, float* __restrict__ Bt) {
    using P = Pre1Tile;
    const int64_t n = n_elem * P::BE;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / P::BE;
        const int t = (int)(i % P::BE);                   // destination index in [qi][a][g][b]
        const int b = t % P::NG, g = (t / P::NG) % 5, a = (t / (5 * P::NG)) % P::NG, qi = t / (5 * P::NG * P::NG);
        Bt[i] = B[e * P::BE + ((4 * g + qi) * P::NG + a) * P::NG + b];
    }
}

__global__ void __launch_bounds__(64) pre1_apply_tile_kernel(int64_t n_elem, const float* __restrict__ V,
                                                             const float* __restrict__ B, const float* __restrict__ r,
                                                             const int* __restrict__ ridx, int64_t ld,
                                                             float* __restrict__ z, int* __restrict__ err) {
    using P = Pre1Tile;
    constexpr int N = P::N, NG = P::NG, NP = P::NP, NV = P::NV, EPW = P::EPW, VE = P::VE, BE = P::BE;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[2][2];
    if (ridx) r += (int64_t)(*ridx) * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    float* base = reinterpret_cast<float*>(smraw) + warp * P::PER_WARP;
    const uint32_t bar0 = smem_u32(&bars[warp][0]), bar1 = smem_u32(&bars[warp][1]);
    if (lane == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int el = lane / 5, g = lane % 5;    // lanes 30, 31: el = 6, idle
    const int64_t n_grp = (n_elem + EPW - 1) / EPW;
    const int64_t stride = (int64_t)gridDim.x * wpb;
    constexpr long kPollLimit = 1L << 24;
    auto issue = [&](int64_t p, int st) {   // lane 0 only
        const int64_t e0 = p * EPW;
        const int ne = (int)min((int64_t)EPW, n_elem - e0);
        float* sg = base + st * P::STAGE;
        const uint32_t bar = st ? bar1 : bar0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, (uint32_t)(ne * (VE + BE + NV) * sizeof(float)));
        bulk_g2s(smem_u32(sg), V + e0 * VE, ne * VE * sizeof(float), bar);
        bulk_g2s(smem_u32(sg + P::SB), B + e0 * BE, ne * BE * sizeof(float), bar);
        bulk_g2s(smem_u32(sg + P::SR), r + e0 * NV, ne * NV * sizeof(float), bar);
    };
    int64_t p = blockIdx.x * (int64_t)wpb + warp;
    if (p < n_grp && lane == 0) issue(p, 0);
    uint32_t ph0 = 0, ph1 = 0;
    int st = 0;
    for (; p < n_grp; p += stride) {
        const int64_t pn = p + stride;
        if (pn < n_grp && lane == 0) issue(pn, st ^ 1);
        if (!__all_sync(0xffffffffu, mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0, kPollLimit))) {
            if (lane == 0) atomicExch(err, 1);
            bool drained = mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0, kPollLimit);
            if (pn < n_grp) drained = mbar_wait(st ? bar0 : bar1, st ? ph0 : ph1, kPollLimit) && drained;
            if (!drained && lane == 0) atomicExch(err, 2);
            break;
        }
        if (st) ph1 ^= 1u; else ph0 ^= 1u;
        float* sg = base + st * P::STAGE;
        const int64_t e0 = p * EPW;
        const int ne = (int)min((int64_t)EPW, n_elem - e0);
        const bool act = el < ne;
        const float* sV = sg + (act ? el : 0) * VE;
        float* sB = sg + P::SB + (act ? el : 0) * BE;
        float* sR = sg + P::SR + (act ? el : 0) * NV;
        // ---- u = V^T r for columns 4g..4g+3, then w_q = B_q u_q
        float wq[4][NG];
        if (act) {
            float u[4][NG];
#pragma unroll
            for (int qi = 0; qi < 4; ++qi)
#pragma unroll
                for (int a = 0; a < NG; ++a) u[qi][a] = 0.f;
#pragma unroll
            for (int row = 0; row < N; ++row) {
                const float4 v4 = *reinterpret_cast<const float4*>(sV + row * N + 4 * g);
                const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
                const int k = row / NP, n = row % NP;
                float ra[NG];
#pragma unroll
                for (int a = 0; a < NG; ++a) ra[a] = sR[(k * NG + a) * NP + n];
#pragma unroll
                for (int qi = 0; qi < 4; ++qi)
#pragma unroll
                    for (int a = 0; a < NG; ++a) u[qi][a] = fmaf(vv[qi], ra[a], u[qi][a]);
            }
#pragma unroll
            for (int qi = 0; qi < 4; ++qi) {
#pragma unroll
                for (int a = 0; a < NG; ++a) {   // B in the lane order [qi][a][g][b]
                    const float4 b4 = *reinterpret_cast<const float4*>(sB + ((qi * NG + a) * 5 + g) * NG);
                    wq[qi][a] = fmaf(b4.x, u[qi][0], fmaf(b4.y, u[qi][1], fmaf(b4.z, u[qi][2], b4.w * u[qi][3])));
                }
            }
        }
        __syncwarp();   // the element's r and B have been read
        if (act) {
#pragma unroll
            for (int qi = 0; qi < 4; ++qi)
                *reinterpret_cast<float4*>(sR + (4 * g + qi) * NG) = make_float4(wq[qi][0], wq[qi][1], wq[qi][2], wq[qi][3]);
        }
        __syncwarp();
        // ---- z = V w for rows g + 5 ri, into the element's B slot in the element layout
        if (act) {
            float zz[4][NG];
#pragma unroll
            for (int ri = 0; ri < 4; ++ri)
#pragma unroll
                for (int a = 0; a < NG; ++a) zz[ri][a] = 0.f;
#pragma unroll
            for (int qc = 0; qc < N / 4; ++qc) {
                float4 wv[4];
#pragma unroll
                for (int qi = 0; qi < 4; ++qi) wv[qi] = *reinterpret_cast<const float4*>(sR + (4 * qc + qi) * NG);
#pragma unroll
                for (int ri = 0; ri < 4; ++ri) {   // rows g + 5 ri: 20 floats apart across lanes, no conflict
                    const float4 v4 = *reinterpret_cast<const float4*>(sV + (g + 5 * ri) * N + 4 * qc);
                    const float vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int qi = 0; qi < 4; ++qi) {
                        zz[ri][0] = fmaf(vv[qi], wv[qi].x, zz[ri][0]);
                        zz[ri][1] = fmaf(vv[qi], wv[qi].y, zz[ri][1]);
                        zz[ri][2] = fmaf(vv[qi], wv[qi].z, zz[ri][2]);
                        zz[ri][3] = fmaf(vv[qi], wv[qi].w, zz[ri][3]);
                    }
                }
            }
#pragma unroll
            for (int ri = 0; ri < 4; ++ri) {
                const int row = g + 5 * ri, k = row / NP, n = row % NP;
#pragma unroll
                for (int a = 0; a < NG; ++a) sB[(k * NG + a) * NP + n] = zz[ri][a];
            }
        }
        __syncwarp();
        for (int t = lane; t < ne * (NV / 4); t += 32) {
            const int e2 = t / (NV / 4), j = t % (NV / 4);
            *reinterpret_cast<float4*>(z + (e0 + e2) * NV + 4 * j) =
                *reinterpret_cast<const float4*>(sg + P::SB + e2 * BE + 4 * j);
        }
        __syncwarp();   // stage st is free for the next group
        st ^= 1;
    }
}

template <typename R>
static bool pre1_apply_fast(stdg_ctx* c, const R* V, const R* B, const R* r, R* z, const int* ridx, int64_t ld,
                            cudaError_t* err, int nshots) {
    const int64_t blocks = std::min<int64_t>((c->n_elem + 3) / 4, 1 << 30);
    const int d = c->dim, np = c->Nphi, ng = c->Ng;
    if constexpr (std::is_same<R, float>::value) {
        if (d == 2 && np == 10 && ng == 4 && nshots == 1 && c->d_err && c->d_preB32t && B == c->d_preB32 &&
            reinterpret_cast<uintptr_t>(r) % 16 == 0 &&
            reinterpret_cast<uintptr_t>(z) % 16 == 0 && reinterpret_cast<uintptr_t>(V) % 16 == 0 &&
            reinterpret_cast<uintptr_t>(B) % 16 == 0 && (ld * (int64_t)sizeof(R)) % 16 == 0) {
            constexpr int wpb = 1;   // 38.4 KB of stages per warp
            const size_t smem = sizeof(float) * wpb * Pre1Tile::PER_WARP;
            const int64_t n_grp = (c->n_elem + Pre1Tile::EPW - 1) / Pre1Tile::EPW;
            const int64_t nb = std::min<int64_t>((n_grp + wpb - 1) / wpb, (int64_t)c->n_sm * 16);
            cudaFuncSetAttribute(pre1_apply_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            pre1_apply_tile_kernel<<<(unsigned)nb, 32 * wpb, smem, c->stream>>>(c->n_elem, V, c->d_preB32t, r, ridx, ld, z,
                                                                              c->d_err);
            note_launch(c);
            *err = cudaGetLastError();
            return true;
        }
        if (d == 2 && np == 6 && ng == 3 && nshots >= 16 && reinterpret_cast<uintptr_t>(r) % 16 == 0 &&
            reinterpret_cast<uintptr_t>(z) % 16 == 0 && reinterpret_cast<uintptr_t>(V) % 16 == 0 &&
            reinterpret_cast<uintptr_t>(B) % 16 == 0 && (ld * (int64_t)sizeof(R)) % 16 == 0) {
            constexpr int wpb = 4;
            const size_t smem = sizeof(float) * wpb * Pre1Shots::PER_WARP;
            const int64_t nb = std::min<int64_t>((c->n_elem + wpb - 1) / wpb, (int64_t)c->n_sm * 16);
            cudaFuncSetAttribute(pre1_apply_shots_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            pre1_apply_shots_kernel<<<(unsigned)nb, 32 * wpb, smem, c->stream>>>(c->n_elem, V, B, r, ridx, ld, z, nshots,
                                                                                c->nvel);
            note_launch(c);
            *err = cudaGetLastError();
            return true;
        }
    }
#define STDG_PRE_FAST(D_, NP_, NG_)                                                                        \
    if (d == D_ && np == NP_ && ng == NG_) {                                                              \
        pre1_apply_reg_kernel<D_, NP_, NG_, R><<<(unsigned)blocks, 128, 0, c->stream>>>(c->n_elem, V, B, r, ridx, ld, z, nshots, c->nvel); \
        note_launch(c);                                                                                    \
        *err = cudaGetLastError();                                                                         \
        return true;                                                                                       \
    }
    STDG_PRE_FAST(2, 10, 4)
    STDG_PRE_FAST(2, 6, 3)
    STDG_PRE_FAST(3, 10, 3)
    STDG_PRE_FAST(2, 3, 1)
#undef STDG_PRE_FAST
    return false;
}

cudaError_t launch_pre1_setup(stdg_ctx* c, const double* d_Rinv, const int32_t* d_elem_face, int* d_status) {
    const int n = c->dim * c->Nphi;
    const size_t smem = sizeof(double) * ((size_t)2 * n * (n + 1) + (size_t)c->dim * c->Nphi * c->Nphi + c->Nphi * c->Nphi +
                                          2 * (kMaxN / 2 + 1)) +
                        sizeof(int) * 2 * (kMaxN / 2 + 1);
    cudaFuncSetAttribute(pre1_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = (int)std::min<int64_t>(c->n_elem, c->n_sm * 16);
    pre1_setup_kernel<<<grid, kPreThreads, smem, c->stream>>>(c->n_elem, c->dim, c->d_rt, d_elem_face, c->d_face_l, c->d_D,
                                                              c->d_lamf, c->d_muf, c->d_rhoJ, d_Rinv, c->d_preV, c->d_preLam,
                                                              d_status); note_launch(c);
    return cudaGetLastError();
}

cudaError_t launch_pre1_time(stdg_ctx* c, double dt) {
    const double cfac = c->opt.scheme == STDG_SCHEME_CN ? 0.25 : 1.0;
    const int64_t nq = c->n_elem * c->dim * c->Nphi;
    pre1_time_kernel<double><<<(unsigned)((nq + 127) / 128), 128, 0, c->stream>>>(nq, c->Ng, c->d_rt, c->d_preLam,
                                                                               cfac * dt * dt, c->d_preB); note_launch(c);
    if (c->d_preB32) {
        pre1_time_kernel<float><<<(unsigned)((nq + 127) / 128), 128, 0, c->stream>>>(nq, c->Ng, c->d_rt, c->d_preLam,
                                                                                  cfac * dt * dt, c->d_preB32); note_launch(c);
    }
    if (c->d_preB32t) {
        const int64_t nb = c->n_elem * Pre1Tile::BE;
        pre1_b_lane_order_kernel<<<(unsigned)std::min<int64_t>((nb + 255) / 256, (int64_t)c->n_sm * 32), 256, 0, c->stream>>>(
            c->n_elem, c->d_preB32, c->d_preB32t); note_launch(c);
    }
    return cudaGetLastError();
}

template <typename R>
static cudaError_t pre1_apply_t(stdg_ctx* c, const R* V, const R* B, const R* r, R* z, const int* ridx, int64_t ld,
                                int nshots) {
    cudaError_t fe;
    if (pre1_apply_fast<R>(c, V, B, r, z, ridx, ld, &fe, nshots)) return fe;
    const int n = c->dim * c->Nphi;
    const int wpb = 4;
    const size_t smem = sizeof(R) * (size_t)wpb * (n * (n + 1) + 2 * n * c->Ng);
    cudaFuncSetAttribute(pre1_apply_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t blocks = std::min<int64_t>((c->n_elem + wpb - 1) / wpb, 1 << 30);
    pre1_apply_kernel<R><<<(unsigned)blocks, 32 * wpb, smem, c->stream>>>(c->n_elem, c->dim, c->Nphi, c->Ng, V, B, r, ridx, ld, z,
                                                                          nshots, c->nvel); note_launch(c);
    return cudaGetLastError();
}

cudaError_t launch_pre1_apply(stdg_ctx* c, const double* r, double* z, const int* ridx, int64_t ld, int nshots) {
    return pre1_apply_t<double>(c, c->d_preV, c->d_preB, r, z, ridx, ld, nshots);
}

cudaError_t launch_pre1_apply32(stdg_ctx* c, const float* r, float* z, const int* ridx, int64_t ld, int nshots) {
    return pre1_apply_t<float>(c, c->d_preV32, c->d_preB32, r, z, ridx, ld, nshots);
}

}  // namespace stdg
