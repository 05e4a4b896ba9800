// Stencil preconditioner "Pre2" (Appendix A, Eqs. APPRE1 - APPRE2): for element i with
// face neighbours e, the first block row of the inverse of the local system A_i formed
// by i and its neighbours, applied to the stencil's values.
//
// In a simplex mesh no two face neighbours of an element share a face (that would need
// a closed fan of three elements around an interior vertex in 2D, or around an interior
// edge in 3D, which the meshes here do not contain), so A_i is an "arrow": D_i in the
// corner, the couplings N_{i,e} and N_{e,i} in its first block row and column, and the
// neighbours' own diagonal blocks D_e.  Block elimination of the neighbours gives the
// first block row of A_i^{-1} in closed form:
//   z_i = S_i^{-1} (r_i - sum_e N_{i,e} D_e^{-1} r_e),   S_i = D_i - sum_e N_{i,e} D_e^{-1} N_{e,i},
// so one application is: y = P_1 r (the block-Jacobi apply), t = r - N y = 2 r - A y (since
// D y = r), z = S^{-1} t (one dense block per element).
//
// Set-up, per slab size dt, FP64, one CTA per element.  Every block has the Kronecker
// form of the operator (space (x) time): D_i = M_i (x) T + c dt^2 K_ii (x) S and
// N_{i,e} = c dt^2 K_ie (x) S, with K_ie the spatial face coupling of elements i and e
// and K_ei = K_ie^T.  With D_e^{-1} = (V_e (x) I) blockdiag_q(B_{e,q}) (V_e^T (x) I) from
// the block-Jacobi set-up,
//   N_{i,e} D_e^{-1} N_{e,i} = (c dt^2)^2 sum_q (k_q k_q^T) (x) (S B_{e,q} S),  k_q = K_ie V_e[:, q],
// which assembles S_i without any n^3 product; S_i (order d N_phi N_gamma) is then
// inverted by Gauss-Jordan elimination with partial pivoting and stored column-major, in
// FP64 for the FP64 solver and in FP32 for the FP32 inner solver of the mixed path.  (BF16
// blocks halve the bytes, but on the heterogeneous 60,024-triangle inversion medium they
// made the inner GMRES stagnate after 16 slabs; FP32 blocks converge there.)
#include <algorithm>
#include <cmath>
#include <type_traits>

#include <cuda_fp16.h>


#include "stdg_internal.h"

namespace stdg {

constexpr int kP2Threads = 256;
constexpr int kP2MaxRows = 4;                 // rows per lane in the apply: N <= 128

// K^{(j)}[(k,n),(k',n')] += lam P(k,k') + mu P(k',k) + delta_kk' mu sum_l P(l,l),
// P(a,b)[n][n'] = sum_m Da[a][n][m] Db[b][n'][m]   (Da: row element's D~, Db: column element's)
__device__ void add_face_coupling(double* K, int n, int dim, int NP, const double* Da, const double* Db, double lam,
                                  double mu, double scale) {
    for (int ent = threadIdx.x; ent < n * n; ent += blockDim.x) {
        const int r = ent / n, c = ent % n;
        const int k = r / NP, nn = r % NP, k2 = c / NP, n2 = c % NP;
        auto P = [&](int a, int b) {
            const double* x = Da + (a * NP + nn) * NP;
            const double* y = Db + (b * NP + n2) * NP;
            double s = 0;
            for (int m = 0; m < NP; ++m) s += x[m] * y[m];
            return s;
        };
        double v = lam * P(k, k2) + mu * P(k2, k);
        if (k == k2)
            for (int l = 0; l < dim; ++l) v += mu * P(l, l);
        K[ent] += scale * v;
    }
}

// smem: A (N x 2N augmented), K (n x n), kv (n x n), W (n x NG x NG), Da, Db (dim NP NP each), f (N)
__global__ void __launch_bounds__(kP2Threads) pre2_setup_kernel(
    int64_t n_elem, int dim, const RefTables* __restrict__ rtp, const int32_t* __restrict__ elem_face,
    const int32_t* __restrict__ face_l, const int32_t* __restrict__ face_r, const double* __restrict__ D,
    const double* __restrict__ lamf, const double* __restrict__ muf, const double* __restrict__ rhoJ,
    const double* __restrict__ preV, const double* __restrict__ preB, double cdt2, double* __restrict__ out64,
    float* __restrict__ out32, int64_t stride32, int* __restrict__ status) {
    extern __shared__ double sm[];
    const int NP = rtp->Nphi, NG = rtp->Ng;
    const int n = dim * NP;
    const int N = n * NG;
    const int ldA = 2 * N;
    double* A = sm;                         // N x 2N
    double* K = A + (size_t)N * ldA;        // n x n
    double* kv = K + n * n;                 // n x n: kv[s][q] = (K_ie V_e)[s][q]
    double* W = kv + n * n;                 // n x NG x NG: S B_q S
    double* Da = W + n * NG * NG;
    double* Db = Da + dim * NP * NP;
    double* f = Db + dim * NP * NP;         // N
    __shared__ int s_piv;
    __shared__ int s_sing;
    const int tid = threadIdx.x;
    for (int64_t e = blockIdx.x; e < n_elem; e += gridDim.x) {
        // ---- D_i: rho|J| (I (x) M_ref) (x) T + c dt^2 K_ii (x) S, and [ . | I ]
        for (int t = tid; t < n * n; t += blockDim.x) K[t] = 0.0;
        __syncthreads();
        for (int fi = 0; fi <= dim; ++fi) {
            const int j = elem_face[e * (dim + 1) + fi];
            const int side = face_l[j] == (int)e ? 0 : 1;
            const double* Dg = D + ((int64_t)j * 2 + side) * dim * NP * NP;
            for (int t = tid; t < dim * NP * NP; t += blockDim.x) Da[t] = Dg[t];
            __syncthreads();
            add_face_coupling(K, n, dim, NP, Da, Da, lamf[j], muf[j], 1.0);
            __syncthreads();
        }
        const double rj = rhoJ[e];
        for (int ent = tid; ent < N * N; ent += blockDim.x) {
            const int R = ent / N, C = ent % N;
            const int k = R / (NG * NP), a = (R / NP) % NG, nn = R % NP;
            const int k2 = C / (NG * NP), a2 = (C / NP) % NG, n2 = C % NP;
            double v = cdt2 * K[(k * NP + nn) * n + k2 * NP + n2] * rtp->S[a * NG + a2];
            if (k == k2) v += rj * rtp->Mref[nn * NP + n2] * rtp->T[a * NG + a2];
            A[R * ldA + C] = v;
            A[R * ldA + N + C] = R == C ? 1.0 : 0.0;
        }
        __syncthreads();
        // ---- minus N_{i,e} D_e^{-1} N_{e,i} for every face neighbour e
        for (int fi = 0; fi <= dim; ++fi) {
            const int j = elem_face[e * (dim + 1) + fi];
            const int l = face_l[j], r = face_r[j];
            if (r < 0) continue;
            const int side = l == (int)e ? 0 : 1;
            const int64_t nb = side == 0 ? r : l;
            if (nb == e) continue;          // a periodic self-neighbour is part of D_i already
            const double* Dg = D + (int64_t)j * 2 * dim * NP * NP;
            for (int t = tid; t < dim * NP * NP; t += blockDim.x) {
                Da[t] = Dg[side * dim * NP * NP + t];
                Db[t] = Dg[(1 - side) * dim * NP * NP + t];
            }
            for (int t = tid; t < n * n; t += blockDim.x) K[t] = 0.0;
            __syncthreads();
            add_face_coupling(K, n, dim, NP, Da, Db, lamf[j], muf[j], 1.0);   // K_ie
            __syncthreads();
            const double* Ve = preV + nb * (int64_t)n * n;
            for (int ent = tid; ent < n * n; ent += blockDim.x) {
                const int s = ent / n, q = ent % n;
                double acc = 0;
                for (int s2 = 0; s2 < n; ++s2) acc += K[s * n + s2] * Ve[s2 * n + q];
                kv[ent] = acc;
            }
            const double* Be = preB + nb * (int64_t)n * NG * NG;
            for (int ent = tid; ent < n * NG * NG; ent += blockDim.x) {
                const int q = ent / (NG * NG), a = (ent / NG) % NG, a2 = ent % NG;
                double acc = 0;
                for (int b = 0; b < NG; ++b)
                    for (int b2 = 0; b2 < NG; ++b2)
                        acc += rtp->S[a * NG + b] * Be[q * NG * NG + b * NG + b2] * rtp->S[b2 * NG + a2];
                W[ent] = acc;
            }
            __syncthreads();
            const double c2 = cdt2 * cdt2;
            for (int ent = tid; ent < N * N; ent += blockDim.x) {
                const int R = ent / N, C = ent % N;
                const int k = R / (NG * NP), a = (R / NP) % NG, nn = R % NP;
                const int k2 = C / (NG * NP), a2 = (C / NP) % NG, n2 = C % NP;
                const double* k1 = kv + (k * NP + nn) * n;
                const double* kk2 = kv + (k2 * NP + n2) * n;
                double acc = 0;
                for (int q = 0; q < n; ++q) acc += k1[q] * kk2[q] * W[(q * NG + a) * NG + a2];
                A[R * ldA + C] -= c2 * acc;
            }
            __syncthreads();
        }
        // ---- Gauss-Jordan on [S_i | I] with partial pivoting
        if (tid == 0) s_sing = 0;
        for (int col = 0; col < N; ++col) {
            if (tid == 0) {
                int p = col;
                double best = fabs(A[col * ldA + col]);
                for (int rr = col + 1; rr < N; ++rr) {
                    const double v = fabs(A[rr * ldA + col]);
                    if (v > best) { best = v; p = rr; }
                }
                s_piv = p;
                if (!(best > 0.0)) s_sing = 1;
            }
            __syncthreads();
            if (s_sing) break;
            const int p = s_piv;
            if (p != col)
                for (int t = tid; t < ldA; t += blockDim.x) {
                    const double u = A[col * ldA + t];
                    A[col * ldA + t] = A[p * ldA + t];
                    A[p * ldA + t] = u;
                }
            __syncthreads();
            const double inv = 1.0 / A[col * ldA + col];
            __syncthreads();
            for (int t = tid; t < ldA; t += blockDim.x) A[col * ldA + t] *= inv;
            for (int t = tid; t < N; t += blockDim.x) f[t] = A[t * ldA + col];
            __syncthreads();
            for (int ent = tid; ent < N * ldA; ent += blockDim.x) {
                const int rr = ent / ldA, cc = ent % ldA;
                if (rr != col && cc >= col) A[ent] -= f[rr] * A[col * ldA + cc];
            }
            __syncthreads();
        }
        if (s_sing && tid == 0) atomicExch(status, 1);
        // ---- store S_i^{-1} column-major: out[e][C][R]
        for (int ent = tid; ent < N * N; ent += blockDim.x) {
            const int C = ent / N, R = ent % N;
            const double v = A[R * ldA + N + C];
            if (out64) out64[e * (int64_t)N * N + ent] = v;
            if (out32) out32[e * stride32 + ent] = (float)v;
        }
        __syncthreads();
    }
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ double to_f(double v) { return v; }

// z_e = S_e^{-1} (2 r_e - w_e), w = A P_1 r: one warp per element; lane holds rows lane + 32 i,
// columns of S^{-1} (contiguous, blocks `es` entries apart) are streamed once per group of
// SG shots.  R: arithmetic type, S: storage type of S^{-1}.
template <typename R, typename S, int SG>
__global__ void __launch_bounds__(128) pre2_local_kernel(int64_t n_elem, int N, int64_t es, const S* __restrict__ Sinv,
                                                         const R* __restrict__ r, const int* __restrict__ ridx,
                                                         int64_t ld, const R* __restrict__ w, R* __restrict__ z,
                                                         int nshots, int64_t nvec) {
    extern __shared__ unsigned char smraw[];
    if (ridx) r += (int64_t)(*ridx) * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    R* st = reinterpret_cast<R*>(smraw) + (size_t)warp * SG * N;
    for (int64_t e = blockIdx.x * (int64_t)wpb + warp; e < n_elem; e += (int64_t)gridDim.x * wpb) {
        const S* Se = Sinv + e * es;
        for (int s0 = 0; s0 < nshots; s0 += SG) {
            const int sg = min(SG, nshots - s0);
            for (int q = lane; q < SG * N; q += 32) {
                const int g = q / N, c = q % N;
                const int64_t i = (int64_t)(s0 + g) * nvec + e * N + c;
                st[q] = g < sg ? (R)2 * r[i] - w[i] : (R)0;
            }
            __syncwarp();
            R acc[kP2MaxRows][SG];
#pragma unroll
            for (int i = 0; i < kP2MaxRows; ++i)
#pragma unroll
                for (int g = 0; g < SG; ++g) acc[i][g] = 0;
            for (int c = 0; c < N; ++c) {
                const S* col = Se + (int64_t)c * N;
#pragma unroll
                for (int i = 0; i < kP2MaxRows; ++i) {
                    const int rr = lane + 32 * i;
                    if (rr < N) {
                        const R a = (R)to_f(col[rr]);
#pragma unroll
                        for (int g = 0; g < SG; ++g) acc[i][g] = fma(a, st[g * N + c], acc[i][g]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < kP2MaxRows; ++i) {
                const int rr = lane + 32 * i;
                if (rr < N)
#pragma unroll
                    for (int g = 0; g < SG; ++g)
                        if (g < sg) z[(int64_t)(s0 + g) * nvec + e * N + rr] = acc[i][g];
            }
            __syncwarp();
        }
    }
}

// FP16 storage of the FP32 path's blocks.  Each block is balanced, S^{-1} = diag(r) H diag(c)
// with r_i = max_j |S_ij| and c_j = max_i |S_ij| / r_i, so that every row and column of H
// has its largest entry at magnitude 1 and H is stored in FP16 (11-bit significand, as the
// TF32 rounding of the tensor-core batch path).  One warp per element; lane holds rows
// lane + 32 i of the column-major FP32 block.
__global__ void __launch_bounds__(128) pre2_half_kernel(int64_t n_elem, int N, int64_t es, const float* __restrict__ S32,
                                                        __half* __restrict__ H, float* __restrict__ scl) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int64_t e = blockIdx.x * (int64_t)wpb + warp; e < n_elem; e += (int64_t)gridDim.x * wpb) {
        const float* Se = S32 + e * es;
        __half* He = H + e * (int64_t)N * N;
        float* se = scl + e * 2 * (int64_t)N;
        float rmax[kP2MaxRows];
#pragma unroll
        for (int i = 0; i < kP2MaxRows; ++i) rmax[i] = 0.f;
        for (int c = 0; c < N; ++c)
#pragma unroll
            for (int i = 0; i < kP2MaxRows; ++i) {
                const int rr = lane + 32 * i;
                if (rr < N) rmax[i] = fmaxf(rmax[i], fabsf(Se[(int64_t)c * N + rr]));
            }
        float rinv[kP2MaxRows];
#pragma unroll
        for (int i = 0; i < kP2MaxRows; ++i) {
            const int rr = lane + 32 * i;
            const float rs = rmax[i] > 0.f ? rmax[i] : 1.f;
            rinv[i] = 1.f / rs;
            if (rr < N) se[rr] = rs;
        }
        for (int c = 0; c < N; ++c) {
            float m = 0.f;
#pragma unroll
            for (int i = 0; i < kP2MaxRows; ++i) {
                const int rr = lane + 32 * i;
                if (rr < N) m = fmaxf(m, fabsf(Se[(int64_t)c * N + rr]) * rinv[i]);
            }
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            const float cs = m > 0.f ? m : 1.f;
            if (lane == 0) se[N + c] = cs;
            const float cinv = 1.f / cs;
#pragma unroll
            for (int i = 0; i < kP2MaxRows; ++i) {
                const int rr = lane + 32 * i;
                if (rr < N) He[(int64_t)c * N + rr] = __float2half_rn(Se[(int64_t)c * N + rr] * rinv[i] * cinv);
            }
        }
    }
}

bool pre2_half_supported(const stdg_ctx* c) {
    const int N = c->dim * c->Nphi * c->Ng;
    return N % 2 == 0 && N <= 64 * kP2MaxRows / 2 && N <= 32 * kP2MaxRows;
}

cudaError_t launch_pre2_half(stdg_ctx* c) {
    const int N = c->dim * c->Nphi * c->Ng;
    const int64_t blocks = std::min<int64_t>((c->n_elem + 3) / 4, (int64_t)c->n_sm * 16);
    pre2_half_kernel<<<(unsigned)blocks, 128, 0, c->stream>>>(c->n_elem, N, pre2_stride32(c), c->d_pre2_32,
                                                             reinterpret_cast<__half*>(c->d_pre2_16), c->d_pre2_scl);
    note_launch(c);
    return cudaGetLastError();
}

// z_e = diag(r) H diag(c) (2 r_e - w_e) with FP16 H, one shot: one warp per element, lane
// holds row pairs 2(lane + 32 i), +1 (one 4-byte load of two FP16 values per column); the
// column scales multiply the staged vector, the row scales the accumulated rows.
__global__ void __launch_bounds__(128) pre2_local_half_kernel(int64_t n_elem, int N, const __half* __restrict__ H,
                                                              const float* __restrict__ scl, const float* __restrict__ r,
                                                              const int* __restrict__ ridx, int64_t ld,
                                                              const float* __restrict__ w, float* __restrict__ z) {
    constexpr int PAIRS = kP2MaxRows / 2;   // row pairs per lane: N <= 128
    extern __shared__ unsigned char smraw[];
    if (ridx) r += (int64_t)(*ridx) * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    float* st = reinterpret_cast<float*>(smraw) + (size_t)warp * N;
    for (int64_t e = blockIdx.x * (int64_t)wpb + warp; e < n_elem; e += (int64_t)gridDim.x * wpb) {
        const __half2* He = reinterpret_cast<const __half2*>(H + e * (int64_t)N * N);
        const float* se = scl + e * 2 * (int64_t)N;
        for (int q = lane; q < N; q += 32) {
            const int64_t i = e * N + q;
            st[q] = (2.f * r[i] - w[i]) * se[N + q];
        }
        __syncwarp();
        float2 acc[PAIRS];
#pragma unroll
        for (int i = 0; i < PAIRS; ++i) acc[i] = make_float2(0.f, 0.f);
        const int NH = N / 2;
        for (int c = 0; c < N; ++c) {
            const float x = st[c];
            const __half2* col = He + (int64_t)c * NH;
#pragma unroll
            for (int i = 0; i < PAIRS; ++i) {
                const int pr = lane + 32 * i;
                if (pr < NH) {
                    const float2 a = __half22float2(col[pr]);
                    acc[i].x = fmaf(a.x, x, acc[i].x);
                    acc[i].y = fmaf(a.y, x, acc[i].y);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < PAIRS; ++i) {
            const int pr = lane + 32 * i;
            if (pr < NH) {
                const float2 rs = *reinterpret_cast<const float2*>(se + 2 * pr);
                *reinterpret_cast<float2*>(z + e * N + 2 * pr) = make_float2(acc[i].x * rs.x, acc[i].y * rs.y);
            }
        }
        __syncwarp();
    }
}

static size_t pre2_setup_smem(int dim, int NP, int NG) {
    const int n = dim * NP, N = n * NG;
    return sizeof(double) * ((size_t)N * 2 * N + 2 * (size_t)n * n + (size_t)n * NG * NG + 2 * (size_t)dim * NP * NP + N);
}

bool pre2_supported(const stdg_ctx* c) {
    const int N = c->dim * c->Nphi * c->Ng;
    return N <= 32 * kP2MaxRows && pre2_setup_smem(c->dim, c->Nphi, c->Ng) <= 227 * 1024;
}

cudaError_t launch_pre2_setup(stdg_ctx* c, double dt, int* d_status) {
    const double cfac = c->opt.scheme == STDG_SCHEME_CN ? 0.25 : 1.0;
    const size_t smem = pre2_setup_smem(c->dim, c->Nphi, c->Ng);
    cudaFuncSetAttribute(pre2_setup_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = (int)std::min<int64_t>(c->n_elem, c->n_sm * 8);
    pre2_setup_kernel<<<grid, kP2Threads, smem, c->stream>>>(c->n_elem, c->dim, c->d_rt, c->d_elem_face, c->d_face_l,
                                                             c->d_face_r, c->d_D, c->d_lamf, c->d_muf, c->d_rhoJ, c->d_preV,
                                                             c->d_preB, cfac * dt * dt, c->d_pre2, c->d_pre2_32,
                                                             pre2_stride32(c), d_status);
    note_launch(c);
    return cudaGetLastError();
}

template <typename R, typename S>
static cudaError_t pre2_local_t(stdg_ctx* c, const S* Sinv, int64_t es, const R* r, const int* ridx, int64_t ld,
                                const R* w, R* z, int nshots) {
    const int N = c->dim * c->Nphi * c->Ng;
    if constexpr (std::is_same<R, float>::value) {   // a batch of shots: one GEMM per element pair on the tensor cores
        cudaError_t e;
        if (nshots > 1 && launch_pre2_local_mma(c, r, ridx, ld, w, z, nshots, &e)) return e;
    }
    const int wpb = c->tune.pre2_wpb;
    const int64_t blocks = std::min<int64_t>((c->n_elem + wpb - 1) / wpb, 1 << 30);
    if constexpr (std::is_same<R, float>::value && std::is_same<S, float>::value) {
        // one shot with the FP16 copy of the blocks (half the bytes of the dominant stream)
        if (nshots == 1 && c->d_pre2_16 && c->pre2_bits == 16 && Sinv == c->d_pre2_32) {
            pre2_local_half_kernel<<<(unsigned)blocks, 32 * wpb, sizeof(float) * wpb * N, c->stream>>>(
                c->n_elem, N, reinterpret_cast<const __half*>(c->d_pre2_16), c->d_pre2_scl, r, ridx, ld, w, z);
            note_launch(c);
            return cudaGetLastError();
        }
    }
    if (nshots == 1) {
        pre2_local_kernel<R, S, 1><<<(unsigned)blocks, 32 * wpb, sizeof(R) * wpb * N, c->stream>>>(
            c->n_elem, N, es, Sinv, r, ridx, ld, w, z, nshots, c->nvel);
    } else {
        pre2_local_kernel<R, S, 4><<<(unsigned)blocks, 32 * wpb, sizeof(R) * wpb * 4 * N, c->stream>>>(
            c->n_elem, N, es, Sinv, r, ridx, ld, w, z, nshots, c->nvel);
    }
    note_launch(c);
    return cudaGetLastError();
}

// the element-local step alone, z = S^{-1} (2 r - w), one shot (kernel timing)
cudaError_t launch_pre2_local(stdg_ctx* c, int fp32, const void* r, const void* w, void* z) {
    const int64_t N = c->dim * c->Nphi * c->Ng;
    if (fp32)
        return pre2_local_t<float, float>(c, c->d_pre2_32, pre2_stride32(c), (const float*)r, nullptr, 0,
                                           (const float*)w, (float*)z, 1);
    return pre2_local_t<double, double>(c, c->d_pre2, N * N, (const double*)r, nullptr, 0, (const double*)w, (double*)z, 1);
}

// the element-local step alone for all the context's shots, FP32 (the tensor-core kernel
// for a batch of shots where it applies)
cudaError_t launch_pre2_local_batch(stdg_ctx* c, const float* r, const float* w, float* z) {
    return pre2_local_t<float, float>(c, c->d_pre2_32, pre2_stride32(c), r, nullptr, 0, w, z, c->n_shots);
}

// z = P_2 r for nshots stacked shots: y = P_1 r, w = A y, z = S^{-1} (2 r - w).
// Since D_i y_i = r_i, (2 r - A y)_i = r_i - sum_e N_{i,e} y_e: the neighbour coupling comes
// out of one ordinary operator application.
template <typename R, typename S>
static cudaError_t pre2_apply_t(stdg_ctx* c, const S* Sinv, int64_t es, const R* r, R* z, const int* ridx, int64_t ld,
                                int nshots, bool fp32) {
    R* y = reinterpret_cast<R*>(c->d_p2y);
    R* w = reinterpret_cast<R*>(c->d_p2t);
    cudaError_t e;
    if (fp32) {
        if ((e = launch_pre1_apply32(c, (const float*)r, (float*)y, ridx, ld, nshots)) != cudaSuccess) return e;
        if ((e = launch_apply32(c, c->pre_dt, (const float*)y, (float*)w, 1.0, nullptr, 0, nshots)) != cudaSuccess) return e;
    } else {
        if ((e = launch_pre1_apply(c, (const double*)r, (double*)y, ridx, ld, nshots)) != cudaSuccess) return e;
        if ((e = launch_apply(c, c->pre_dt, (const double*)y, (double*)w, 1.0, nullptr, 0, nshots)) != cudaSuccess) return e;
    }
    return pre2_local_t<R, S>(c, Sinv, es, r, ridx, ld, w, z, nshots);
}

cudaError_t launch_pre2_apply(stdg_ctx* c, const double* r, double* z, const int* ridx, int64_t ld, int nshots) {
    const int64_t N = c->dim * c->Nphi * c->Ng;
    return pre2_apply_t<double, double>(c, c->d_pre2, N * N, r, z, ridx, ld, nshots, false);
}

cudaError_t launch_pre2_apply32(stdg_ctx* c, const float* r, float* z, const int* ridx, int64_t ld, int nshots) {
    return pre2_apply_t<float, float>(c, c->d_pre2_32, pre2_stride32(c), r, z, ridx, ld, nshots, true);
}

}  // namespace stdg
