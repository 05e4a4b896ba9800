// Per-step solve of the Schur velocity system, entirely on the device (Sec. 4,
// "... we can still solve the system using a matrix-free GMRES algorithm ..."; CG for the
// symmetric positive definite Crank-Nicolson case, Theorems 1-2).
//
// Every Krylov scalar (dot products, Hessenberg column, Givens rotations, residual
// estimate, loop flags) lives in device memory; loops are CUDA-graph WHILE nodes whose
// condition a small kernel sets with cudaGraphSetConditional, so one graph launch runs
// a whole time step with no host round trip.  With use_graph = 0 the same kernels run
// from a host loop that reads the flag after each body (a debugging aid).
//
// Solvers
//   CG        (Crank-Nicolson)  r = b - A x; standard recurrences; FP64 dots.
//   GMRES(m)  (space-time DG)   restarted, classical Gram-Schmidt with one
//                               re-orthogonalisation pass, Givens rotations on the device,
//                               true residual checked at every restart.
//   Mixed     FP64 iterative refinement around an FP32 CG / GMRES: r = b - A64 x in FP64,
//             solve A32 d = r/|r| to inner_tol, x += |r| d, stop at rel_tol in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "stdg_internal.h"

namespace stdg {

constexpr int kMaxRestart = 64;
constexpr int kRedBlocks = 1216;    // 8 x 152 SMs
constexpr int kRedThreads = 256;
constexpr int kDotChunk = 16;       // basis vectors per pass of the multi-dot kernels

struct DevScalars {
    // current Krylov level
    double bnorm, tol_abs;
    double bmin;          // min over shots of ||b_shot|| (stacked multi-shot solves)
    double rr, pq, alpha, beta;                   // CG
    double gbeta, resid;                          // GMRES
    double hcol[kMaxRestart + 2], hpass[kMaxRestart + 2];
    double H[(kMaxRestart + 1) * kMaxRestart];
    double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
    int j, iters, converged, flag_outer, flag_inner, max_iters, m, zero_x;
    // FP64 refinement level (mixed precision)
    double ir_bnorm, ir_tol_abs, ir_rnorm, ir_scale;
    int ir_flag, ir_count, ir_max, ir_conv;
    // statistics, reset by the host before a batch of steps
    int st_total, st_max, st_refine, st_notconv;
    double st_final_rel, st_iters_sum;
    unsigned long long launches;      // kernel executions since the last reset
};

struct Workspace {
    int m = 30;
    int64_t n = 0, ldv = 0;
    DevScalars* sc = nullptr;
    double* partials = nullptr;   // (kMaxRestart + 2) * kRedBlocks
    double* dparams = nullptr;    // t^n, dt, step index
    double *V = nullptr, *w = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *t = nullptr;   // FP64
    float *V32 = nullptr, *w32 = nullptr, *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    float *z32 = nullptr, *t32 = nullptr;
    cudaStream_t side[6] = {};
    int depth = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double graph_dt = -1.0;
    std::vector<void*> owned;   // device buffers of this workspace
};

static Workspace* W(stdg_ctx* c) { return reinterpret_cast<Workspace*>(c->ws); }

// ---------------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    return s;   // valid in thread 0
}

// Per-thread dot-product accumulator: FP64 for FP64 vectors; for FP32 vectors an error-free
// (TwoProduct + TwoSum) pair of floats, so FP32 inner products carry FP64-level accuracy
// without FP64 arithmetic (GB300's FP64 rate is 1/64 of FP32).
template <typename R> struct Acc;
template <> struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float a, float b) {
        const float p = a * b;
        const float pe = fmaf(a, b, -p);
        const float t = s + p;
        const float z = t - s;
        const float te = (s - (t - z)) + (p - z);
        s = t;
        c += te + pe;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// 16-byte vector access: VW = 4 floats or 2 doubles per load/store.  Streaming kernels walk
// n / VW vectors with a grid-stride loop and give the n % VW tail to one thread; every
// pointer they vectorise is 16-byte aligned (separate allocations, or basis columns at a
// leading dimension that is a multiple of 64 elements).
template <typename R> struct VL;
template <> struct VL<float> {
    static constexpr int W = 4;
    __device__ __forceinline__ static void ld(const float* p, float (&o)[4]) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    }
    __device__ __forceinline__ static void st(float* p, const float (&o)[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    }
};
template <> struct VL<double> {
    static constexpr int W = 2;
    __device__ __forceinline__ static void ld(const double* p, double (&o)[2]) {
        const double2 t = *reinterpret_cast<const double2*>(p);
        o[0] = t.x; o[1] = t.y;
    }
    __device__ __forceinline__ static void st(double* p, const double (&o)[2]) {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
    }
};

// sum of partials[0..nb) in a single block; result in thread 0
__device__ __forceinline__ double sum_partials(const double* p, int nb) {
    double v = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) v += p[i];
    return block_sum(v);
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int use, int v) {
    if (use) cudaGraphSetConditional(h, v ? 1u : 0u);
}

template <typename A, typename B>
__global__ void dot_partial_kernel(int64_t n, const A* __restrict__ a, const B* __restrict__ b, double* __restrict__ out) {
    Acc<A> acc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc.add(a[i], b[i]);
    double s = block_sum(acc.value());
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// per-shot partial sums of ||b_s||^2: grid (G, nshots), part[s * G + blk]
__global__ void shot_norm_partial_kernel(int64_t nvec, const double* __restrict__ b, double* __restrict__ part) {
    const double* bs = b + (int64_t)blockIdx.y * nvec;
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x)
        acc = fma(bs[i], bs[i], acc);
    double s = block_sum(acc);
    if (threadIdx.x == 0) part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// sc->bmin = min_s ||b_s||: a stacked solve stopped at ||r|| <= tol * bmin meets tol for every shot
__global__ void shot_min_kernel(DevScalars* sc, const double* part, int G, int nshots) {
    double mn = 0.0;
    for (int s = 0; s < nshots; ++s) {
        double t = sum_partials(part + s * G, G);
        if (threadIdx.x == 0) {
            const double nrm = sqrt(t);
            mn = (s == 0 || nrm < mn) ? nrm : mn;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) sc->bmin = mn;
}

__global__ void zero_if_kernel(int64_t n, double* x, const int* flag) {
    if (!*flag) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = 0;
}

// ---------------------------------------------------------------------------------
// (Preconditioned) CG kernels (R = vector type, scalars FP64).  Without a preconditioner
// z aliases r and rz = rr.
// ---------------------------------------------------------------------------------
template <typename R>
__global__ void cg_res_kernel(int64_t n, const R* __restrict__ b, const R* __restrict__ Ax, R* __restrict__ r,
                              double* __restrict__ part) {
    double rr = 0, bb = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R ri = b[i] - Ax[i];
        r[i] = ri;
        rr += (double)ri * (double)ri;
        bb += (double)b[i] * (double)b[i];
    }
    double s1 = block_sum(rr);
    double s2 = block_sum(bb);
    if (threadIdx.x == 0) { part[blockIdx.x] = s1; part[kRedBlocks + blockIdx.x] = s2; }
}

// bnorm_given < 0: use ||b|| from the partials; partials: [0] rr, [1] bb, [2] rz
__global__ void cg_init_final_kernel(DevScalars* sc, const double* part, double rel_tol, int max_iters,
                                     double bnorm_given, int gate_ir, cudaGraphConditionalHandle h, int use_h,
                                     int use_bmin) {
    double rr = sum_partials(part, kRedBlocks);
    double bb = sum_partials(part + kRedBlocks, kRedBlocks);
    double rz = sum_partials(part + 2 * kRedBlocks, kRedBlocks);
    if (threadIdx.x == 0) {
        const int active = gate_ir ? sc->ir_flag : 1;
        sc->rr = rr;
        sc->pq = rz;                       // holds r.z between iterations
        sc->bnorm = bnorm_given >= 0 ? bnorm_given : sqrt(bb);
        sc->tol_abs = rel_tol * (use_bmin ? sc->bmin : sc->bnorm);
        sc->iters = 0;
        sc->max_iters = max_iters;
        sc->zero_x = active && sc->bnorm == 0.0;
        sc->converged = !active || sqrt(rr) <= sc->tol_abs;
        sc->flag_inner = !sc->converged && max_iters > 0;
        set_cond(h, use_h, sc->flag_inner);
    }
}

template <typename R>
__global__ void copy_kernel(int64_t n, const R* __restrict__ a, R* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = a[i];
}

__global__ void cg_alpha_kernel(DevScalars* sc, const double* part) {
    double pq = sum_partials(part, kRedBlocks);
    if (threadIdx.x == 0) sc->alpha = pq != 0.0 ? sc->pq / pq : 0.0;
}

template <typename R>
__global__ void cg_update_kernel(int64_t n, const DevScalars* __restrict__ sc, R* __restrict__ x, R* __restrict__ r,
                                 const R* __restrict__ p, const R* __restrict__ q, double* __restrict__ part) {
    const double a = sc->alpha;
    double rr = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] = (R)((double)x[i] + a * (double)p[i]);
        const R ri = (R)((double)r[i] - a * (double)q[i]);
        r[i] = ri;
        rr += (double)ri * (double)ri;
    }
    double s = block_sum(rr);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// partials: [0] rr, [2] rz (r.z after the preconditioner)
__global__ void cg_beta_kernel(DevScalars* sc, const double* part, cudaGraphConditionalHandle h, int use_h) {
    double rr = sum_partials(part, kRedBlocks);
    double rz = sum_partials(part + 2 * kRedBlocks, kRedBlocks);
    if (threadIdx.x == 0) {
        sc->beta = sc->pq != 0.0 ? rz / sc->pq : 0.0;
        sc->pq = rz;
        sc->rr = rr;
        sc->iters += 1;
        sc->converged = sqrt(rr) <= sc->tol_abs;
        sc->flag_inner = !sc->converged && sc->iters < sc->max_iters;
        set_cond(h, use_h, sc->flag_inner);
    }
}

template <typename R>
__global__ void cg_p_kernel(int64_t n, const DevScalars* __restrict__ sc, const R* __restrict__ z, R* __restrict__ p) {
    const double b = sc->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (R)((double)z[i] + b * (double)p[i]);
}

// ---------------------------------------------------------------------------------
// GMRES kernels
// ---------------------------------------------------------------------------------
template <typename R>
__global__ void gm_res_kernel(int64_t n, const R* __restrict__ b, const R* __restrict__ Ax, R* __restrict__ v0,
                             double* __restrict__ part) {
    constexpr int W = VL<R>::W;
    const int64_t nv = n / W;
    Acc<R> rr;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
        R bb[W], aa[W];
        VL<R>::ld(b + g * W, bb);
        VL<R>::ld(Ax + g * W, aa);
#pragma unroll
        for (int u = 0; u < W; ++u) { bb[u] -= aa[u]; rr.add(bb[u], bb[u]); }
        VL<R>::st(v0 + g * W, bb);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = nv * W; i < n; ++i) { const R ri = b[i] - Ax[i]; v0[i] = ri; rr.add(ri, ri); }
    double s = block_sum(rr.value());
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// set up one GMRES solve: ||b|| (from partials, or given), tolerance, counters
__global__ void gm_init_kernel(DevScalars* sc, const double* part, double rel_tol, int max_iters, int m,
                               double bnorm_given, int gate_ir, cudaGraphConditionalHandle h, int use_h, int use_bmin) {
    double bb = sum_partials(part, kRedBlocks);
    if (threadIdx.x == 0) {
        const int active = gate_ir ? sc->ir_flag : 1;
        sc->bnorm = bnorm_given >= 0 ? bnorm_given : sqrt(bb);
        sc->tol_abs = rel_tol * (use_bmin ? sc->bmin : sc->bnorm);
        sc->iters = 0;
        sc->max_iters = max_iters;
        sc->m = m;
        sc->converged = !active;
        sc->zero_x = active && sc->bnorm == 0.0;
        sc->flag_outer = active && sc->bnorm != 0.0;
        if (sc->zero_x) sc->converged = 1;
        set_cond(h, use_h, sc->flag_outer);
    }
}

__global__ void gm_cycle_start_kernel(DevScalars* sc, const double* part, cudaGraphConditionalHandle h, int use_h) {
    double rr = sum_partials(part, kRedBlocks);
    if (threadIdx.x == 0) {
        const double beta = sqrt(rr);
        sc->gbeta = beta;
        sc->resid = beta;
        sc->j = 0;
        sc->converged = beta <= sc->tol_abs;
        for (int k = 0; k <= sc->m; ++k) sc->g[k] = 0.0;
        sc->g[0] = beta;
        sc->flag_inner = !sc->converged && sc->iters < sc->max_iters;
        set_cond(h, use_h, sc->flag_inner);
    }
}

template <typename R>
__global__ void gm_scale0_kernel(int64_t n, const DevScalars* __restrict__ sc, R* __restrict__ v0) {
    if (!sc->flag_inner) return;
    constexpr int W = VL<R>::W;
    const R s = (R)(1.0 / sc->gbeta);
    const int64_t nv = n / W;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
        R a[W];
        VL<R>::ld(v0 + g * W, a);
#pragma unroll
        for (int u = 0; u < W; ++u) a[u] *= s;
        VL<R>::st(v0 + g * W, a);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = nv * W; i < n; ++i) v0[i] *= s;
}

// partials[k][blk] = sum_i V_k[i] w[i], k = 0..j  (basis columns at stride ldv)
template <typename R>
__global__ void __launch_bounds__(256) gm_mdot_kernel(int64_t n, int64_t ldv, const DevScalars* __restrict__ sc,
                                                      const R* __restrict__ V, const R* __restrict__ w,
                                                      double* __restrict__ part) {
    constexpr int W = VL<R>::W;
    const int J = sc->j;
    const int64_t nv = n / W;
    for (int k0 = 0; k0 <= J; k0 += kDotChunk) {
        Acc<R> acc[kDotChunk];
        const int kn = min(kDotChunk, J + 1 - k0);
        for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
            R wv[W];
            VL<R>::ld(w + g * W, wv);
#pragma unroll
            for (int kk = 0; kk < kDotChunk; ++kk)
                if (kk < kn) {
                    R vv[W];
                    VL<R>::ld(V + (int64_t)(k0 + kk) * ldv + g * W, vv);
#pragma unroll
                    for (int u = 0; u < W; ++u) acc[kk].add(vv[u], wv[u]);
                }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0)
            for (int64_t i = nv * W; i < n; ++i)
#pragma unroll
                for (int kk = 0; kk < kDotChunk; ++kk)
                    if (kk < kn) acc[kk].add(V[(int64_t)(k0 + kk) * ldv + i], w[i]);
#pragma unroll
        for (int kk = 0; kk < kDotChunk; ++kk) {   // constant bound keeps acc[] in registers
            if (kk < kn) {                            // kn is uniform over the block
                double s = block_sum(acc[kk].value());
                if (threadIdx.x == 0) part[(k0 + kk) * kRedBlocks + blockIdx.x] = s;
            }
        }
    }
}

// Second Gram-Schmidt pass fused with the first subtraction:
// w <- w - sum_k h1[k] V_k, then partials of V_k . w for the re-orthogonalisation.
template <typename R>
__global__ void __launch_bounds__(256) gm_orth_fused_kernel(int64_t n, int64_t ldv, const DevScalars* __restrict__ sc,
                                                            const R* __restrict__ V, R* __restrict__ w,
                                                            double* __restrict__ part) {
    constexpr int W = VL<R>::W;
    const int J = sc->j;
    __shared__ R h[kMaxRestart + 2];
    for (int k = threadIdx.x; k <= J; k += blockDim.x) h[k] = (R)sc->hpass[k];
    __syncthreads();
    const int64_t nv = n / W;
    for (int k0 = 0; k0 <= J; k0 += kDotChunk) {
        Acc<R> acc[kDotChunk];
        const int kn = min(kDotChunk, J + 1 - k0);
        for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
            R wv[W];
            VL<R>::ld(w + g * W, wv);
            if (k0 == 0) {   // first chunk: form and store the projected w (in the vector precision)
                for (int k = 0; k <= J; ++k) {
                    R vv[W];
                    VL<R>::ld(V + (int64_t)k * ldv + g * W, vv);
#pragma unroll
                    for (int u = 0; u < W; ++u) wv[u] = fma(-h[k], vv[u], wv[u]);
                }
                VL<R>::st(w + g * W, wv);
            }
#pragma unroll
            for (int kk = 0; kk < kDotChunk; ++kk)
                if (kk < kn) {
                    R vv[W];
                    VL<R>::ld(V + (int64_t)(k0 + kk) * ldv + g * W, vv);
#pragma unroll
                    for (int u = 0; u < W; ++u) acc[kk].add(vv[u], wv[u]);
                }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0)
            for (int64_t i = nv * W; i < n; ++i) {
                R wi = w[i];
                if (k0 == 0) {
                    for (int k = 0; k <= J; ++k) wi = fma(-h[k], V[(int64_t)k * ldv + i], wi);
                    w[i] = wi;
                }
#pragma unroll
                for (int kk = 0; kk < kDotChunk; ++kk)
                    if (kk < kn) acc[kk].add(V[(int64_t)(k0 + kk) * ldv + i], wi);
            }
#pragma unroll
        for (int kk = 0; kk < kDotChunk; ++kk) {
            if (kk < kn) {
                double s = block_sum(acc[kk].value());
                if (threadIdx.x == 0) part[(k0 + kk) * kRedBlocks + blockIdx.x] = s;
            }
        }
    }
}

__global__ void gm_mdot_final_kernel(DevScalars* sc, const double* part, int pass) {
    const int J = sc->j;
    for (int k = 0; k <= J; ++k) {
        double s = sum_partials(part + k * kRedBlocks, kRedBlocks);
        if (threadIdx.x == 0) {
            sc->hpass[k] = s;
            sc->hcol[k] = pass == 0 ? s : sc->hcol[k] + s;
        }
        __syncthreads();
    }
}

// w -= sum_k hpass[k] V_k; optionally partial ||w||^2
template <typename R>
__global__ void __launch_bounds__(256) gm_maxpy_kernel(int64_t n, int64_t ldv, const DevScalars* __restrict__ sc,
                                                       const R* __restrict__ V, R* __restrict__ w, double* __restrict__ part,
                                                       int want_norm) {
    constexpr int W = VL<R>::W;
    const int J = sc->j;
    __shared__ R h[kMaxRestart + 2];
    for (int k = threadIdx.x; k <= J; k += blockDim.x) h[k] = (R)sc->hpass[k];
    __syncthreads();
    const int64_t nv = n / W;
    Acc<R> nn;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
        R wv[W];
        VL<R>::ld(w + g * W, wv);
        for (int k = 0; k <= J; ++k) {
            R vv[W];
            VL<R>::ld(V + (int64_t)k * ldv + g * W, vv);
#pragma unroll
            for (int u = 0; u < W; ++u) wv[u] = fma(-h[k], vv[u], wv[u]);
        }
        VL<R>::st(w + g * W, wv);
#pragma unroll
        for (int u = 0; u < W; ++u) nn.add(wv[u], wv[u]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = nv * W; i < n; ++i) {
            R wi = w[i];
            for (int k = 0; k <= J; ++k) wi = fma(-h[k], V[(int64_t)k * ldv + i], wi);
            w[i] = wi;
            nn.add(wi, wi);
        }
    if (want_norm) {
        double s = block_sum(nn.value());
        if (threadIdx.x == 0) part[blockIdx.x] = s;
    }
}

__global__ void gm_norm_final_kernel(DevScalars* sc, const double* part) {
    double s = sum_partials(part, kRedBlocks);
    if (threadIdx.x == 0) sc->hcol[sc->j + 1] = sqrt(s);
}

template <typename R>
__global__ void gm_next_kernel(int64_t n, int64_t ldv, const DevScalars* __restrict__ sc, const R* __restrict__ w,
                               R* __restrict__ V) {
    constexpr int W = VL<R>::W;
    const int J = sc->j;
    const double hh = sc->hcol[J + 1];
    const R s = (R)(hh > 0.0 ? 1.0 / hh : 0.0);
    R* vn = V + (int64_t)(J + 1) * ldv;
    const int64_t nv = n / W;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
        R a[W];
        VL<R>::ld(w + g * W, a);
#pragma unroll
        for (int u = 0; u < W; ++u) a[u] *= s;
        VL<R>::st(vn + g * W, a);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = nv * W; i < n; ++i) vn[i] = w[i] * s;
}

__global__ void gm_givens_kernel(DevScalars* sc, cudaGraphConditionalHandle h, int use_h) {
    if (threadIdx.x != 0) return;
    const int J = sc->j, m = sc->m;
    double* hc = sc->hcol;
    for (int i = 0; i < J; ++i) {
        const double t = sc->cs[i] * hc[i] + sc->sn[i] * hc[i + 1];
        hc[i + 1] = -sc->sn[i] * hc[i] + sc->cs[i] * hc[i + 1];
        hc[i] = t;
    }
    const double a = hc[J], b = hc[J + 1];
    const double den = hypot(a, b);
    double cs = 1.0, sn = 0.0;
    if (den > 0.0) { cs = a / den; sn = b / den; }
    sc->cs[J] = cs;
    sc->sn[J] = sn;
    hc[J] = den;
    hc[J + 1] = 0.0;
    for (int i = 0; i <= J; ++i) sc->H[i * kMaxRestart + J] = hc[i];
    sc->g[J + 1] = -sn * sc->g[J];
    sc->g[J] = cs * sc->g[J];
    sc->resid = fabs(sc->g[J + 1]);
    sc->iters += 1;
    sc->j = J + 1;
    const int done = sc->resid <= sc->tol_abs || den == 0.0;
    sc->flag_inner = !done && sc->j < m && sc->iters < sc->max_iters;
    set_cond(h, use_h, sc->flag_inner);
}

// y = R^{-1} g (upper triangular, size j)
__global__ void gm_solve_kernel(DevScalars* sc) {
    if (threadIdx.x != 0) return;
    const int J = sc->j;
    for (int i = J - 1; i >= 0; --i) {
        double s = sc->g[i];
        for (int k = i + 1; k < J; ++k) s -= sc->H[i * kMaxRestart + k] * sc->y[k];
        const double d = sc->H[i * kMaxRestart + i];
        sc->y[i] = d != 0.0 ? s / d : 0.0;
    }
}

template <typename R>
__global__ void gm_update_x_kernel(int64_t n, int64_t ldv, const DevScalars* __restrict__ sc, const R* __restrict__ V,
                                   R* __restrict__ x) {
    constexpr int W = VL<R>::W;
    const int J = sc->j;
    if (J == 0) return;
    __shared__ R y[kMaxRestart];
    for (int k = threadIdx.x; k < J; k += blockDim.x) y[k] = (R)sc->y[k];
    __syncthreads();
    const int64_t nv = n / W;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
        R a[W];
        VL<R>::ld(x + g * W, a);
        for (int k = 0; k < J; ++k) {
            R vv[W];
            VL<R>::ld(V + (int64_t)k * ldv + g * W, vv);
#pragma unroll
            for (int u = 0; u < W; ++u) a[u] = fma(y[k], vv[u], a[u]);
        }
        VL<R>::st(x + g * W, a);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = nv * W; i < n; ++i) {
            R a = x[i];
            for (int k = 0; k < J; ++k) a = fma(y[k], V[(int64_t)k * ldv + i], a);
            x[i] = a;
        }
}

// t = sum_{k<j} y_k V_k (right preconditioning: x += P^{-1} t afterwards)
template <typename R>
__global__ void gm_combine_kernel(int64_t n, int64_t ldv, const DevScalars* __restrict__ sc, const R* __restrict__ V,
                                  R* __restrict__ t) {
    constexpr int W = VL<R>::W;
    const int J = sc->j;
    __shared__ R y[kMaxRestart];
    for (int k = threadIdx.x; k < J; k += blockDim.x) y[k] = (R)sc->y[k];
    __syncthreads();
    const int64_t nv = n / W;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
        R a[W];
#pragma unroll
        for (int u = 0; u < W; ++u) a[u] = 0;
        for (int k = 0; k < J; ++k) {
            R vv[W];
            VL<R>::ld(V + (int64_t)k * ldv + g * W, vv);
#pragma unroll
            for (int u = 0; u < W; ++u) a[u] = fma(y[k], vv[u], a[u]);
        }
        VL<R>::st(t + g * W, a);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = nv * W; i < n; ++i) {
            R a = 0;
            for (int k = 0; k < J; ++k) a = fma(y[k], V[(int64_t)k * ldv + i], a);
            t[i] = a;
        }
}

template <typename R>
__global__ void axpy_kernel(int64_t n, R* __restrict__ x, const R* __restrict__ z) {
    constexpr int W = VL<R>::W;
    const int64_t nv = n / W;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
        R a[W], b[W];
        VL<R>::ld(x + g * W, a);
        VL<R>::ld(z + g * W, b);
#pragma unroll
        for (int u = 0; u < W; ++u) a[u] += b[u];
        VL<R>::st(x + g * W, a);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = nv * W; i < n; ++i) x[i] += z[i];
}

__global__ void gm_cycle_end_kernel(DevScalars* sc, cudaGraphConditionalHandle h, int use_h) {
    if (threadIdx.x != 0) return;
    sc->j = 0;
    sc->flag_outer = !sc->converged && sc->iters < sc->max_iters;
    set_cond(h, use_h, sc->flag_outer);
}

// ---------------------------------------------------------------------------------
// FP64 iterative refinement around the FP32 solver
// ---------------------------------------------------------------------------------
__global__ void ir_init_kernel(DevScalars* sc, const double* part, double rel_tol, int ir_max,
                               cudaGraphConditionalHandle h, int use_h, int use_bmin) {
    double bb = sum_partials(part, kRedBlocks);
    if (threadIdx.x == 0) {
        sc->ir_bnorm = sqrt(bb);
        sc->ir_tol_abs = rel_tol * (use_bmin ? sc->bmin : sc->ir_bnorm);
        sc->ir_count = 0;
        sc->ir_max = ir_max;
        sc->ir_flag = 1;
        sc->ir_conv = 0;
        sc->zero_x = sc->ir_bnorm == 0.0;
        if (sc->zero_x) sc->ir_conv = 1;
        if (sc->zero_x) sc->ir_flag = 0;
        set_cond(h, use_h, sc->ir_flag);
    }
}

__global__ void ir_check_kernel(DevScalars* sc, const double* part, int max_total) {
    double rr = sum_partials(part, kRedBlocks);
    if (threadIdx.x == 0) {
        sc->ir_rnorm = sqrt(rr);
        const int conv = sc->ir_rnorm <= sc->ir_tol_abs;
        sc->ir_conv = conv;
        sc->ir_flag = !conv && sc->ir_count < sc->ir_max && sc->st_total < max_total;
        sc->ir_scale = sc->ir_rnorm > 0.0 ? 1.0 / sc->ir_rnorm : 0.0;
    }
}

// r32 = r64 * scale; x32 = 0   (when the refinement continues)
__global__ void ir_convert_kernel(int64_t n, const DevScalars* __restrict__ sc, const double* __restrict__ r64,
                                  float* __restrict__ r32, float* __restrict__ x32) {
    if (!sc->ir_flag) return;
    const double s = sc->ir_scale;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        r32[i] = (float)(r64[i] * s);
        x32[i] = 0.0f;
    }
}

// x += x32 / scale
__global__ void ir_update_kernel(int64_t n, const DevScalars* __restrict__ sc, const float* __restrict__ x32, double* __restrict__ x) {
    if (!sc->ir_flag) return;
    const double s = sc->ir_rnorm;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += s * (double)x32[i];
}

__global__ void ir_end_kernel(DevScalars* sc, cudaGraphConditionalHandle h, int use_h) {
    if (threadIdx.x != 0) return;
    if (sc->ir_flag) {
        sc->ir_count += 1;
        sc->st_total += sc->iters;
    }
    set_cond(h, use_h, sc->ir_flag);
}

// per-solve statistics; mode 0 = GMRES, 1 = CG, 2 = mixed (refinement level)
__global__ void solve_stats_kernel(DevScalars* sc, int mode, int use_bmin) {
    if (threadIdx.x != 0) return;
    int it;
    double rel;
    if (mode == 2) {
        it = sc->st_total;          // accumulated by ir_end over the refinement sweeps
        sc->st_total = 0;
        const double bn = use_bmin ? sc->bmin : sc->ir_bnorm;
        rel = bn > 0 ? sc->ir_rnorm / bn : 0.0;
        sc->st_refine += sc->ir_count;
        if (!sc->ir_conv) sc->st_notconv = 1;
    } else {
        it = sc->iters;
        const double r = mode == 1 ? sqrt(sc->rr) : sc->resid;
        const double bn = use_bmin ? sc->bmin : sc->bnorm;
        rel = bn > 0 ? r / bn : 0.0;
        if (!sc->converged) sc->st_notconv = 1;
    }
    sc->st_final_rel = rel;
    sc->st_max = max(sc->st_max, it);
    sc->st_iters_sum += (double)it;
}

// adds a loop body's (or a step's straight-line) kernel count, itself included
__global__ void count_kernel(DevScalars* sc, long k) {
    if (threadIdx.x == 0) sc->launches += (unsigned long long)k;
}

__global__ void step_begin_kernel(double* dparams, double dt) {
    if (threadIdx.x == 0) dparams[1] = dt;
}
__global__ void step_end_kernel(double* dparams, double dt) {
    if (threadIdx.x == 0) { dparams[0] += dt; dparams[2] += 1.0; }
}

// ---------------------------------------------------------------------------------
// control flow: a WHILE loop either as a graph conditional node (during capture) or a
// host loop that reads the flag after each body.
// ---------------------------------------------------------------------------------
struct Flow {
    stdg_ctx* c;
    Workspace* ws;
    bool graph;
    cudaError_t err = cudaSuccess;

    template <class Init, class Body>
    void loop(const int* d_flag, Init init, Body body) {
        if (err != cudaSuccess) return;
        if (!graph) {
            init(cudaGraphConditionalHandle(0), 0);
            for (long guard = 0; guard < 100000000L; ++guard) {
                int f = 0;
                err = cudaMemcpyAsync(&f, d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
                if (err == cudaSuccess) err = cudaStreamSynchronize(c->stream);
                if (err != cudaSuccess || !f) break;
                run_body(body, cudaGraphConditionalHandle(0), 0);
            }
            return;
        }
        cudaStream_t s = c->stream;
        cudaStreamCaptureStatus st;
        cudaGraph_t g;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        if ((err = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd)) != cudaSuccess) return;
        cudaGraphConditionalHandle h;
        if ((err = cudaGraphConditionalHandleCreate(&h, g, 0, 0)) != cudaSuccess) return;
        init(h, 1);
        if ((err = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd)) != cudaSuccess) return;
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        if ((err = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p)) != cudaSuccess) return;
        cudaGraph_t body_g = p.conditional.phGraph_out[0];
        cudaStream_t s2 = ws->side[ws->depth++];
        err = cudaStreamBeginCaptureToGraph(s2, body_g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (err == cudaSuccess) {
            c->stream = s2;
            run_body(body, h, 1);
            c->stream = s;
            cudaGraph_t tmp;
            cudaError_t e2 = cudaStreamEndCapture(s2, &tmp);
            if (err == cudaSuccess) err = e2;
        }
        ws->depth--;
        if (err == cudaSuccess) err = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    }
    void check(cudaError_t e) { if (err == cudaSuccess && e != cudaSuccess) err = e; }

    // one loop body in its own launch-count scope, closed by a count kernel
    template <class Body>
    void run_body(Body& body, cudaGraphConditionalHandle h, int use) {
        c->scopes.push_back(0);
        body(h, use);
        const long k = c->scopes.back() + 1;
        c->scopes.pop_back();
        count_kernel<<<1, 32, 0, c->stream>>>(ws->sc, k);
    }
};

static unsigned vec_blocks(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, kRedBlocks); }

// ---- (P)CG on vectors of type R; apply(x, y): y = A x; prec(r, z): z = P^{-1} r or null --------
template <typename R, class Apply, class Prec>
static void solve_cg(Flow& F, Apply apply, Prec prec, bool use_prec, const R* b, R* x, R* r, R* p, R* q, R* z,
                     double rel_tol, int max_iters, double bnorm_given, int gate_ir, int use_bmin) {
    stdg_ctx* c = F.c;
    Workspace* ws = F.ws;
    const int64_t n = ws->n;
    R* zz = use_prec ? z : r;
    F.loop(&ws->sc->flag_inner,
           [&](cudaGraphConditionalHandle h, int use) {
               F.check(apply(x, q));
               cg_res_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, b, q, r, ws->partials); note_launch(c);
               if (use_prec) F.check(prec(r, zz));
               dot_partial_kernel<R, R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, r, zz, ws->partials + 2 * kRedBlocks); note_launch(c);
               cg_init_final_kernel<<<1, kRedThreads, 0, c->stream>>>(ws->sc, ws->partials, rel_tol, max_iters, bnorm_given,
                                                                      gate_ir, h, use, use_bmin); note_launch(c);
               copy_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, zz, p); note_launch(c);
           },
           [&](cudaGraphConditionalHandle h, int use) {
               F.check(apply(p, q));
               dot_partial_kernel<R, R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, p, q, ws->partials); note_launch(c);
               cg_alpha_kernel<<<1, kRedThreads, 0, c->stream>>>(ws->sc, ws->partials); note_launch(c);
               cg_update_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ws->sc, x, r, p, q, ws->partials); note_launch(c);
               if (use_prec) F.check(prec(r, zz));
               dot_partial_kernel<R, R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, r, zz, ws->partials + 2 * kRedBlocks); note_launch(c);
               cg_beta_kernel<<<1, kRedThreads, 0, c->stream>>>(ws->sc, ws->partials, h, use); note_launch(c);
               cg_p_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ws->sc, zz, p); note_launch(c);
               F.check(cudaGetLastError());
           });
}

// ---- GMRES(m) on vectors of type R -----------------------------------------------------
template <typename R, class Apply, class ApplyIdx, class Prec>
static void solve_gmres(Flow& F, Apply apply, ApplyIdx apply_idx, Prec prec, bool use_prec, const R* b, R* x, R* V, R* w,
                        R* zbuf, R* tbuf, double rel_tol, int max_iters, double bnorm_given, int gate_ir, int use_bmin) {
    stdg_ctx* c = F.c;
    Workspace* ws = F.ws;
    const int64_t n = ws->n, ldv = ws->ldv;
    const int m = ws->m;
    DevScalars* sc = ws->sc;
    F.loop(&sc->flag_outer,
           [&](cudaGraphConditionalHandle h, int use) {
               dot_partial_kernel<R, R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, b, b, ws->partials); note_launch(c);
               gm_init_kernel<<<1, kRedThreads, 0, c->stream>>>(sc, ws->partials, rel_tol, max_iters, m, bnorm_given, gate_ir, h, use,
                                                                use_bmin); note_launch(c);
           },
           [&](cudaGraphConditionalHandle h_outer, int use_outer) {
               // restart cycle: true residual, then Arnoldi
               F.check(apply(x, w));
               gm_res_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, b, w, V, ws->partials); note_launch(c);
               F.loop(&sc->flag_inner,
                      [&](cudaGraphConditionalHandle h, int use) {
                          gm_cycle_start_kernel<<<1, kRedThreads, 0, c->stream>>>(sc, ws->partials, h, use); note_launch(c);
                          gm_scale0_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, sc, V); note_launch(c);
                      },
                      [&](cudaGraphConditionalHandle h, int use) {
                          if (use_prec) {   // right preconditioning: w = A P^{-1} v_j
                              F.check(prec(V, zbuf, &sc->j, ldv));
                              F.check(apply(zbuf, w));
                          } else {
                              F.check(apply_idx(V, &sc->j, w));
                          }
                          // classical Gram-Schmidt twice, in three passes over the basis
                          gm_mdot_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ldv, sc, V, w, ws->partials); note_launch(c);
                          gm_mdot_final_kernel<<<1, kRedThreads, 0, c->stream>>>(sc, ws->partials, 0); note_launch(c);
                          gm_orth_fused_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ldv, sc, V, w, ws->partials); note_launch(c);
                          gm_mdot_final_kernel<<<1, kRedThreads, 0, c->stream>>>(sc, ws->partials, 1); note_launch(c);
                          gm_maxpy_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ldv, sc, V, w, ws->partials, 1); note_launch(c);
                          gm_norm_final_kernel<<<1, kRedThreads, 0, c->stream>>>(sc, ws->partials); note_launch(c);
                          gm_next_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ldv, sc, w, V); note_launch(c);
                          gm_givens_kernel<<<1, 32, 0, c->stream>>>(sc, h, use); note_launch(c);
                          F.check(cudaGetLastError());
                      });
               gm_solve_kernel<<<1, 32, 0, c->stream>>>(sc); note_launch(c);
               if (use_prec) {   // x += P^{-1} (V y)
                   gm_combine_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ldv, sc, V, tbuf); note_launch(c);
                   F.check(prec(tbuf, zbuf, nullptr, 0));
                   axpy_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, x, zbuf); note_launch(c);
               } else {
                   gm_update_x_kernel<R><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ldv, sc, V, x); note_launch(c);
               }
               gm_cycle_end_kernel<<<1, 32, 0, c->stream>>>(sc, h_outer, use_outer); note_launch(c);
               F.check(cudaGetLastError());
           });
}

// ---- one shot, one slab ----------------------------------------------------------------
static void record_solve(Flow& F, double dt, double* b, double* x) {
    stdg_ctx* c = F.c;
    Workspace* ws = F.ws;
    const int64_t n = ws->n;                 // stacked length: n_shots x velocity values
    const int ns = c->n_shots;
    const int bm = ns > 1 ? 1 : 0;            // stacked solves stop on min-shot norms
    const bool cn = c->opt.scheme == STDG_SCHEME_CN;
    const bool pre = c->opt.preconditioner != 0;
    const int64_t ldv = ws->ldv;
    auto A64 = [&](const double* xx, double* yy) { return launch_apply(c, dt, xx, yy, 1.0, nullptr, 0, ns); };
    auto A64i = [&](const double* V, const int* idx, double* yy) { return launch_apply(c, dt, V, yy, 1.0, idx, ldv, ns); };
    auto A32 = [&](const float* xx, float* yy) { return launch_apply32(c, dt, xx, yy, 1.0, nullptr, 0, ns); };
    auto A32i = [&](const float* V, const int* idx, float* yy) { return launch_apply32(c, dt, V, yy, 1.0, idx, ldv, ns); };
    auto P64 = [&](const double* r, double* z, const int* idx, int64_t ld) { return launch_pre1_apply(c, r, z, idx, ld, ns); };
    auto P32 = [&](const float* r, float* z, const int* idx, int64_t ld) { return launch_pre1_apply32(c, r, z, idx, ld, ns); };
    auto P64c = [&](const double* r, double* z) { return launch_pre1_apply(c, r, z, nullptr, 0, ns); };
    auto P32c = [&](const float* r, float* z) { return launch_pre1_apply32(c, r, z, nullptr, 0, ns); };
    const double tol = c->opt.rel_tol;
    const int maxit = c->opt.max_iters;
    if (bm) {   // min over shots of ||b_s||
        const int G = (int)std::min<int64_t>(kRedBlocks, (int64_t)(kMaxRestart + 2) * kRedBlocks / ns);
        shot_norm_partial_kernel<<<dim3(G, ns), kRedThreads, 0, c->stream>>>(c->nvel, b, ws->partials); note_launch(c);
        shot_min_kernel<<<1, kRedThreads, 0, c->stream>>>(ws->sc, ws->partials, G, ns); note_launch(c);
    }
    if (c->opt.precision == STDG_FP64) {
        if (cn) solve_cg<double>(F, A64, P64c, pre, b, x, ws->r, ws->p, ws->q, ws->z, tol, maxit, -1.0, 0, bm);
        else solve_gmres<double>(F, A64, A64i, P64, pre, b, x, ws->V, ws->w, ws->z, ws->t, tol, maxit, -1.0, 0, bm);
        zero_if_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, x, &ws->sc->zero_x); note_launch(c);
        solve_stats_kernel<<<1, 32, 0, c->stream>>>(ws->sc, cn ? 1 : 0, bm); note_launch(c);
        return;
    }
    // mixed: FP64 refinement, FP32 inner solve with zero initial guess and unit RHS
    F.loop(&ws->sc->ir_flag,
           [&](cudaGraphConditionalHandle h, int use) {
               dot_partial_kernel<double, double><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, b, b, ws->partials); note_launch(c);
               ir_init_kernel<<<1, kRedThreads, 0, c->stream>>>(ws->sc, ws->partials, tol, 64, h, use, bm); note_launch(c);
           },
           [&](cudaGraphConditionalHandle h, int use) {
               F.check(A64(x, ws->w));
               gm_res_kernel<double><<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, b, ws->w, ws->r, ws->partials); note_launch(c);
               ir_check_kernel<<<1, kRedThreads, 0, c->stream>>>(ws->sc, ws->partials, maxit); note_launch(c);
               ir_convert_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ws->sc, ws->r, ws->b32, ws->x32); note_launch(c);
               if (cn)
                   solve_cg<float>(F, A32, P32c, pre, ws->b32, ws->x32, ws->r32, ws->p32, ws->q32, ws->z32, c->opt.inner_tol,
                                   maxit, 1.0, 1, 0);
               else
                   solve_gmres<float>(F, A32, A32i, P32, pre, ws->b32, ws->x32, ws->V32, ws->w32, ws->z32, ws->t32,
                                      c->opt.inner_tol, maxit, 1.0, 1, 0);
               ir_update_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, ws->sc, ws->x32, x); note_launch(c);
               ir_end_kernel<<<1, 32, 0, c->stream>>>(ws->sc, h, use); note_launch(c);
               F.check(cudaGetLastError());
           });
    zero_if_kernel<<<kRedBlocks, kRedThreads, 0, c->stream>>>(n, x, &ws->sc->zero_x); note_launch(c);
    solve_stats_kernel<<<1, 32, 0, c->stream>>>(ws->sc, 2, bm); note_launch(c);
}

// One slab for every shot: per-shot right-hand sides and initial guesses, ONE stacked
// (block-diagonal) solve whose operator and preconditioner kernels load each face's and
// element's blocks once for all shots, then per-shot stress, traces and receivers.
static void record_step(Flow& F, double dt) {
    stdg_ctx* c = F.c;
    Workspace* ws = F.ws;
    c->scopes.assign(1, 0);
    step_begin_kernel<<<1, 32, 0, c->stream>>>(ws->dparams, dt); note_launch(c);
    for (int shot = 0; shot < c->n_shots && F.err == cudaSuccess; ++shot) {
        F.check(launch_rhs(c, dt, ws->dparams, shot, c->d_b + (int64_t)shot * c->nvel));
        F.check(launch_initial_guess(c, shot, c->d_x + (int64_t)shot * c->nvel));
    }
    record_solve(F, dt, c->d_b, c->d_x);
    for (int shot = 0; shot < c->n_shots && F.err == cudaSuccess; ++shot) {
        F.check(launch_stress_update(c, dt, shot, c->d_x + (int64_t)shot * c->nvel));
        F.check(launch_traces(c, shot, c->d_x + (int64_t)shot * c->nvel));
        F.check(launch_receivers(c, ws->dparams, shot));
    }
    step_end_kernel<<<1, 32, 0, c->stream>>>(ws->dparams, dt); note_launch(c);
    const long k = c->scopes.back() + 1;
    c->scopes.clear();
    count_kernel<<<1, 32, 0, c->stream>>>(ws->sc, k);
    F.check(cudaGetLastError());
}

int solver_setup(stdg_ctx* c) {
    solver_free(c);
    Workspace* ws = new Workspace();
    c->ws = ws;
    ws->m = std::max(2, std::min(c->opt.gmres_restart > 0 ? c->opt.gmres_restart : 30, kMaxRestart));
    ws->n = c->nvel * (int64_t)c->n_shots;
    const int64_t n = ws->n;
    const bool cn = c->opt.scheme == STDG_SCHEME_CN;
    const bool mixed = c->opt.precision != STDG_FP64;
    const bool pre = c->opt.preconditioner != 0;
    int rc;
#define ALLOC(ptr, bytes) do { if ((rc = dev_alloc(c, (void**)&(ptr), (bytes))) != STDG_OK) return rc; \
                               ws->owned.push_back((void*)(ptr)); } while (0)
    ALLOC(ws->sc, sizeof(DevScalars));
    ALLOC(ws->partials, sizeof(double) * (kMaxRestart + 2) * kRedBlocks);
    ALLOC(ws->dparams, sizeof(double) * 4);
    ALLOC(c->d_b, sizeof(double) * n);
    ALLOC(c->d_x, sizeof(double) * n);
    ALLOC(ws->w, sizeof(double) * n);
    ALLOC(ws->r, sizeof(double) * n);
    ws->ldv = (n + 63) / 64 * 64;   // 16-byte aligned basis columns for vector loads
    if (cn && !mixed) { ALLOC(ws->p, sizeof(double) * n); ALLOC(ws->q, sizeof(double) * n); }
    if (!cn && !mixed) ALLOC(ws->V, sizeof(double) * ws->ldv * (ws->m + 1));
    if (pre && !mixed) { ALLOC(ws->z, sizeof(double) * n); if (!cn) ALLOC(ws->t, sizeof(double) * n); }
    if (mixed) {
        ALLOC(ws->b32, sizeof(float) * n);
        ALLOC(ws->x32, sizeof(float) * n);
        if (cn) { ALLOC(ws->r32, sizeof(float) * n); ALLOC(ws->p32, sizeof(float) * n); ALLOC(ws->q32, sizeof(float) * n); }
        else { ALLOC(ws->V32, sizeof(float) * ws->ldv * (ws->m + 1)); ALLOC(ws->w32, sizeof(float) * n); }
        if (pre) { ALLOC(ws->z32, sizeof(float) * n); if (!cn) ALLOC(ws->t32, sizeof(float) * n); }
    }
#undef ALLOC
    cudaMemsetAsync(ws->sc, 0, sizeof(DevScalars), c->stream);
    cudaMemsetAsync(ws->dparams, 0, sizeof(double) * 4, c->stream);
    for (auto& s : ws->side) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    return STDG_OK;
}

void solver_free(stdg_ctx* c) {
    Workspace* ws = W(c);
    if (!ws) return;
    if (ws->exec) cudaGraphExecDestroy(ws->exec);
    if (ws->graph) cudaGraphDestroy(ws->graph);
    for (auto& s : ws->side) if (s) cudaStreamDestroy(s);
    cudaStreamSynchronize(c->stream);
    for (void* p : ws->owned) dev_release(c, p);
    c->d_b = c->d_x = nullptr;
    delete ws;
    c->ws = nullptr;
}

void solver_invalidate_graph(stdg_ctx* c) {
    Workspace* ws = W(c);
    if (!ws) return;
    if (ws->exec) cudaGraphExecDestroy(ws->exec);
    if (ws->graph) cudaGraphDestroy(ws->graph);
    ws->exec = nullptr;
    ws->graph = nullptr;
    ws->graph_dt = -1.0;
}

double* solver_dparams(stdg_ctx* c) { return W(c) ? W(c)->dparams : nullptr; }

int solver_step(stdg_ctx* c, double dt, int n_steps, stdg_stats* st) {
    Workspace* ws = W(c);
    if (!ws) STDG_FAIL(c, STDG_ESTATE, "solver not set up");
    // statistics reset (outside any graph)
    STDG_CUDA(c, cudaMemsetAsync(&ws->sc->st_total, 0, sizeof(int) * 4, c->stream));
    STDG_CUDA(c, cudaMemsetAsync(&ws->sc->st_final_rel, 0, sizeof(double) * 2, c->stream));
    STDG_CUDA(c, cudaMemsetAsync(&ws->sc->launches, 0, sizeof(unsigned long long), c->stream));
    if (c->opt.preconditioner && c->pre_dt != dt) {
        STDG_CUDA(c, launch_pre1_time(c, dt));
        c->pre_dt = dt;
    }
    const double t0 = c->t;
    STDG_CUDA(c, cudaMemcpyAsync(ws->dparams, &t0, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    {
        double stepidx = (double)c->rec_steps;
        STDG_CUDA(c, cudaMemcpyAsync(ws->dparams + 2, &stepidx, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
    if (c->opt.use_graph) {
        if (!ws->exec || ws->graph_dt != dt) {
            solver_invalidate_graph(c);
            cudaStream_t s0 = c->stream;
            STDG_CUDA(c, cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed));
            Flow F{c, ws, true};
            record_step(F, dt);
            c->stream = s0;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(s0, &g);
            if (F.err != cudaSuccess || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                c->err = std::string("graph capture failed: ") + cudaGetErrorString(F.err != cudaSuccess ? F.err : e);
                cudaGetLastError();
                return STDG_ECUDA;
            }
            ws->graph = g;
            STDG_CUDA(c, cudaGraphInstantiate(&ws->exec, g, 0));
            ws->graph_dt = dt;
        }
        for (int s = 0; s < n_steps; ++s) STDG_CUDA(c, cudaGraphLaunch(ws->exec, c->stream));
    } else {
        for (int s = 0; s < n_steps; ++s) {
            Flow F{c, ws, false};
            record_step(F, dt);
            if (F.err != cudaSuccess) STDG_CUDA(c, F.err);
        }
    }
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    STDG_CUDA(c, cudaGetLastError());
    c->t = t0 + n_steps * dt;
    c->rec_steps += n_steps;
    DevScalars h;
    STDG_CUDA(c, cudaMemcpy(&h, ws->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    if (st) {
        st->iters_total = (int)h.st_iters_sum;
        st->iters_max = h.st_max;
        st->refinements = h.st_refine;
        st->final_rel_res = h.st_final_rel;
        st->status = h.st_notconv ? STDG_ENOTCONV : STDG_OK;
    }
    c->last_launches = (int64_t)h.launches;
    if (c->d_err) {
        int e = 0;
        STDG_CUDA(c, cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) STDG_FAIL(c, STDG_ECUDA, "a device-side wait gave up (bounded mbarrier wait)");
    }
    if (h.st_notconv) STDG_FAIL(c, STDG_ENOTCONV, "Krylov solve reached max_iters");
    return STDG_OK;
}

}  // namespace stdg
