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
// Several shots (right-hand sides on one mesh) are solved together: their vectors are
// stacked shot-major, the operator and preconditioner kernels load each face's and
// element's blocks once for all shots, and every Krylov scalar is kept PER SHOT, so each
// shot runs its own CG / GMRES recurrence (the same iterates as a solve of that shot
// alone) and stops at ||r_s|| <= rel_tol ||b_s||.  A shot that has converged is frozen
// (zero step length) while the others continue; the loops end when every shot has.
//
// Solvers
//   CG        (Crank-Nicolson)  r = b - A x; standard recurrences; FP64 dots.
//   GMRES(m)  (space-time DG)   restarted, classical Gram-Schmidt with a second
//                               pass only where the first one cancelled more than 99%
//                               of ||w||^2, Givens rotations on the device,
//                               true residual checked at every restart.
//   Mixed     FP64 iterative refinement around an FP32 CG / GMRES: r = b - A64 x in FP64,
//             solve A32 d = r/|r| to inner_tol, x += |r| d, stop at rel_tol in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "stdg_internal.h"

namespace stdg {

constexpr int kMaxRestart = 64;
constexpr int kRedThreads = 256;
constexpr int kFinThreads = 1024;   // single-block reduction / control kernels
constexpr int kDotChunk = 16;       // basis vectors per pass of the multi-dot kernels

// Krylov state of one shot
struct ShotScalars {
    double bnorm, tol_abs;
    double rr, pq, alpha, beta;                   // CG
    double gbeta, resid;                          // GMRES
    double hcol[kMaxRestart + 2], hpass[kMaxRestart + 2];
    double H[(kMaxRestart + 1) * kMaxRestart];
    double cs[kMaxRestart], sn[kMaxRestart], g[kMaxRestart + 1], y[kMaxRestart];
    double red[3];                                // reduced sums handed between warps
    int jj;            // basis columns this shot uses in the current cycle
    int active;        // still iterating in the current cycle / CG solve
    int reorth;        // this Arnoldi step needs the second Gram-Schmidt pass
    int converged, zero_x;                        // zero_x: b_s = 0, so x_s = 0
    // FP64 refinement level (mixed precision)
    double ir_bnorm, ir_tol_abs, ir_rnorm, ir_scale;
    int ir_conv, ir_zero;
};

// loop control shared by all shots
struct DevScalars {
    int j, iters, flag_outer, flag_inner, max_iters, m;
    int ir_flag, ir_count, ir_max;
    // statistics, reset by the host before a batch of steps
    int st_total, st_max, st_refine, st_notconv, st_nonfinite;
    double st_final_rel, st_iters_sum;
    unsigned long long launches;      // kernel executions since the last reset
};

struct Workspace {
    int m = 30;
    int ns = 1;                   // shots
    int64_t nvec = 0;             // values per shot (velocity DOFs)
    int64_t n = 0, ldv = 0;       // stacked length, basis leading dimension
    unsigned G = 1;               // blocks per shot of the streaming kernels (grid G x ns)
    unsigned red_blocks = 1;      // blocks of the single-vector streaming kernels: 8 per SM
    DevScalars* sc = nullptr;
    ShotScalars* ss = nullptr;    // [ns]
    double* partials = nullptr;   // [slot][shot][block], (kMaxRestart + 2) slots
    double* dparams = nullptr;    // t^n, dt, step index
    double *V = nullptr, *w = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *t = nullptr;   // FP64
    float *V32 = nullptr, *w32 = nullptr, *b32 = nullptr, *x32 = nullptr, *r32 = nullptr, *p32 = nullptr, *q32 = nullptr;
    float *z32 = nullptr, *t32 = nullptr;
    cudaStream_t side[6] = {};
    int depth = 0;
    // cached graphs: [0] one whole step, [1] the solve alone (adjoint)
    cudaGraph_t graph[2] = {};
    cudaGraphExec_t exec[2] = {};
    double graph_dt[2] = {-1.0, -1.0};
    std::vector<void*> owned;   // device buffers of this workspace
    dim3 grid() const { return dim3(G, (unsigned)ns); }
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

// sum of p[0..n) by one warp; valid in every lane
__device__ __forceinline__ double warp_sum(const double* p, int n) {
    double v = 0;
    for (int i = threadIdx.x & 31; i < n; i += 32) v += p[i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// partial sums of slot k, shot s: part + (k * ns + s) * G
__device__ __forceinline__ const double* slot(const double* part, int k, int s, int ns, int G) {
    return part + ((int64_t)k * ns + s) * G;
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

// 16-byte vector access: VW = 4 floats or 2 doubles per load/store.  Every pointer that is
// vectorised is 16-byte aligned (separate allocations, or basis columns at a leading
// dimension that is a multiple of 64 elements).
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

// Streaming over one shot's segment [s*nvec, (s+1)*nvec), s = blockIdx.y, by the
// gridDim.x blocks of that shot: fv(i) handles the VW values from i (i a multiple of VW),
// fs(i) one value of the unaligned head or tail (thread 0 of the shot's first block).
template <typename R, class FV, class FS>
__device__ __forceinline__ void seg_loop(int64_t nvec, FV&& fv, FS&& fs) {
    constexpr int VW = VL<R>::W;
    const int64_t lo = (int64_t)blockIdx.y * nvec, hi = lo + nvec;
    const int64_t a0 = min(hi, (lo + VW - 1) / VW * VW);
    const int64_t a1 = max(a0, hi / VW * VW);
    for (int64_t g = a0 / VW + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a1 / VW;
         g += (int64_t)gridDim.x * blockDim.x)
        fv(g * VW);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int64_t i = lo; i < a0; ++i) fs(i);
        for (int64_t i = a1; i < hi; ++i) fs(i);
    }
}

// block's partial sum into slot k of its shot
__device__ __forceinline__ void put_partial(double* part, int k, double v) {
    const double s = block_sum(v);
    if (threadIdx.x == 0) part[((int64_t)k * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = s;
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int use, int v) {
    if (use) cudaGraphSetConditional(h, v ? 1u : 0u);
}

// per-shot dot products a_s . b_s into slot k
template <typename A, typename B>
__global__ void dot_partial_kernel(int64_t nvec, const A* __restrict__ a, const B* __restrict__ b, double* __restrict__ part,
                                   int k) {
    Acc<A> acc;
    const int64_t lo = (int64_t)blockIdx.y * nvec;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x)
        acc.add(a[lo + i], b[lo + i]);
    put_partial(part, k, acc.value());
}

// x_s = 0 for the shots whose right-hand side is zero (level 0: Krylov, 1: refinement)
__global__ void zero_if_kernel(int64_t nvec, double* x, const ShotScalars* ss, int level) {
    if (!(level ? ss[blockIdx.y].ir_zero : ss[blockIdx.y].zero_x)) return;
    const int64_t lo = (int64_t)blockIdx.y * nvec;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x)
        x[lo + i] = 0;
}

// ---------------------------------------------------------------------------------
// (Preconditioned) CG kernels (R = vector type, scalars FP64, one recurrence per shot).
// Without a preconditioner z aliases r and rz = rr.
// ---------------------------------------------------------------------------------
template <typename R>
__global__ void cg_res_kernel(int64_t nvec, const R* __restrict__ b, const R* __restrict__ Ax, R* __restrict__ r,
                              double* __restrict__ part) {
    double rr = 0, bb = 0;
    const int64_t lo = (int64_t)blockIdx.y * nvec;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x) {
        const R ri = b[lo + i] - Ax[lo + i];
        r[lo + i] = ri;
        rr += (double)ri * (double)ri;
        bb += (double)b[lo + i] * (double)b[lo + i];
    }
    put_partial(part, 0, rr);
    put_partial(part, 1, bb);
}

// bnorm_given < 0: use ||b_s|| from the partials; slots: 0 rr, 1 bb, 2 rz
__global__ void __launch_bounds__(kFinThreads) cg_init_final_kernel(DevScalars* sc, ShotScalars* ss, const double* part,
                                                                    int ns, int G, double rel_tol, int max_iters,
                                                                    double bnorm_given, int gate_ir,
                                                                    cudaGraphConditionalHandle h, int use_h) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < 3 * ns; q += nw) {
        const double v = warp_sum(slot(part, q % 3, q / 3, ns, G), G);
        if ((threadIdx.x & 31) == 0) ss[q / 3].red[q % 3] = v;
    }
    __syncthreads();
    const int active = gate_ir ? sc->ir_flag : 1;
    int any = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        ShotScalars& t = ss[s];
        t.rr = t.red[0];
        t.pq = t.red[2];                   // holds r.z between iterations
        t.bnorm = bnorm_given >= 0 ? bnorm_given : sqrt(t.red[1]);
        t.tol_abs = rel_tol * t.bnorm;
        t.zero_x = active && t.bnorm == 0.0;
        t.converged = !active || sqrt(t.rr) <= t.tol_abs;
        t.active = !t.converged && isfinite(t.rr) && isfinite(t.bnorm);   // a NaN/Inf residual stops the shot
        t.alpha = t.beta = 0.0;
        any |= t.active;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        sc->iters = 0;
        sc->max_iters = max_iters;
        sc->flag_inner = any && max_iters > 0;
        set_cond(h, use_h, sc->flag_inner);
    }
}

template <typename R>
__global__ void copy_kernel(int64_t n, const R* __restrict__ a, R* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = a[i];
}

// alpha_s = (r.z)_s / (p.q)_s for the shots still iterating, 0 for the frozen ones
__global__ void __launch_bounds__(kFinThreads) cg_alpha_kernel(ShotScalars* ss, const double* part, int ns, int G) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = warp; s < ns; s += nw) {
        const double pq = warp_sum(slot(part, 0, s, ns, G), G);
        if ((threadIdx.x & 31) == 0) ss[s].alpha = ss[s].active && pq != 0.0 ? ss[s].pq / pq : 0.0;
    }
}

template <typename R>
__global__ void cg_update_kernel(int64_t nvec, const ShotScalars* __restrict__ ss, R* __restrict__ x, R* __restrict__ r,
                                 const R* __restrict__ p, const R* __restrict__ q, double* __restrict__ part) {
    const double a = ss[blockIdx.y].alpha;
    const int64_t lo = (int64_t)blockIdx.y * nvec;
    double rr = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x) {
        x[lo + i] = (R)((double)x[lo + i] + a * (double)p[lo + i]);
        const R ri = (R)((double)r[lo + i] - a * (double)q[lo + i]);
        r[lo + i] = ri;
        rr += (double)ri * (double)ri;
    }
    put_partial(part, 0, rr);
}

// slots: 0 rr, 2 rz (r.z after the preconditioner)
__global__ void __launch_bounds__(kFinThreads) cg_beta_kernel(DevScalars* sc, ShotScalars* ss, const double* part, int ns,
                                                              int G, cudaGraphConditionalHandle h, int use_h) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < 2 * ns; q += nw) {
        const int k = q % 2 == 0 ? 0 : 2;
        const double v = warp_sum(slot(part, k, q / 2, ns, G), G);
        if ((threadIdx.x & 31) == 0) ss[q / 2].red[k] = v;
    }
    __syncthreads();
    int any = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        ShotScalars& t = ss[s];
        if (t.active) {
            const double rz = t.red[2];
            t.beta = t.pq != 0.0 ? rz / t.pq : 0.0;
            t.pq = rz;
            t.rr = t.red[0];
            t.converged = sqrt(t.rr) <= t.tol_abs;
            t.active = !t.converged && isfinite(t.rr);
        }
        if (!t.active) t.beta = 0.0;
        any |= t.active;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        sc->iters += 1;
        sc->flag_inner = any && sc->iters < sc->max_iters;
        set_cond(h, use_h, sc->flag_inner);
    }
}

template <typename R>
__global__ void cg_p_kernel(int64_t nvec, const ShotScalars* __restrict__ ss, const R* __restrict__ z, R* __restrict__ p) {
    const double b = ss[blockIdx.y].beta;
    const int64_t lo = (int64_t)blockIdx.y * nvec;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x)
        p[lo + i] = (R)((double)z[lo + i] + b * (double)p[lo + i]);
}

// ---------------------------------------------------------------------------------
// GMRES kernels (one Arnoldi process and one Hessenberg matrix per shot)
// ---------------------------------------------------------------------------------
template <typename R>
__global__ void gm_res_kernel(int64_t nvec, const R* __restrict__ b, const R* __restrict__ Ax, R* __restrict__ v0,
                             double* __restrict__ part) {
    constexpr int VW = VL<R>::W;
    Acc<R> rr;
    seg_loop<R>(nvec,
        [&](int64_t i) {
            R bb[VW], aa[VW];
            VL<R>::ld(b + i, bb);
            VL<R>::ld(Ax + i, aa);
#pragma unroll
            for (int u = 0; u < VW; ++u) { bb[u] -= aa[u]; rr.add(bb[u], bb[u]); }
            VL<R>::st(v0 + i, bb);
        },
        [&](int64_t i) { const R ri = b[i] - Ax[i]; v0[i] = ri; rr.add(ri, ri); });
    put_partial(part, 0, rr.value());
}

// set up one GMRES solve: ||b_s|| (from slot 0, or given), tolerances, counters
__global__ void __launch_bounds__(kFinThreads) gm_init_kernel(DevScalars* sc, ShotScalars* ss, const double* part, int ns,
                                                              int G, double rel_tol, int max_iters, int m,
                                                              double bnorm_given, int gate_ir,
                                                              cudaGraphConditionalHandle h, int use_h) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (bnorm_given < 0)
        for (int s = warp; s < ns; s += nw) {
            const double v = warp_sum(slot(part, 0, s, ns, G), G);
            if ((threadIdx.x & 31) == 0) ss[s].red[0] = v;
        }
    __syncthreads();
    const int active = gate_ir ? sc->ir_flag : 1;
    int any = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        ShotScalars& t = ss[s];
        t.bnorm = bnorm_given >= 0 ? bnorm_given : sqrt(t.red[0]);
        t.tol_abs = rel_tol * t.bnorm;
        t.zero_x = active && t.bnorm == 0.0;
        t.converged = !active || t.zero_x;
        t.active = 0;
        t.jj = 0;
        any |= !t.converged;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        sc->iters = 0;
        sc->max_iters = max_iters;
        sc->m = m;
        sc->j = 0;
        sc->flag_outer = any;
        set_cond(h, use_h, sc->flag_outer);
    }
}

// restart: beta_s = ||r_s|| (the true residual), convergence test, g = beta_s e_1
__global__ void __launch_bounds__(kFinThreads) gm_cycle_start_kernel(DevScalars* sc, ShotScalars* ss, const double* part,
                                                                     int ns, int G, cudaGraphConditionalHandle h,
                                                                     int use_h) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = warp; s < ns; s += nw) {
        const double v = warp_sum(slot(part, 0, s, ns, G), G);
        if ((threadIdx.x & 31) == 0) ss[s].red[0] = v;
    }
    __syncthreads();
    const int m = sc->m;
    int any = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        ShotScalars& t = ss[s];
        const double beta = sqrt(t.red[0]);
        t.gbeta = beta;
        t.resid = beta;
        t.jj = 0;
        if (!t.converged) t.converged = beta <= t.tol_abs;
        t.active = !t.converged && isfinite(beta) && isfinite(t.tol_abs);   // a NaN/Inf residual stops the shot
        for (int k = 0; k <= m; ++k) t.g[k] = 0.0;
        t.g[0] = beta;
        any |= t.active;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        sc->j = 0;
        sc->flag_inner = any && sc->iters < sc->max_iters;
        set_cond(h, use_h, sc->flag_inner);
    }
}

template <typename R>
__global__ void gm_scale0_kernel(int64_t nvec, const DevScalars* __restrict__ sc, const ShotScalars* __restrict__ ss,
                                 R* __restrict__ v0) {
    if (!sc->flag_inner) return;
    constexpr int VW = VL<R>::W;
    const double gb = ss[blockIdx.y].gbeta;
    const R s = (R)(gb > 0.0 ? 1.0 / gb : 0.0);
    seg_loop<R>(nvec,
        [&](int64_t i) {
            R a[VW];
            VL<R>::ld(v0 + i, a);
#pragma unroll
            for (int u = 0; u < VW; ++u) a[u] *= s;
            VL<R>::st(v0 + i, a);
        },
        [&](int64_t i) { v0[i] *= s; });
}

// slot k, shot s: sum_i V_k[i] w[i] over the shot's segment, k = 0..j (basis columns at stride ldv)
template <typename R>
__global__ void __launch_bounds__(256, 4) gm_mdot_kernel(int64_t nvec, int64_t ldv, const DevScalars* __restrict__ sc,
                                                      const R* __restrict__ V, const R* __restrict__ w,
                                                      double* __restrict__ part) {
    constexpr int VW = VL<R>::W;
    const int J = sc->j;
    for (int k0 = 0; k0 <= J; k0 += kDotChunk) {
        Acc<R> acc[kDotChunk];
        Acc<R> ww;                                // ||w||^2, first chunk only
        const int kn = min(kDotChunk, J + 1 - k0);
        seg_loop<R>(nvec,
            [&](int64_t i) {
                R wv[VW];
                VL<R>::ld(w + i, wv);
                if (k0 == 0) {
#pragma unroll
                    for (int u = 0; u < VW; ++u) ww.add(wv[u], wv[u]);
                }
#pragma unroll
                for (int kk = 0; kk < kDotChunk; ++kk)
                    if (kk < kn) {
                        R vv[VW];
                        VL<R>::ld(V + (int64_t)(k0 + kk) * ldv + i, vv);
#pragma unroll
                        for (int u = 0; u < VW; ++u) acc[kk].add(vv[u], wv[u]);
                    }
            },
            [&](int64_t i) {
                if (k0 == 0) ww.add(w[i], w[i]);
#pragma unroll
                for (int kk = 0; kk < kDotChunk; ++kk)
                    if (kk < kn) acc[kk].add(V[(int64_t)(k0 + kk) * ldv + i], w[i]);
            });
#pragma unroll
        for (int kk = 0; kk < kDotChunk; ++kk)   // constant bound keeps acc[] in registers
            if (kk < kn) put_partial(part, k0 + kk, acc[kk].value());   // kn is uniform over the block
        if (k0 == 0) put_partial(part, J + 1, ww.value());
    }
}

// Second Gram-Schmidt pass fused with the first subtraction:
// w_s <- w_s - sum_k h1_s[k] V_k, then partials of V_k . w_s for the re-orthogonalisation.
template <typename R>
__global__ void __launch_bounds__(256, 3) gm_orth_fused_kernel(int64_t nvec, int64_t ldv, const DevScalars* __restrict__ sc,
                                                            const ShotScalars* __restrict__ ss, const R* __restrict__ V,
                                                            R* __restrict__ w, double* __restrict__ part) {
    constexpr int VW = VL<R>::W;
    const int J = sc->j;
    if (!ss[blockIdx.y].reorth) return;           // this shot's first pass was enough
    __shared__ R h[kMaxRestart + 2];
    for (int k = threadIdx.x; k <= J; k += blockDim.x) h[k] = (R)ss[blockIdx.y].hpass[k];
    __syncthreads();
    for (int k0 = 0; k0 <= J; k0 += kDotChunk) {
        Acc<R> acc[kDotChunk];
        const int kn = min(kDotChunk, J + 1 - k0);
        seg_loop<R>(nvec,
            [&](int64_t i) {
                R wv[VW];
                VL<R>::ld(w + i, wv);
                if (k0 == 0) {   // first chunk: form and store the projected w (in the vector precision)
                    for (int k = 0; k <= J; ++k) {
                        R vv[VW];
                        VL<R>::ld(V + (int64_t)k * ldv + i, vv);
#pragma unroll
                        for (int u = 0; u < VW; ++u) wv[u] = fma(-h[k], vv[u], wv[u]);
                    }
                    VL<R>::st(w + i, wv);
                }
#pragma unroll
                for (int kk = 0; kk < kDotChunk; ++kk)
                    if (kk < kn) {
                        R vv[VW];
                        VL<R>::ld(V + (int64_t)(k0 + kk) * ldv + i, vv);
#pragma unroll
                        for (int u = 0; u < VW; ++u) acc[kk].add(vv[u], wv[u]);
                    }
            },
            [&](int64_t i) {
                R wi = w[i];
                if (k0 == 0) {
                    for (int k = 0; k <= J; ++k) wi = fma(-h[k], V[(int64_t)k * ldv + i], wi);
                    w[i] = wi;
                }
#pragma unroll
                for (int kk = 0; kk < kDotChunk; ++kk)
                    if (kk < kn) acc[kk].add(V[(int64_t)(k0 + kk) * ldv + i], wi);
            });
#pragma unroll
        for (int kk = 0; kk < kDotChunk; ++kk)
            if (kk < kn) put_partial(part, k0 + kk, acc[kk].value());
    }
}

// hpass_s[k] = reduced slot k (k = 0..j); pass 0 starts the Hessenberg column, pass 1 adds
// Pass 0 also decides, per shot, whether the second pass is needed: one classical
// Gram-Schmidt pass leaves w orthogonal to the basis to about eps ||w|| / ||w - V h||, so the
// pass is repeated when that ratio would exceed 10, i.e. when
// ||w - V h||^2 = ||w||^2 - |h|^2 < 1e-2 ||w||^2 (V orthonormal; the dots are FP64-accurate).
__global__ void __launch_bounds__(kFinThreads) gm_mdot_final_kernel(const DevScalars* sc, ShotScalars* ss,
                                                                    const double* part, int ns, int G, int pass) {
    const int J = sc->j;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nk = pass == 0 ? J + 2 : J + 1;    // pass 0: slot J+1 holds ||w||^2
    for (int q = warp; q < nk * ns; q += nw) {
        const int k = q / ns, s = q % ns;
        if (pass == 1 && !ss[s].reorth) continue;
        const double v = warp_sum(slot(part, k, s, ns, G), G);
        if ((threadIdx.x & 31) == 0) {
            if (k <= J) {
                ss[s].hpass[k] = v;
                ss[s].hcol[k] = pass == 0 ? v : ss[s].hcol[k] + v;
            } else {
                ss[s].red[0] = v;
            }
        }
    }
    if (pass != 0) return;
    __syncthreads();
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        ShotScalars& t = ss[s];
        double h2 = 0.0;
        for (int k = 0; k <= J; ++k) h2 += t.hcol[k] * t.hcol[k];
        t.reorth = t.red[0] - h2 < 1e-2 * t.red[0];
    }
}

// w_s -= sum_k hpass_s[k] V_k; partial ||w_s||^2 into slot 0
template <typename R>
__global__ void __launch_bounds__(256) gm_maxpy_kernel(int64_t nvec, int64_t ldv, const DevScalars* __restrict__ sc,
                                                       const ShotScalars* __restrict__ ss, const R* __restrict__ V,
                                                       R* __restrict__ w, double* __restrict__ part) {
    constexpr int VW = VL<R>::W;
    const int J = sc->j;
    __shared__ R h[kMaxRestart + 2];
    for (int k = threadIdx.x; k <= J; k += blockDim.x) h[k] = (R)ss[blockIdx.y].hpass[k];
    __syncthreads();
    Acc<R> nn;
    seg_loop<R>(nvec,
        [&](int64_t i) {
            R wv[VW];
            VL<R>::ld(w + i, wv);
            for (int k = 0; k <= J; ++k) {
                R vv[VW];
                VL<R>::ld(V + (int64_t)k * ldv + i, vv);
#pragma unroll
                for (int u = 0; u < VW; ++u) wv[u] = fma(-h[k], vv[u], wv[u]);
            }
            VL<R>::st(w + i, wv);
#pragma unroll
            for (int u = 0; u < VW; ++u) nn.add(wv[u], wv[u]);
        },
        [&](int64_t i) {
            R wi = w[i];
            for (int k = 0; k <= J; ++k) wi = fma(-h[k], V[(int64_t)k * ldv + i], wi);
            w[i] = wi;
            nn.add(wi, wi);
        });
    put_partial(part, 0, nn.value());
}

__global__ void __launch_bounds__(kFinThreads) gm_norm_final_kernel(const DevScalars* sc, ShotScalars* ss, const double* part,
                                                                    int ns, int G) {
    const int J = sc->j;
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = warp; s < ns; s += nw) {
        const double v = warp_sum(slot(part, 0, s, ns, G), G);
        if ((threadIdx.x & 31) == 0) ss[s].hcol[J + 1] = sqrt(v);
    }
}

template <typename R>
__global__ void gm_next_kernel(int64_t nvec, int64_t ldv, const DevScalars* __restrict__ sc,
                               const ShotScalars* __restrict__ ss, const R* __restrict__ w, R* __restrict__ V) {
    constexpr int VW = VL<R>::W;
    const int J = sc->j;
    const double hh = ss[blockIdx.y].hcol[J + 1];
    const R s = (R)(hh > 0.0 ? 1.0 / hh : 0.0);
    R* vn = V + (int64_t)(J + 1) * ldv;
    seg_loop<R>(nvec,
        [&](int64_t i) {
            R a[VW];
            VL<R>::ld(w + i, a);
#pragma unroll
            for (int u = 0; u < VW; ++u) a[u] *= s;
            VL<R>::st(vn + i, a);
        },
        [&](int64_t i) { vn[i] = w[i] * s; });
}

// Givens update of every shot still iterating; a shot stops at its residual estimate or on
// breakdown, and keeps the columns it has (jj)
__global__ void __launch_bounds__(kFinThreads) gm_givens_kernel(DevScalars* sc, ShotScalars* ss, int ns,
                                                                cudaGraphConditionalHandle h, int use_h) {
    const int J = sc->j, m = sc->m;
    int any = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        ShotScalars& t = ss[s];
        if (t.active) {
            double* hc = t.hcol;
            for (int i = 0; i < J; ++i) {
                const double u = t.cs[i] * hc[i] + t.sn[i] * hc[i + 1];
                hc[i + 1] = -t.sn[i] * hc[i] + t.cs[i] * hc[i + 1];
                hc[i] = u;
            }
            const double a = hc[J], b = hc[J + 1];
            const double den = hypot(a, b);
            double cs = 1.0, sn = 0.0;
            if (den > 0.0) { cs = a / den; sn = b / den; }
            t.cs[J] = cs;
            t.sn[J] = sn;
            hc[J] = den;
            hc[J + 1] = 0.0;
            for (int i = 0; i <= J; ++i) t.H[i * kMaxRestart + J] = hc[i];
            t.g[J + 1] = -sn * t.g[J];
            t.g[J] = cs * t.g[J];
            t.resid = fabs(t.g[J + 1]);
            t.jj = J + 1;
            if (t.resid <= t.tol_abs || den == 0.0 || !isfinite(t.resid)) t.active = 0;
        }
        any |= t.active;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        sc->iters += 1;
        sc->j = J + 1;
        sc->flag_inner = any && sc->j < m && sc->iters < sc->max_iters;
        set_cond(h, use_h, sc->flag_inner);
    }
}

// y_s = R_s^{-1} g_s (upper triangular, size jj_s)
__global__ void gm_solve_kernel(ShotScalars* ss, int ns) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += gridDim.x * blockDim.x) {
        ShotScalars& t = ss[s];
        const int J = t.jj;
        for (int i = J - 1; i >= 0; --i) {
            double v = t.g[i];
            for (int k = i + 1; k < J; ++k) v -= t.H[i * kMaxRestart + k] * t.y[k];
            const double d = t.H[i * kMaxRestart + i];
            t.y[i] = d != 0.0 ? v / d : 0.0;
        }
    }
}

// x_s += sum_{k<jj_s} y_s[k] V_k  (accumulate = 1), or t_s = sum_k y_s[k] V_k (accumulate = 0;
// right preconditioning applies P^{-1} to t afterwards)
template <typename R>
__global__ void gm_combine_kernel(int64_t nvec, int64_t ldv, const ShotScalars* __restrict__ ss, const R* __restrict__ V,
                                  R* __restrict__ x, int accumulate) {
    constexpr int VW = VL<R>::W;
    const int J = ss[blockIdx.y].jj;
    if (accumulate && J == 0) return;
    __shared__ R y[kMaxRestart];
    for (int k = threadIdx.x; k < J; k += blockDim.x) y[k] = (R)ss[blockIdx.y].y[k];
    __syncthreads();
    seg_loop<R>(nvec,
        [&](int64_t i) {
            R a[VW];
            if (accumulate) VL<R>::ld(x + i, a);
            else {
#pragma unroll
                for (int u = 0; u < VW; ++u) a[u] = 0;
            }
            for (int k = 0; k < J; ++k) {
                R vv[VW];
                VL<R>::ld(V + (int64_t)k * ldv + i, vv);
#pragma unroll
                for (int u = 0; u < VW; ++u) a[u] = fma(y[k], vv[u], a[u]);
            }
            VL<R>::st(x + i, a);
        },
        [&](int64_t i) {
            R a = accumulate ? x[i] : (R)0;
            for (int k = 0; k < J; ++k) a = fma(y[k], V[(int64_t)k * ldv + i], a);
            x[i] = a;
        });
}

template <typename R>
__global__ void axpy_kernel(int64_t n, R* __restrict__ x, const R* __restrict__ z) {
    constexpr int VW = VL<R>::W;
    const int64_t nv = n / VW;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nv; g += (int64_t)gridDim.x * blockDim.x) {
        R a[VW], b[VW];
        VL<R>::ld(x + g * VW, a);
        VL<R>::ld(z + g * VW, b);
#pragma unroll
        for (int u = 0; u < VW; ++u) a[u] += b[u];
        VL<R>::st(x + g * VW, a);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (int64_t i = nv * VW; i < n; ++i) x[i] += z[i];
}

__global__ void __launch_bounds__(kFinThreads) gm_cycle_end_kernel(DevScalars* sc, const ShotScalars* ss, int ns,
                                                                   cudaGraphConditionalHandle h, int use_h) {
    int any = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) any |= !ss[s].converged;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        sc->j = 0;
        sc->flag_outer = any && sc->iters < sc->max_iters;
        set_cond(h, use_h, sc->flag_outer);
    }
}

// ---------------------------------------------------------------------------------
// FP64 iterative refinement around the FP32 solver (per shot)
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(kFinThreads) ir_init_kernel(DevScalars* sc, ShotScalars* ss, const double* part, int ns,
                                                              int G, double rel_tol, int ir_max,
                                                              cudaGraphConditionalHandle h, int use_h) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = warp; s < ns; s += nw) {
        const double v = warp_sum(slot(part, 0, s, ns, G), G);
        if ((threadIdx.x & 31) == 0) ss[s].red[0] = v;
    }
    __syncthreads();
    int any = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        ShotScalars& t = ss[s];
        t.ir_bnorm = sqrt(t.red[0]);
        t.ir_tol_abs = rel_tol * t.ir_bnorm;
        t.ir_rnorm = t.ir_bnorm;
        t.ir_zero = t.ir_bnorm == 0.0;
        t.ir_conv = t.ir_zero;
        any |= !t.ir_conv && isfinite(t.ir_bnorm);
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        sc->ir_count = 0;
        sc->ir_max = ir_max;
        sc->ir_flag = any;
        set_cond(h, use_h, sc->ir_flag);
    }
}

__global__ void __launch_bounds__(kFinThreads) ir_check_kernel(DevScalars* sc, ShotScalars* ss, const double* part, int ns,
                                                               int G, int max_total) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int s = warp; s < ns; s += nw) {
        const double v = warp_sum(slot(part, 0, s, ns, G), G);
        if ((threadIdx.x & 31) == 0) ss[s].red[0] = v;
    }
    __syncthreads();
    int any = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        ShotScalars& t = ss[s];
        t.ir_rnorm = sqrt(t.red[0]);
        t.ir_conv = t.ir_zero || t.ir_rnorm <= t.ir_tol_abs;
        t.ir_scale = !t.ir_conv && t.ir_rnorm > 0.0 ? 1.0 / t.ir_rnorm : 0.0;
        any |= !t.ir_conv && isfinite(t.ir_rnorm) && isfinite(t.ir_bnorm);   // no refinement of a NaN/Inf residual
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) sc->ir_flag = any && sc->ir_count < sc->ir_max && sc->st_total < max_total;
}

// r32_s = r64_s * scale_s (0 for converged shots); x32 = 0   (when the refinement continues)
__global__ void ir_convert_kernel(int64_t nvec, const DevScalars* __restrict__ sc, const ShotScalars* __restrict__ ss,
                                  const double* __restrict__ r64, float* __restrict__ r32, float* __restrict__ x32) {
    if (!sc->ir_flag) return;
    const double s = ss[blockIdx.y].ir_scale;
    const int64_t lo = (int64_t)blockIdx.y * nvec;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x) {
        r32[lo + i] = (float)(r64[lo + i] * s);
        x32[lo + i] = 0.0f;
    }
}

// x_s += |r_s| x32_s
__global__ void ir_update_kernel(int64_t nvec, const DevScalars* __restrict__ sc, const ShotScalars* __restrict__ ss,
                                 const float* __restrict__ x32, double* __restrict__ x) {
    if (!sc->ir_flag || ss[blockIdx.y].ir_conv) return;
    const double s = ss[blockIdx.y].ir_rnorm;
    const int64_t lo = (int64_t)blockIdx.y * nvec;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvec; i += (int64_t)gridDim.x * blockDim.x)
        x[lo + i] += s * (double)x32[lo + i];
}

__global__ void ir_end_kernel(DevScalars* sc, cudaGraphConditionalHandle h, int use_h) {
    if (threadIdx.x != 0) return;
    if (sc->ir_flag) {
        sc->ir_count += 1;
        sc->st_total += sc->iters;
    }
    set_cond(h, use_h, sc->ir_flag);
}

// per-solve statistics (worst shot); mode 0 = GMRES, 1 = CG, 2 = mixed (refinement level)
__global__ void __launch_bounds__(kFinThreads) solve_stats_kernel(DevScalars* sc, const ShotScalars* ss, int ns, int mode) {
    __shared__ double worst[kFinThreads];
    double rel = 0.0;
    int notconv = 0, nonfinite = 0;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const ShotScalars& t = ss[s];
        double r, bn;
        if (mode == 2) { r = t.ir_zero ? 0.0 : t.ir_rnorm; bn = t.ir_bnorm; notconv |= !t.ir_conv; }
        else { r = t.zero_x ? 0.0 : mode == 1 ? sqrt(t.rr) : t.resid; bn = t.bnorm; notconv |= !t.converged; }
        nonfinite |= !isfinite(r) || !isfinite(bn);
        rel = fmax(rel, bn > 0 ? r / bn : 0.0);
    }
    worst[threadIdx.x] = rel;
    notconv = __syncthreads_or(notconv);
    nonfinite = __syncthreads_or(nonfinite);
    if (threadIdx.x != 0) return;
    for (int i = 1; i < (int)blockDim.x; ++i) rel = fmax(rel, worst[i]);
    int it;
    if (mode == 2) {
        it = sc->st_total;          // accumulated by ir_end over the refinement sweeps
        sc->st_total = 0;
        sc->st_refine += sc->ir_count;
    } else {
        it = sc->iters;
    }
    if (notconv) sc->st_notconv = 1;
    if (nonfinite) sc->st_nonfinite = 1;
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


// ---- (P)CG on vectors of type R; apply(x, y): y = A x; prec(r, z): z = P^{-1} r or null --------
template <typename R, class Apply, class Prec>
static void solve_cg(Flow& F, Apply apply, Prec prec, bool use_prec, const R* b, R* x, R* r, R* p, R* q, R* z,
                     double rel_tol, int max_iters, double bnorm_given, int gate_ir) {
    stdg_ctx* c = F.c;
    Workspace* ws = F.ws;
    const int64_t n = ws->n, nv = ws->nvec;
    const int ns = ws->ns, G = (int)ws->G;
    const dim3 grid = ws->grid();
    R* zz = use_prec ? z : r;
    F.loop(&ws->sc->flag_inner,
           [&](cudaGraphConditionalHandle h, int use) {
               F.check(apply(x, q));
               cg_res_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, b, q, r, ws->partials); note_launch(c);
               if (use_prec) F.check(prec(r, zz));
               dot_partial_kernel<R, R><<<grid, kRedThreads, 0, c->stream>>>(nv, r, zz, ws->partials, 2); note_launch(c);
               cg_init_final_kernel<<<1, kFinThreads, 0, c->stream>>>(ws->sc, ws->ss, ws->partials, ns, G, rel_tol, max_iters,
                                                                      bnorm_given, gate_ir, h, use); note_launch(c);
               copy_kernel<R><<<ws->red_blocks, kRedThreads, 0, c->stream>>>(n, zz, p); note_launch(c);
           },
           [&](cudaGraphConditionalHandle h, int use) {
               F.check(apply(p, q));
               dot_partial_kernel<R, R><<<grid, kRedThreads, 0, c->stream>>>(nv, p, q, ws->partials, 0); note_launch(c);
               cg_alpha_kernel<<<1, kFinThreads, 0, c->stream>>>(ws->ss, ws->partials, ns, G); note_launch(c);
               cg_update_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, ws->ss, x, r, p, q, ws->partials); note_launch(c);
               if (use_prec) F.check(prec(r, zz));
               dot_partial_kernel<R, R><<<grid, kRedThreads, 0, c->stream>>>(nv, r, zz, ws->partials, 2); note_launch(c);
               cg_beta_kernel<<<1, kFinThreads, 0, c->stream>>>(ws->sc, ws->ss, ws->partials, ns, G, h, use); note_launch(c);
               cg_p_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, ws->ss, zz, p); note_launch(c);
               F.check(cudaGetLastError());
           });
}

// ---- GMRES(m) on vectors of type R -----------------------------------------------------
template <typename R, class Apply, class ApplyIdx, class Prec>
static void solve_gmres(Flow& F, Apply apply, ApplyIdx apply_idx, Prec prec, bool use_prec, const R* b, R* x, R* V, R* w,
                        R* zbuf, R* tbuf, double rel_tol, int max_iters, double bnorm_given, int gate_ir) {
    stdg_ctx* c = F.c;
    Workspace* ws = F.ws;
    const int64_t n = ws->n, nv = ws->nvec, ldv = ws->ldv;
    const int m = ws->m;
    const int ns = ws->ns, G = (int)ws->G;
    const dim3 grid = ws->grid();
    DevScalars* sc = ws->sc;
    ShotScalars* ss = ws->ss;
    double* part = ws->partials;
    F.loop(&sc->flag_outer,
           [&](cudaGraphConditionalHandle h, int use) {
               if (bnorm_given < 0) {
                   dot_partial_kernel<R, R><<<grid, kRedThreads, 0, c->stream>>>(nv, b, b, part, 0); note_launch(c);
               }
               gm_init_kernel<<<1, kFinThreads, 0, c->stream>>>(sc, ss, part, ns, G, rel_tol, max_iters, m, bnorm_given,
                                                                gate_ir, h, use); note_launch(c);
           },
           [&](cudaGraphConditionalHandle h_outer, int use_outer) {
               // restart cycle: true residual, then Arnoldi
               F.check(apply(x, w));
               gm_res_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, b, w, V, part); note_launch(c);
               F.loop(&sc->flag_inner,
                      [&](cudaGraphConditionalHandle h, int use) {
                          gm_cycle_start_kernel<<<1, kFinThreads, 0, c->stream>>>(sc, ss, part, ns, G, h, use); note_launch(c);
                          gm_scale0_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, sc, ss, V); note_launch(c);
                      },
                      [&](cudaGraphConditionalHandle h, int use) {
                          if (use_prec) {   // right preconditioning: w = A P^{-1} v_j
                              F.check(prec(V, zbuf, &sc->j, ldv));
                              F.check(apply(zbuf, w));
                          } else {
                              F.check(apply_idx(V, &sc->j, w));
                          }
                          // classical Gram-Schmidt: dots and ||w||^2; a second pass (with the first
                          // subtraction fused in) only for the shots that need it; subtraction + norm
                          gm_mdot_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, ldv, sc, V, w, part); note_launch(c);
                          gm_mdot_final_kernel<<<1, kFinThreads, 0, c->stream>>>(sc, ss, part, ns, G, 0); note_launch(c);
                          gm_orth_fused_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, ldv, sc, ss, V, w, part); note_launch(c);
                          gm_mdot_final_kernel<<<1, kFinThreads, 0, c->stream>>>(sc, ss, part, ns, G, 1); note_launch(c);
                          gm_maxpy_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, ldv, sc, ss, V, w, part); note_launch(c);
                          gm_norm_final_kernel<<<1, kFinThreads, 0, c->stream>>>(sc, ss, part, ns, G); note_launch(c);
                          gm_next_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, ldv, sc, ss, w, V); note_launch(c);
                          gm_givens_kernel<<<1, kFinThreads, 0, c->stream>>>(sc, ss, ns, h, use); note_launch(c);
                          F.check(cudaGetLastError());
                      });
               gm_solve_kernel<<<(ns + 127) / 128, 128, 0, c->stream>>>(ss, ns); note_launch(c);
               if (use_prec) {   // x += P^{-1} (V y)
                   gm_combine_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, ldv, ss, V, tbuf, 0); note_launch(c);
                   F.check(prec(tbuf, zbuf, nullptr, 0));
                   axpy_kernel<R><<<ws->red_blocks, kRedThreads, 0, c->stream>>>(n, x, zbuf); note_launch(c);
               } else {
                   gm_combine_kernel<R><<<grid, kRedThreads, 0, c->stream>>>(nv, ldv, ss, V, x, 1); note_launch(c);
               }
               gm_cycle_end_kernel<<<1, kFinThreads, 0, c->stream>>>(sc, ss, ns, h_outer, use_outer); note_launch(c);
               F.check(cudaGetLastError());
           });
}

// ---- all shots, one slab -----------------------------------------------------------------
static void record_solve(Flow& F, double dt, double* b, double* x) {
    stdg_ctx* c = F.c;
    Workspace* ws = F.ws;
    const int64_t nv = ws->nvec;
    const int ns = ws->ns, G = (int)ws->G;
    const dim3 grid = ws->grid();
    // CG for the SPD Crank-Nicolson system unless the preconditioner is the (non-symmetric) stencil one
    const bool cn = c->opt.scheme == STDG_SCHEME_CN && c->opt.preconditioner != 2;
    const bool pre = c->opt.preconditioner != 0;
    const bool p2 = c->opt.preconditioner == 2;
    const int64_t ldv = ws->ldv;
    auto A64 = [&](const double* xx, double* yy) { return launch_apply(c, dt, xx, yy, 1.0, nullptr, 0, ns); };
    auto A64i = [&](const double* V, const int* idx, double* yy) { return launch_apply(c, dt, V, yy, 1.0, idx, ldv, ns); };
    auto A32 = [&](const float* xx, float* yy) { return launch_apply32(c, dt, xx, yy, 1.0, nullptr, 0, ns); };
    auto A32i = [&](const float* V, const int* idx, float* yy) { return launch_apply32(c, dt, V, yy, 1.0, idx, ldv, ns); };
    auto P64 = [&](const double* r, double* z, const int* idx, int64_t ld) {
        return p2 ? launch_pre2_apply(c, r, z, idx, ld, ns) : launch_pre1_apply(c, r, z, idx, ld, ns);
    };
    auto P32 = [&](const float* r, float* z, const int* idx, int64_t ld) {
        return p2 ? launch_pre2_apply32(c, r, z, idx, ld, ns) : launch_pre1_apply32(c, r, z, idx, ld, ns);
    };
    auto P64c = [&](const double* r, double* z) { return launch_pre1_apply(c, r, z, nullptr, 0, ns); };
    auto P32c = [&](const float* r, float* z) { return launch_pre1_apply32(c, r, z, nullptr, 0, ns); };
    const double tol = c->opt.rel_tol;
    const int maxit = c->opt.max_iters;
    if (c->opt.precision == STDG_FP64) {
        if (cn) solve_cg<double>(F, A64, P64c, pre, b, x, ws->r, ws->p, ws->q, ws->z, tol, maxit, -1.0, 0);
        else solve_gmres<double>(F, A64, A64i, P64, pre, b, x, ws->V, ws->w, ws->z, ws->t, tol, maxit, -1.0, 0);
        zero_if_kernel<<<grid, kRedThreads, 0, c->stream>>>(nv, x, ws->ss, 0); note_launch(c);
        solve_stats_kernel<<<1, kFinThreads, 0, c->stream>>>(ws->sc, ws->ss, ns, cn ? 1 : 0); note_launch(c);
        return;
    }
    // mixed: FP64 refinement, FP32 inner solve with zero initial guess and unit RHS per shot
    F.loop(&ws->sc->ir_flag,
           [&](cudaGraphConditionalHandle h, int use) {
               dot_partial_kernel<double, double><<<grid, kRedThreads, 0, c->stream>>>(nv, b, b, ws->partials, 0); note_launch(c);
               ir_init_kernel<<<1, kFinThreads, 0, c->stream>>>(ws->sc, ws->ss, ws->partials, ns, G, tol, 64, h, use); note_launch(c);
           },
           [&](cudaGraphConditionalHandle h, int use) {
               F.check(A64(x, ws->w));
               gm_res_kernel<double><<<grid, kRedThreads, 0, c->stream>>>(nv, b, ws->w, ws->r, ws->partials); note_launch(c);
               ir_check_kernel<<<1, kFinThreads, 0, c->stream>>>(ws->sc, ws->ss, ws->partials, ns, G, maxit); note_launch(c);
               ir_convert_kernel<<<grid, kRedThreads, 0, c->stream>>>(nv, ws->sc, ws->ss, ws->r, ws->b32, ws->x32); note_launch(c);
               if (cn)
                   solve_cg<float>(F, A32, P32c, pre, ws->b32, ws->x32, ws->r32, ws->p32, ws->q32, ws->z32, c->opt.inner_tol,
                                   maxit, 1.0, 1);
               else
                   solve_gmres<float>(F, A32, A32i, P32, pre, ws->b32, ws->x32, ws->V32, ws->w32, ws->z32, ws->t32,
                                      c->opt.inner_tol, maxit, 1.0, 1);
               ir_update_kernel<<<grid, kRedThreads, 0, c->stream>>>(nv, ws->sc, ws->ss, ws->x32, x); note_launch(c);
               ir_end_kernel<<<1, 32, 0, c->stream>>>(ws->sc, h, use); note_launch(c);
               F.check(cudaGetLastError());
           });
    zero_if_kernel<<<grid, kRedThreads, 0, c->stream>>>(nv, x, ws->ss, 1); note_launch(c);
    solve_stats_kernel<<<1, kFinThreads, 0, c->stream>>>(ws->sc, ws->ss, ns, 2); note_launch(c);
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
    ws->ns = c->n_shots;
    ws->nvec = c->nvel;
    ws->n = c->nvel * (int64_t)c->n_shots;
    ws->red_blocks = (unsigned)(8 * c->n_sm);
    ws->G = (unsigned)std::max(1, (int)ws->red_blocks / ws->ns);
    const int64_t n = ws->n;
    const bool cn = c->opt.scheme == STDG_SCHEME_CN && c->opt.preconditioner != 2;   // CG workspace
    const bool mixed = c->opt.precision != STDG_FP64;
    const bool pre = c->opt.preconditioner != 0;
    int rc;
#define ALLOC(ptr, bytes) do { if ((rc = dev_alloc(c, (void**)&(ptr), (bytes))) != STDG_OK) return rc; \
                               ws->owned.push_back((void*)(ptr)); } while (0)
    ALLOC(ws->sc, sizeof(DevScalars));
    ALLOC(ws->ss, sizeof(ShotScalars) * ws->ns);
    ALLOC(ws->partials, sizeof(double) * (kMaxRestart + 2) * ws->G * ws->ns);
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
    cudaMemsetAsync(ws->ss, 0, sizeof(ShotScalars) * ws->ns, c->stream);
    cudaMemsetAsync(ws->dparams, 0, sizeof(double) * 4, c->stream);
    for (auto& s : ws->side) cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    return STDG_OK;
}

void solver_free(stdg_ctx* c) {
    Workspace* ws = W(c);
    if (!ws) return;
    for (int k = 0; k < 2; ++k) {
        if (ws->exec[k]) cudaGraphExecDestroy(ws->exec[k]);
        if (ws->graph[k]) cudaGraphDestroy(ws->graph[k]);
    }
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
    for (int k = 0; k < 2; ++k) {
        if (ws->exec[k]) cudaGraphExecDestroy(ws->exec[k]);
        if (ws->graph[k]) cudaGraphDestroy(ws->graph[k]);
        ws->exec[k] = nullptr;
        ws->graph[k] = nullptr;
        ws->graph_dt[k] = -1.0;
    }
}

double* solver_dparams(stdg_ctx* c) { return W(c) ? W(c)->dparams : nullptr; }

// the solve alone: A x = b on the stacked c->d_b / c->d_x (x holds the initial guess)
static void record_solve_only(Flow& F, double dt) {
    stdg_ctx* c = F.c;
    c->scopes.assign(1, 0);
    record_solve(F, dt, c->d_b, c->d_x);
    const long k = c->scopes.back() + 1;
    c->scopes.clear();
    count_kernel<<<1, 32, 0, c->stream>>>(F.ws->sc, k);
    F.check(cudaGetLastError());
}

// Runs `n` repetitions of a recorded body (kind 0: a whole step, 1: the solve alone), as one
// cached CUDA graph per kind and dt, or from the host loop; then reads the statistics.
static int run_body_n(stdg_ctx* c, double dt, int n, int kind, stdg_stats* st) {
    Workspace* ws = W(c);
    STDG_CUDA(c, cudaMemsetAsync(&ws->sc->st_total, 0, sizeof(int) * 5, c->stream));
    STDG_CUDA(c, cudaMemsetAsync(&ws->sc->st_final_rel, 0, sizeof(double) * 2, c->stream));
    STDG_CUDA(c, cudaMemsetAsync(&ws->sc->launches, 0, sizeof(unsigned long long), c->stream));
    auto record = [&](Flow& F) {
        if (kind == 0) record_step(F, dt);
        else record_solve_only(F, dt);
    };
    if (c->opt.use_graph) {
        if (!ws->exec[kind] || ws->graph_dt[kind] != dt) {
            if (ws->exec[kind]) cudaGraphExecDestroy(ws->exec[kind]);
            if (ws->graph[kind]) cudaGraphDestroy(ws->graph[kind]);
            ws->exec[kind] = nullptr;
            ws->graph[kind] = nullptr;
            cudaStream_t s0 = c->stream;
            STDG_CUDA(c, cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed));
            Flow F{c, ws, true};
            record(F);
            c->stream = s0;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(s0, &g);
            if (F.err != cudaSuccess || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                c->err = std::string("graph capture failed: ") + cudaGetErrorString(F.err != cudaSuccess ? F.err : e);
                cudaGetLastError();
                return STDG_ECUDA;
            }
            ws->graph[kind] = g;
            STDG_CUDA(c, cudaGraphInstantiate(&ws->exec[kind], g, 0));
            ws->graph_dt[kind] = dt;
        }
        for (int s = 0; s < n; ++s) STDG_CUDA(c, cudaGraphLaunch(ws->exec[kind], c->stream));
    } else {
        for (int s = 0; s < n; ++s) {
            Flow F{c, ws, false};
            record(F);
            if (F.err != cudaSuccess) STDG_CUDA(c, F.err);
        }
    }
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    STDG_CUDA(c, cudaGetLastError());
    DevScalars h;
    STDG_CUDA(c, cudaMemcpy(&h, ws->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost));
    if (st) {
        st->iters_total = (int)h.st_iters_sum;
        st->iters_max = h.st_max;
        st->refinements = h.st_refine;
        st->final_rel_res = h.st_final_rel;
        st->status = h.st_nonfinite ? STDG_ENONFINITE : h.st_notconv ? STDG_ENOTCONV : STDG_OK;
    }
    c->last_launches = (int64_t)h.launches;
    {
        const int rc = take_device_error(c);
        if (rc != STDG_OK) return rc;
    }
    if (h.st_nonfinite) STDG_FAIL(c, STDG_ENONFINITE, "a residual or right-hand-side norm is NaN or Inf (input overflow?)");
    if (h.st_notconv) STDG_FAIL(c, STDG_ENOTCONV, "Krylov solve reached max_iters");
    return STDG_OK;
}

int solver_step(stdg_ctx* c, double dt, int n_steps, stdg_stats* st) {
    Workspace* ws = W(c);
    if (!ws) STDG_FAIL(c, STDG_ESTATE, "solver not set up");
    {
        const int rc = precond_for_dt(c, dt);
        if (rc != STDG_OK) return rc;
    }
    const double t0 = c->t;
    STDG_CUDA(c, cudaMemcpyAsync(ws->dparams, &t0, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    {
        double stepidx = (double)c->rec_steps;
        STDG_CUDA(c, cudaMemcpyAsync(ws->dparams + 2, &stepidx, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    }
    c->wait_gave_up = false;
    const int rc = run_body_n(c, dt, n_steps, 0, st);
    // the state advanced when the solve did not converge and when a bounded wait gave up
    // (then with invalid values); a CUDA error proper leaves time and records where they were
    if (rc == STDG_OK || rc == STDG_ENOTCONV || rc == STDG_ENONFINITE || c->wait_gave_up) {
        c->t = t0 + n_steps * dt;
        c->rec_steps += n_steps;
    }
    return rc;
}

int solver_solve(stdg_ctx* c, double dt, stdg_stats* st) {
    Workspace* ws = W(c);
    if (!ws) STDG_FAIL(c, STDG_ESTATE, "solver not set up");
    const int rc = precond_for_dt(c, dt);
    if (rc != STDG_OK) return rc;
    return run_body_n(c, dt, 1, 1, st);
}

}  // namespace stdg
