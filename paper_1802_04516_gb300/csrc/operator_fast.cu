// Face kernels of the Schur velocity operator with compile-time sizes (dimension d,
// N_phi, N_gamma) for the production shapes; other shapes use the generic kernel in
// kernels.cu.  Same arithmetic as the generic kernel (Eq. velocity.sys with Q~ = -D^T
// and the orthonormalised dual basis):
//   g = sum_side D~_side^T v_side,  t = E_j : g,  h = scale * S t,  y_side += D~_side h.
// One warp per face.  Lanes hold one column (gather) and one row (scatter) of the face's
// D~ blocks in registers; the rows of v and h they multiply are read by all lanes at once
// from shared memory (broadcast), in adjacent pairs through one 8-byte load and one packed
// FP32 FMA.  Two variants: a register kernel that loops over the shots of a stacked
// multi-shot vector with D~ kept in registers (two shots at a time, one per half-warp, when
// a column and a row of D~ fit in 16 lanes: 2D with p <= 2), and a single-shot kernel that streams the
// next face's D~ block and element rows into shared memory with cp.async.bulk while the
// warp computes the current face.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "stdg_internal.h"
#include "tma.h"

namespace stdg {

template <typename R> struct Vec;
template <> struct Vec<float> { using T = float4; static constexpr int W = 4; };
template <> struct Vec<double> { using T = double2; static constexpr int W = 2; };

__host__ __device__ constexpr int round_up(int v, int w) { return (v + w - 1) / w * w; }

template <int DIM>
__device__ __forceinline__ int symc(int a, int b) {
    if (a == b) return a;
    if (DIM == 2) return 2;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return (lo == 0 && hi == 1) ? 3 : (lo == 1 ? 4 : 5);
}

template <int DIM, int NP, int NG, typename R>
struct FaceReg {
    static constexpr int NS = DIM == 2 ? 3 : 6;
    static constexpr int W = Vec<R>::W;
    static constexpr int NPP = (NP + W - 1) / W * W;     // padded row length (16-byte multiple)
    static constexpr int NVS = DIM * NG * NP;            // values per element
    static constexpr int SZ_V = 2 * DIM * NG * NPP;      // rows (s,k,b) of the neighbours' values
    static constexpr int SZ_G = round_up(DIM * DIM * NG * NP, W);   // g[k][l][b][m]
    static constexpr int SZ_T = round_up(NS * NG * NP, W);          // t[c][b][m]
    static constexpr int SZ_H = NS * NG * NPP;           // rows (c,b) of h
    static constexpr int PER_WARP = 2 * SZ_V + SZ_G + SZ_T + SZ_H;   // per shot in flight (two value buffers)
    // several shots: two per warp (one per half-warp) when a column and a row of D~ fit in 16 lanes
    static constexpr int HALVES = (DIM * NP <= 16 && 2 * NP <= 16) ? 2 : 1;
};

// element-sized asynchronous global -> shared copy (zero-filled when `bytes` is 0)
template <typename R>
__device__ __forceinline__ void cp_async_elem(R* dst, const R* src, bool on) {
    const uint32_t d = smem_u32(dst);
    if constexpr (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(on ? 4u : 0u) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(on ? 8u : 0u) : "memory");
}

// acc + sum_{n<NP} a[n] row[n] for a broadcast shared-memory row.  FP32 with NP even: the
// row starts on an 8-byte boundary, so pairs (n, n+1) come in one 8-byte load and go through
// one packed FMA (even and odd partial sums, added at the end).
template <int NP, typename R>
__device__ __forceinline__ R dot_row(const R (&a)[NP], const R* row, R acc) {
    if constexpr (std::is_same<R, float>::value && NP % 2 == 0) {
        const float2* r2 = reinterpret_cast<const float2*>(row);
        float2 s = make_float2(acc, 0.0f);
#pragma unroll
        for (int i = 0; i < NP / 2; ++i) s = ffma2(make_float2(a[2 * i], a[2 * i + 1]), r2[i], s);
        return s.x + s.y;
    } else {
#pragma unroll
        for (int n = 0; n < NP; ++n) acc = fma(a[n], row[n], acc);
        return acc;
    }
}

// Register-blocked face kernel.  Gather lanes own a column (l, m) of D~_s (both sides, N_phi
// values each, in registers); scatter lanes own a row (s, n) of D~_s (all l, m).  The rows
// of v and h they multiply are read by all lanes at once from shared memory (broadcast), so
// almost every instruction of the inner products is an FMA.  HALVES = 2: both half-warps
// hold the same D~ registers and work on shots s0 and s0 + 1, each with its own shared rows.
template <int DIM, int NP, int NG, typename R, int HALVES>
__global__ void __launch_bounds__(128) face_apply_fast_kernel(int64_t n_face, const int32_t* __restrict__ fl,
                                                              const int32_t* __restrict__ fr, const R* __restrict__ D,
                                                              const R* __restrict__ lamf, const R* __restrict__ muf,
                                                              const RefTables* __restrict__ rtp, const R* __restrict__ x0,
                                                              const int* __restrict__ xidx, int64_t ld, R* __restrict__ y0,
                                                              R scale, int nshots, int64_t nvec) {
    using F = FaceReg<DIM, NP, NG, R>;
    const R* x = x0;
    constexpr int NS = F::NS, NPP = F::NPP, NVS = F::NVS;
    constexpr int LANES = 32 / HALVES;
    static_assert(HALVES == 1 || (DIM * NP <= 16 && 2 * NP <= 16), "two shots per warp need d*N_phi <= 16");
    static_assert(DIM * NP <= 32 && 2 * NP <= 32, "register-blocked face kernel needs d*N_phi <= 32");
    extern __shared__ __align__(16) unsigned char smraw[];
    R* sm = reinterpret_cast<R*>(smraw);
    if (xidx) x += (int64_t)(*xidx) * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    __shared__ R sS[NG * NG];
    for (int t = threadIdx.x; t < NG * NG; t += blockDim.x) sS[t] = (R)rtp->S[t];
    // with HALVES = 2 each half-warp works on its own shot (same D~ registers, own buffers)
    const int hv = lane / LANES, li = lane % LANES;
    R* sV0 = sm + (warp * HALVES + hv) * F::PER_WARP;   // [s][k][b][n] rows padded, two buffers
    R* sG = sV0 + 2 * F::SZ_V;         // [k][l][b][m]
    R* sT = sG + F::SZ_G;              // [c][b][m]
    R* sH = sT + F::SZ_T;              // [c][b][m] rows padded
    for (int t = li; t < F::PER_WARP; t += LANES) sV0[t] = (R)0;   // padding stays zero
    __syncthreads();
    const bool gl = li < DIM * NP;            // gather lane: column (gl_l, gl_m)
    const int gl_l = gl ? li / NP : 0, gl_m = gl ? li % NP : 0;
    const bool sc = li < 2 * NP;              // scatter lane: row (sc_s, sc_n)
    const int sc_s = sc ? li / NP : 0, sc_n = sc ? li % NP : 0;
    constexpr int DFACE = 2 * DIM * NP * NP;
    for (int64_t f = blockIdx.x * (int64_t)wpb + warp; f < n_face; f += (int64_t)gridDim.x * wpb) {
        const int el = fl[f], er = fr[f];
        const R* Df = D + f * (int64_t)DFACE;
        // ---- registers: gather column and scatter row of D~
        R Dg[2][NP], Ds[DIM][NP];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int n = 0; n < NP; ++n) Dg[s][n] = gl ? Df[((s * DIM + gl_l) * NP + n) * NP + gl_m] : (R)0;
#pragma unroll
        for (int l = 0; l < DIM; ++l)
#pragma unroll
            for (int m = 0; m < NP; ++m) Ds[l][m] = sc ? Df[((sc_s * DIM + l) * NP + sc_n) * NP + m] : (R)0;
        const R lam = lamf[f], mu = muf[f];
        // the neighbours' values of a shot, rows (s,k,b) padded, copied asynchronously one shot
        // (pair) ahead into the other buffer, so that the loads overlap the current shot's work
        auto issue = [&](int s0n, R* buf) {
            const bool vld = s0n + hv < nshots;
            const int64_t base = (int64_t)(vld ? s0n + hv : 0) * nvec;
            const R* xl = x + base + (int64_t)el * NVS;
            const R* xr = x + base + (int64_t)(er >= 0 ? er : el) * NVS;
#pragma unroll
            for (int e0 = 0; e0 < NVS; e0 += LANES) {
                const int e = e0 + li;
                if (e < NVS) {
                    const int row = e / NP, n = e % NP;
                    cp_async_elem(buf + row * NPP + n, vld ? xl + e : x, vld);
                    cp_async_elem(buf + (DIM * NG + row) * NPP + n, vld && er >= 0 ? xr + e : x, vld && er >= 0);
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        issue(0, sV0);
        // D~ stays in registers for every shot of the batch
        for (int s0 = 0, it = 0; s0 < nshots; s0 += HALVES, ++it) {
        const bool valid = s0 + hv < nshots;
        const int shot = valid ? s0 + hv : s0;
        R* y = y0 + (int64_t)shot * nvec;
        R* sV = sV0 + (it & 1) * F::SZ_V;
        if (s0 + HALVES < nshots) {
            issue(s0 + HALVES, sV0 + ((it + 1) & 1) * F::SZ_V);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        // ---- gather: g[k][l][b][m] = sum_s sum_n D~_s[l][n][m] v_s[k][b][n]
#pragma unroll
        for (int kb = 0; kb < DIM * NG; ++kb) {
            R acc = 0;
#pragma unroll
            for (int s = 0; s < 2; ++s) acc = dot_row<NP, R>(Dg[s], sV + (s * DIM * NG + kb) * NPP, acc);
            if (gl) {
                const int k = kb / NG, b = kb % NG;
                sG[((k * DIM + gl_l) * NG + b) * NP + gl_m] = acc;
            }
        }
        __syncwarp();
        // ---- t = E_j : g
        constexpr int NT_OUT = NS * NG * NP;
#pragma unroll
        for (int e0 = 0; e0 < NT_OUT; e0 += LANES) {
            const int e = e0 + li;
            if (e < NT_OUT) {
                const int c = e / (NG * NP);
                const int bm = e % (NG * NP);
                int a, bb;
                if (c < DIM) { a = c; bb = c; }
                else if (DIM == 2) { a = 0; bb = 1; }
                else { a = c == 3 ? 0 : (c == 4 ? 1 : 0); bb = c == 3 ? 1 : 2; }
                R val = mu * (sG[(a * DIM + bb) * NG * NP + bm] + sG[(bb * DIM + a) * NG * NP + bm]);
                if (a == bb) {
                    R tr = 0;
#pragma unroll
                    for (int q = 0; q < DIM; ++q) tr += sG[(q * DIM + q) * NG * NP + bm];
                    val += lam * tr;
                }
                sT[e] = val;
            }
        }
        __syncwarp();
        // ---- h = scale * S t  (rows (c,b), padded)
#pragma unroll
        for (int e0 = 0; e0 < NT_OUT; e0 += LANES) {
            const int e = e0 + li;
            if (e < NT_OUT) {
                const int c = e / (NG * NP), b = (e / NP) % NG, m = e % NP;
                R acc = 0;
#pragma unroll
                for (int b2 = 0; b2 < NG; ++b2) acc += sS[b * NG + b2] * sT[(c * NG + b2) * NP + m];
                sH[(c * NG + b) * NPP + m] = scale * acc;
            }
        }
        __syncwarp();
        // ---- scatter: y_s[k][b][n] += sum_l sum_m D~_s[l][n][m] h[(k,l)][b][m]
        const int es = sc_s == 0 ? el : er;
        const bool write = sc && es >= 0 && valid;
#pragma unroll
        for (int kb = 0; kb < DIM * NG; ++kb) {
            const int k = kb / NG, b = kb % NG;
            R acc = 0;
#pragma unroll
            for (int l = 0; l < DIM; ++l) acc = dot_row<NP, R>(Ds[l], sH + (symc<DIM>(k, l) * NG + b) * NPP, acc);
            if (write) atomicAdd(&y[(int64_t)es * NVS + kb * NP + sc_n], acc);
        }
        __syncwarp();
        }   // shots
    }
}

// ---------------------------------------------------------------------------------
// TMA-pipelined variant: the next face's D~ block and its two elements' value rows are
// copied into shared memory by cp.async.bulk (one elected lane, completion on a per-warp
// mbarrier) while the warp computes the current face.  Register/broadcast arithmetic as
// above.  Every wait on an mbarrier is bounded; on timeout the kernel records the error
// in *err and the warp stops after draining its copies in flight (bounded too).
// ---------------------------------------------------------------------------------
template <int DIM, int NP, int NG, typename R>
struct FaceTma {
    static constexpr int NS = DIM == 2 ? 3 : 6;
    static constexpr int NVS = DIM * NG * NP;
    static constexpr int DFACE = 2 * DIM * NP * NP;
    static constexpr bool XBULK = (NVS * sizeof(R)) % 16 == 0;        // element rows copyable by TMA
    static constexpr int STAGE = round_up(DFACE, 16 / (int)sizeof(R)) + 2 * round_up(NVS, 16 / (int)sizeof(R));
    static constexpr int SZ_G = round_up(DIM * DIM * NG * NP, 4);
    static constexpr int SZ_T = round_up(NS * NG * NP, 4);
    static constexpr int SZ_H = round_up(NS * NG * NP, 4);
    static constexpr int PER_WARP = round_up(2 * STAGE + SZ_G + SZ_T + SZ_H, 16 / (int)sizeof(R));
    // resident blocks of 4 warps requested per SM when the register cap is on (the autotuner
    // times the kernel with and without it)
    static constexpr int MIN_BLOCKS = (DIM == 2 && NP == 6) ? 6 : (DIM == 2 && NP == 10) ? 6 : (DIM == 3 && NP == 10) ? 4 : 2;
};

template <int DIM, int NP, int NG, typename R, int MINB>
__global__ void __launch_bounds__(128, MINB) face_apply_tma_kernel(int64_t n_face, const int32_t* __restrict__ fl,
                                                             const int32_t* __restrict__ fr, const R* __restrict__ D,
                                                             const R* __restrict__ lamf, const R* __restrict__ muf,
                                                             const RefTables* __restrict__ rtp, const R* __restrict__ x,
                                                             const int* __restrict__ xidx, int64_t ld, R* __restrict__ y,
                                                             R scale, int* __restrict__ err) {
    using F = FaceTma<DIM, NP, NG, R>;
    constexpr int NS = F::NS, NVS = F::NVS, DFACE = F::DFACE;
    constexpr int XOFF = round_up(DFACE, 16 / (int)sizeof(R));
    constexpr int XR = round_up(NVS, 16 / (int)sizeof(R));
    static_assert(DIM * NP <= 32 && 2 * NP <= 32, "register-blocked face kernel needs d*N_phi <= 32");
    static_assert((DFACE * sizeof(R)) % 16 == 0, "D~ block must be a multiple of 16 bytes");
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[4][2];
    __shared__ R sS[NG * NG];
    if (xidx) x += (int64_t)(*xidx) * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int t = threadIdx.x; t < NG * NG; t += blockDim.x) sS[t] = (R)rtp->S[t];
    R* base = reinterpret_cast<R*>(smraw) + warp * F::PER_WARP;
    auto stage = [&](int s_) { return s_ ? base + F::STAGE : base; };
    R* sG = base + 2 * F::STAGE;
    R* sT = sG + F::SZ_G;
    R* sH = sT + F::SZ_T;
    for (int t = lane; t < 2 * F::STAGE; t += 32) base[t] = (R)0;   // the r-side rows of boundary faces stay finite
    const uint32_t bar0 = smem_u32(&bars[warp][0]), bar1 = smem_u32(&bars[warp][1]);
    if (lane == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool gl = lane < DIM * NP;
    const int gl_l = gl ? lane / NP : 0, gl_m = gl ? lane % NP : 0;
    const bool sc = lane < 2 * NP;
    const int sc_s = sc ? lane / NP : 0, sc_n = sc ? lane % NP : 0;
    const int64_t stride = (int64_t)gridDim.x * wpb;
    constexpr long kPollLimit = 1L << 24;

    auto issue = [&](int64_t f, int st) {   // lane 0 only
        const int el = fl[f], er = fr[f];
        const uint32_t bar = st ? bar1 : bar0;
        uint32_t bytes = DFACE * sizeof(R);
        if (F::XBULK) bytes += (er >= 0 ? 2 : 1) * NVS * sizeof(R);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, bytes);
        bulk_g2s(smem_u32(stage(st)), D + f * (int64_t)DFACE, DFACE * sizeof(R), bar);
        if (F::XBULK) {
            bulk_g2s(smem_u32(stage(st) + XOFF), x + (int64_t)el * NVS, NVS * sizeof(R), bar);
            if (er >= 0) bulk_g2s(smem_u32(stage(st) + XOFF + XR), x + (int64_t)er * NVS, NVS * sizeof(R), bar);
        }
    };

    int64_t f = blockIdx.x * (int64_t)wpb + warp;
    if (f < n_face && lane == 0) issue(f, 0);
    uint32_t ph0 = 0, ph1 = 0;
    int st = 0;
    for (; f < n_face; f += stride) {
        const int64_t fn = f + stride;
        if (fn < n_face && lane == 0) issue(fn, st ^ 1);
        if (!mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0, kPollLimit)) {
            if (lane == 0) atomicExch(err, 1);
            // before the CTA leaves, both stages' copies must have landed: the late one for f and
            // the one issued for fn (both waits bounded); if either does not, record code 2
            bool drained = mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0, kPollLimit);
            if (fn < n_face) drained = mbar_wait(st ? bar0 : bar1, st ? ph0 : ph1, kPollLimit) && drained;
            if (!drained && lane == 0) atomicExch(err, 2);
            break;
        }
        if (st) ph1 ^= 1u; else ph0 ^= 1u;
        const R* sD = stage(st);
        const R* sV = stage(st) + XOFF;   // rows (s,k,b), NP values each, side r at +XR
        const int el = fl[f], er = fr[f];
        if (!F::XBULK) {   // element rows by plain loads
            R* w = stage(st) + XOFF;
#pragma unroll
            for (int e0 = 0; e0 < NVS; e0 += 32) {
                const int e = e0 + lane;
                if (e < NVS) {
                    w[e] = x[(int64_t)el * NVS + e];
                    w[XR + e] = er >= 0 ? x[(int64_t)er * NVS + e] : (R)0;
                }
            }
            __syncwarp();
        }
        R Dg[2][NP], Ds[DIM][NP];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int n = 0; n < NP; ++n) Dg[s][n] = sD[((s * DIM + gl_l) * NP + n) * NP + gl_m];
#pragma unroll
        for (int l = 0; l < DIM; ++l)
#pragma unroll
            for (int m = 0; m < NP; ++m) Ds[l][m] = sD[((sc_s * DIM + l) * NP + sc_n) * NP + m];
        // gather (side r contributes zero on a boundary face: its D~ block is zero)
#pragma unroll
        for (int kb = 0; kb < DIM * NG; ++kb) {
            R acc = 0;
#pragma unroll
            for (int s = 0; s < 2; ++s) acc = dot_row<NP, R>(Dg[s], sV + s * XR + kb * NP, acc);
            if (gl) sG[((kb / NG * DIM + gl_l) * NG + kb % NG) * NP + gl_m] = acc;
        }
        __syncwarp();
        const R lam = lamf[f], mu = muf[f];
        constexpr int NT_OUT = NS * NG * NP;
#pragma unroll
        for (int e0 = 0; e0 < NT_OUT; e0 += 32) {
            const int e = e0 + lane;
            if (e < NT_OUT) {
                const int c = e / (NG * NP);
                const int bm = e % (NG * NP);
                int a, bb;
                if (c < DIM) { a = c; bb = c; }
                else if (DIM == 2) { a = 0; bb = 1; }
                else { a = c == 3 ? 0 : (c == 4 ? 1 : 0); bb = c == 3 ? 1 : 2; }
                R val = mu * (sG[(a * DIM + bb) * NG * NP + bm] + sG[(bb * DIM + a) * NG * NP + bm]);
                if (a == bb) {
                    R tr = 0;
#pragma unroll
                    for (int q = 0; q < DIM; ++q) tr += sG[(q * DIM + q) * NG * NP + bm];
                    val += lam * tr;
                }
                sT[e] = val;
            }
        }
        __syncwarp();
#pragma unroll
        for (int e0 = 0; e0 < NT_OUT; e0 += 32) {
            const int e = e0 + lane;
            if (e < NT_OUT) {
                const int c = e / (NG * NP), b = (e / NP) % NG, m = e % NP;
                R acc = 0;
#pragma unroll
                for (int b2 = 0; b2 < NG; ++b2) acc += sS[b * NG + b2] * sT[(c * NG + b2) * NP + m];
                sH[e] = scale * acc;   // rows (c,b), NP values
            }
        }
        __syncwarp();
        const int es = sc_s == 0 ? el : er;
        const bool write = sc && es >= 0;
#pragma unroll
        for (int kb = 0; kb < DIM * NG; ++kb) {
            const int k = kb / NG, b = kb % NG;
            R acc = 0;
#pragma unroll
            for (int l = 0; l < DIM; ++l) acc = dot_row<NP, R>(Ds[l], sH + (symc<DIM>(k, l) * NG + b) * NP, acc);
            if (write) atomicAdd(&y[(int64_t)es * NVS + kb * NP + sc_n], acc);
        }
        __syncwarp();   // stage st is free for the copy issued in the next iteration
        st ^= 1;
    }
}

// ---------------------------------------------------------------------------------
// Tiled single-shot FP32 kernel for 2D, p = 3 (d = 2, N_phi = 10, N_gamma = 4).  Per face the
// gather g[(k,b)][(l,m)] = sum_(s,n) v_s[k][b][n] D~_s[l][n][m] and the scatter
// y_s[k][b][n] += sum_(l,m) D~_s[l][n][m] h[(k,l)][b][m] are 8 x 20 x 20 products.  Four faces
// per warp, eight lanes each; lane (k, q) owns the four time-node rows (k, b) and column group
// q of (l, m) (l = q/2, m in 5(q%2) .. +4):
//   gather:  g[(k,b)][group q] over the full (s, n) contraction, tiles (Rg, q), Rg = 0..3;
//   E : g :  partner lane (1-k, q^2) holds g[1-k][1-l] (one shuffle per value);
//   S t   :  in registers (the lane holds every time node);
//   scatter: partial sums over the lane's own columns with the same tiles (Rg, q), then a
//            reduce-scatter over the four column lanes (shuffles): each lane ends with one
//            time-node row of each row group Rg, 5 values, added to y with packed atomics.
// Shared memory delivers one 4-byte value per lane and clock however many lanes share an
// address, so the work per value loaded decides the rate: every tile value loaded feeds four
// rows.  D~ is stored per face as 16 tiles of 5 x 5 (row group Rg of (s,n) x column group C of
// (l,m)), 28 floats each, at swizzled positions 4Rg + (C+Rg)%4, so the four tiles a quarter-warp
// reads fall in distinct banks.  Inside a tile the values are paired by adjacent rows (the pairs
// that meet adjacent pairs of v in one 8-byte load), so both products run on the packed FP32
// FMA.  The face's D~ block and element rows arrive by cp.async.bulk one group of faces ahead.
// ---------------------------------------------------------------------------------
struct FaceTile {
    static constexpr int NP = 10, NG = 4, NVS = 2 * NG * NP;   // 80 values per element
    static constexpr int TS = 28;                    // floats per 5 x 5 tile (3 of padding)
    static constexpr int DT = 16 * TS;               // 448 floats per face
    static constexpr int XOFF = DT, XR = NVS;        // element rows after the tiles
    static constexpr int FPW = 4;                    // faces per warp
    static constexpr int FACE_SEG = 624;             // 156 x 16 bytes: a half-warp's two faces 4 bank groups apart
    static constexpr int STAGE = FPW * FACE_SEG;
    static constexpr int PER_WARP = 2 * STAGE;
    static_assert(XOFF + 2 * XR <= FACE_SEG && PER_WARP % 4 == 0, "tile kernel layout");
};

__host__ __device__ constexpr int tile_pos(int Rg, int C) { return 4 * Rg + ((C + Rg) & 3); }

// tile slot -> (r, c) of the 5 x 5 tile of row group Rg (rows paired (0,1),(2,3) | 4 for even
// Rg, (1,2),(3,4) | 0 for odd Rg); false for padding
__host__ __device__ inline bool tile_slot_rc(int slot, int odd, int* r, int* c) {
    if (slot < 10) { *c = slot >> 1; *r = (slot & 1) + (odd ? 1 : 0); return true; }
    if (slot < 20) { *c = (slot - 10) >> 1; *r = (slot & 1) + (odd ? 3 : 2); return true; }
    if (slot < 25) { *c = slot - 20; *r = odd ? 0 : 4; return true; }
    return false;
}

// FP64 D~ [face][s][l][n][m] -> FP32 tiles
__global__ void tile_d32_kernel(int64_t n_face, const double* __restrict__ D, float* __restrict__ Dt) {
    using F = FaceTile;
    const int64_t n = n_face * F::DT;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = i / F::DT;
        const int w = (int)(i % F::DT), pos = w / F::TS, slot = w % F::TS;
        const int Rg = pos >> 2, C = ((pos & 3) - Rg) & 3;
        int r, c;
        float v = 0.f;
        if (tile_slot_rc(slot, Rg & 1, &r, &c)) {
            const int s = Rg >> 1, nn = 5 * (Rg & 1) + r, l = C >> 1, m = 5 * (C & 1) + c;
            v = (float)D[f * (2 * 2 * F::NP * F::NP) + ((s * 2 + l) * F::NP + nn) * F::NP + m];
        }
        Dt[i] = v;
    }
}

// y[0] += a (and y[1] += b): reductions without a returned value (y 8-byte aligned for two)
__device__ __forceinline__ void red_add2(float* y, float a, float b) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(y), "f"(a), "f"(b) : "memory");
}
__device__ __forceinline__ void red_add1(float* y, float a) {
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(y), "f"(a) : "memory");
}

__device__ __forceinline__ void load_tile(const float* p, float (&t)[FaceTile::TS]) {
    const float4* p4 = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int j = 0; j < FaceTile::TS / 4; ++j) {
        const float4 v = p4[j];
        t[4 * j] = v.x; t[4 * j + 1] = v.y; t[4 * j + 2] = v.z; t[4 * j + 3] = v.w;
    }
}

template <int MAXREG>
__global__ void __maxnreg__(MAXREG) face_apply_tile_kernel(int64_t n_face, const int32_t* __restrict__ fl,
                                                              const int32_t* __restrict__ fr, const float* __restrict__ Dt,
                                                              const float* __restrict__ lamf, const float* __restrict__ muf,
                                                              const RefTables* __restrict__ rtp, const float* __restrict__ x,
                                                              const int* __restrict__ xidx, int64_t ld, float* __restrict__ y,
                                                              float scale, int* __restrict__ err) {
    using F = FaceTile;
    constexpr int TS = F::TS, NVS = F::NVS, NG = F::NG, FPW = F::FPW;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[4][2];
    if (xidx) x += (int64_t)(*xidx) * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    float* base = reinterpret_cast<float*>(smraw) + warp * F::PER_WARP;
    for (int t = lane; t < F::PER_WARP; t += 32) base[t] = 0.f;   // rows of absent r sides stay finite
    const uint32_t bar0 = smem_u32(&bars[warp][0]), bar1 = smem_u32(&bars[warp][1]);
    if (lane == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int fq = lane >> 3, k = (lane >> 2) & 1, q = lane & 3;
    // qs = q with its two bits swapped.  scale * S with the rows in this lane's order (slot i =
    // time node i ^ qs): the scatter's partial sums then come out in the order in which the
    // reduce-scatter over the column lanes sends and keeps them (first step with lane q^1: slots
    // 0,1 kept, 2,3 sent; second step with lane q^2: slot 0 kept, 1 sent), and the lane ends
    // with time node qs
    const int qs = ((q & 1) << 1) | (q >> 1);
    float Sm[NG][NG];
#pragma unroll
    for (int i = 0; i < NG; ++i)
#pragma unroll
        for (int b = 0; b < NG; ++b) Sm[i][b] = scale * (float)rtp->S[(i ^ qs) * NG + b];
    const int64_t n_grp = (n_face + FPW - 1) / FPW;
    const int64_t stride = (int64_t)gridDim.x * wpb;
    constexpr long kPollLimit = 1L << 24;

    // element ids of the faces of group pp (every lane loads them, one group before the copies
    // that need them are issued, so that lane 0 does not stall the warp on the loads)
    auto load_ids = [&](int64_t pp, int (&el)[FPW], int (&er)[FPW]) {
#pragma unroll
        for (int i = 0; i < FPW; ++i) {
            const int64_t f = FPW * pp + i;
            const bool ok = pp < n_grp && f < n_face;
            el[i] = ok ? fl[f] : -1;
            er[i] = ok ? fr[f] : -1;
        }
    };
    auto issue = [&](int64_t p, int st, const int (&el)[FPW], const int (&er)[FPW]) {   // lane 0 only
        const uint32_t bar = st ? bar1 : bar0;
        float* sg = base + st * F::STAGE;
        uint32_t bytes = 0;
#pragma unroll
        for (int i = 0; i < FPW; ++i)
            if (el[i] >= 0) bytes += (F::DT + (er[i] >= 0 ? 2 : 1) * NVS) * sizeof(float);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, bytes);
#pragma unroll
        for (int i = 0; i < FPW; ++i) {
            if (el[i] < 0) continue;
            float* seg = sg + i * F::FACE_SEG;
            bulk_g2s(smem_u32(seg), Dt + (FPW * p + i) * (int64_t)F::DT, F::DT * sizeof(float), bar);
            bulk_g2s(smem_u32(seg + F::XOFF), x + (int64_t)el[i] * NVS, NVS * sizeof(float), bar);
            if (er[i] >= 0) bulk_g2s(smem_u32(seg + F::XOFF + F::XR), x + (int64_t)er[i] * NVS, NVS * sizeof(float), bar);
        }
    };

    // the lane's face of group pp: element ids and Lame parameters, loaded one group ahead
    auto fetch = [&](int64_t pp, int& a, int& b, float& l, float& m) {
        const int64_t ff = FPW * pp + fq;
        const bool ok = pp < n_grp && ff < n_face;
        a = ok ? fl[ff] : -1;
        b = ok ? fr[ff] : -1;
        l = ok ? lamf[ff] : 0.f;
        m = ok ? muf[ff] : 0.f;
    };
    int64_t p = blockIdx.x * (int64_t)wpb + warp;
    int idl[FPW], idr[FPW];   // ids of the group whose copies are issued next
    load_ids(p, idl, idr);
    if (p < n_grp && lane == 0) issue(p, 0, idl, idr);
    load_ids(p + stride, idl, idr);
    int el, er;
    float lam, mu;
    fetch(p, el, er, lam, mu);
    uint32_t ph0 = 0, ph1 = 0;
    int st = 0;
    for (; p < n_grp; p += stride) {
        const int64_t pn = p + stride;
        if (pn < n_grp && lane == 0) issue(pn, st ^ 1, idl, idr);
        int nidl[FPW], nidr[FPW];
        load_ids(pn + stride, nidl, nidr);
        int el_n, er_n;
        float lam_n, mu_n;
        fetch(pn, el_n, er_n, lam_n, mu_n);
        // the lanes leave together (the shuffles below take the whole warp)
        if (!__all_sync(FULL, mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0, kPollLimit))) {
            if (lane == 0) atomicExch(err, 1);
            bool drained = mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0, kPollLimit);
            if (pn < n_grp) drained = mbar_wait(st ? bar0 : bar1, st ? ph0 : ph1, kPollLimit) && drained;
            if (!drained && lane == 0) atomicExch(err, 2);
            break;
        }
        if (st) ph1 ^= 1u; else ph0 ^= 1u;
        const float* seg = base + st * F::STAGE + fq * F::FACE_SEG;
        // ---- gather: rows (k, b), b = 0..3, columns of group q; the r side's tiles are zero on
        // boundary faces
        float2 acc[NG][5];
#pragma unroll
        for (int b = 0; b < NG; ++b)
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[b][c] = make_float2(0.f, 0.f);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                float T[TS];
                load_tile(seg + TS * tile_pos(2 * s + h, q), T);
#pragma unroll
                for (int b = 0; b < NG; ++b) {
                    const float2* vr = reinterpret_cast<const float2*>(seg + F::XOFF + s * F::XR + (4 * k + b) * F::NP);
                    const float2 pa = vr[h ? 3 : 0];           // n = (6,7) | (0,1)
                    const float2 pb = vr[h ? 4 : 1];           // n = (8,9) | (2,3)
                    const float2 m2 = vr[2];                   // n = (4,5)
                    const float sg = h ? m2.y : m2.x;
#pragma unroll
                    for (int c = 0; c < 5; ++c) {
                        acc[b][c] = ffma2(make_float2(T[2 * c], T[2 * c + 1]), pa, acc[b][c]);
                        acc[b][c] = ffma2(make_float2(T[10 + 2 * c], T[11 + 2 * c]), pb, acc[b][c]);
                        acc[b][c].x = fmaf(T[20 + c], sg, acc[b][c].x);
                    }
                }
            }
        }
        // ---- t = E_j : g with the partner lane (1-k, q^2); h = scale S t in registers
        const bool diag = k == (q >> 1);
        const float al = diag ? 2.f * mu + lam : mu, be = diag ? lam : mu;
        float tv[NG][5];
#pragma unroll
        for (int b = 0; b < NG; ++b)
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const float gv = acc[b][c].x + acc[b][c].y;
                const float gp = __shfl_xor_sync(FULL, gv, 6);
                tv[b][c] = al * gv + be * gp;
            }
        float2 hp[NG][5];   // (h, h) pairs for the packed scatter products, slot i = time node i ^ qs
#pragma unroll
        for (int i = 0; i < NG; ++i)
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                float hv = 0.f;
#pragma unroll
                for (int b2 = 0; b2 < NG; ++b2) hv = fmaf(Sm[i][b2], tv[b2][c], hv);
                hp[i][c] = make_float2(hv, hv);
            }
        // ---- scatter: partial sums over this lane's columns for each row group Rg, reduced
        // over the four column lanes of the face
#pragma unroll
        for (int Rg = 0; Rg < 4; ++Rg) {
            float T[TS];
            load_tile(seg + TS * tile_pos(Rg, q), T);
            float R[NG][5];   // per slot (time node i ^ qs): row pair A, row pair B, single row
#pragma unroll
            for (int b = 0; b < NG; ++b) {
                float2 oA = make_float2(0.f, 0.f), oB = oA;
                float oS = 0.f;
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    oA = ffma2(make_float2(T[2 * c], T[2 * c + 1]), hp[b][c], oA);
                    oB = ffma2(make_float2(T[10 + 2 * c], T[11 + 2 * c]), hp[b][c], oB);
                    oS = fmaf(T[20 + c], hp[b][c].x, oS);
                }
                R[b][0] = oA.x; R[b][1] = oA.y; R[b][2] = oB.x; R[b][3] = oB.y; R[b][4] = oS;
            }
            // step 1 (lane q^1): its slots 2,3 hold this lane's slots 0,1 (time nodes qs, qs^1);
            // step 2 (lane q^2): its slot 1 holds this lane's slot 0 (time node qs)
            float K[2][5];
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int v = 0; v < 5; ++v) K[j][v] = R[j][v] + __shfl_xor_sync(FULL, R[2 + j][v], 1);
            float Y[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) Y[v] = K[0][v] + __shfl_xor_sync(FULL, K[1][v], 2);
            const int es = (Rg >> 1) == 0 ? el : er, odd = Rg & 1, b = qs;
            if (es >= 0) {
                float* yr = y + (int64_t)es * NVS + (4 * k + b) * F::NP + 5 * odd;
                // row pairs (1,2),(3,4) | 0 for odd groups, (0,1),(2,3) | 4 for even: 8-byte aligned
                red_add2(yr + odd, Y[0], Y[1]);
                red_add2(yr + 2 + odd, Y[2], Y[3]);
                red_add1(yr + (odd ? 0 : 4), Y[4]);
            }
        }
        __syncwarp();   // stage st is free for the next group
        st ^= 1;
        el = el_n; er = er_n; lam = lam_n; mu = mu_n;
#pragma unroll
        for (int i = 0; i < FPW; ++i) { idl[i] = nidl[i]; idr[i] = nidr[i]; }
    }
}

// ---------------------------------------------------------------------------------
// Tiled single-shot FP32 kernel for 3D, p = 2 (d = 3, N_phi = 10, N_gamma = 3).  Per face the
// gather is 9 x 30 x 20 (rows (k,b), columns (l,m), contraction (s,n)) and the scatter
// 9 x 20 x 30.  Three faces per warp, nine lanes each (lanes 27..31 idle); lane (k, l) owns
// the three time-node rows (k, b) and the ten columns (l, m):
//   gather:  g[k][l][b][m] over the full (s, n) contraction, tiles (Rg, l), Rg = 0..3;
//   E : g :  off-diagonal lanes take g[l][k] from the transposed lane, diagonal lanes the two
//            other diagonal blocks (the trace): two shuffles per value;
//   S t   :  in registers, slot j = time node (l + j) % 3 (the lane's own rows of S);
//   scatter: partial sums over the lane's ten columns with the same tiles, reduced over the
//            three l-lanes of its k in two shuffle rounds (round r reads slot 3 - r of lane
//            l + r), so that each lane ends with time node l of every row group.
// D~ per face: 12 tiles of 5 rows (s, n) x 10 columns m of one l, 52 floats each (two of
// padding), rows paired as in the 2D tiled kernel; tile (Rg, l) at position 3Rg + l (13
// 16-byte chunks apart: the three tiles a face's lanes read lie in distinct banks).  The
// element rows (90 values, 360 bytes: not a 16-byte multiple) are copied by the lanes in
// 8-byte cp.async pieces; the tiles by cp.async.bulk on the warp's mbarrier.
// ---------------------------------------------------------------------------------
struct FaceTile3 {
    static constexpr int NP = 10, NG = 3, NVS = 3 * NG * NP;   // 90 values per element
    static constexpr int TS = 52;                    // floats per 5 x 10 tile
    static constexpr int DT = 12 * TS;               // 624 floats per face
    static constexpr int XOFF = DT, XR = NVS;
    static constexpr int FPW = 3;                    // faces per warp
    static constexpr int FACE_SEG = 816;             // 204 x 16 bytes: faces 4 bank groups apart
    static constexpr int STAGE = FPW * FACE_SEG;
    static constexpr int PER_WARP = 2 * STAGE;
    static_assert(XOFF + 2 * XR <= FACE_SEG && (DT * 4) % 16 == 0, "3D tile kernel layout");
};

__host__ __device__ inline bool tile3_slot_rc(int slot, int odd, int* r, int* c) {
    if (slot < 20) { *c = slot >> 1; *r = (slot & 1) + (odd ? 1 : 0); return true; }
    if (slot < 40) { *c = (slot - 20) >> 1; *r = (slot & 1) + (odd ? 3 : 2); return true; }
    if (slot < 50) { *c = slot - 40; *r = odd ? 0 : 4; return true; }
    return false;
}

// FP64 D~ [face][s][l][n][m] -> FP32 tiles
__global__ void tile3_d32_kernel(int64_t n_face, const double* __restrict__ D, float* __restrict__ Dt) {
    using F = FaceTile3;
    const int64_t n = n_face * F::DT;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = i / F::DT;
        const int w = (int)(i % F::DT), pos = w / F::TS, slot = w % F::TS;
        const int Rg = pos / 3, l = pos % 3;
        int r, c;
        float v = 0.f;
        if (tile3_slot_rc(slot, Rg & 1, &r, &c))
            v = (float)D[f * (2 * 3 * F::NP * F::NP) + ((((Rg >> 1) * 3 + l) * F::NP) + 5 * (Rg & 1) + r) * F::NP + c];
        Dt[i] = v;
    }
}

__device__ __forceinline__ void cp_async8(float* dst, const float* src, bool on) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(on ? 8u : 0u)
                 : "memory");
}

template <int MAXREG>
__global__ void __maxnreg__(MAXREG) face_apply_tile3_kernel(int64_t n_face, const int32_t* __restrict__ fl,
                                                            const int32_t* __restrict__ fr, const float* __restrict__ Dt,
                                                            const float* __restrict__ lamf, const float* __restrict__ muf,
                                                            const RefTables* __restrict__ rtp, const float* __restrict__ x,
                                                            const int* __restrict__ xidx, int64_t ld, float* __restrict__ y,
                                                            float scale, int* __restrict__ err) {
    using F = FaceTile3;
    constexpr int TS = F::TS, NVS = F::NVS, NG = F::NG, FPW = F::FPW;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[4][2];
    if (xidx) x += (int64_t)(*xidx) * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    float* base = reinterpret_cast<float*>(smraw) + warp * F::PER_WARP;
    for (int t = lane; t < F::PER_WARP; t += 32) base[t] = 0.f;
    const uint32_t bar0 = smem_u32(&bars[warp][0]), bar1 = smem_u32(&bars[warp][1]);
    if (lane == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool active = lane < 9 * FPW;
    const int fq = active ? lane / 9 : FPW - 1, kl = active ? lane % 9 : 0, k = kl / 3, l = kl % 3;
    const int fb = fq * 9;                            // first lane of the face
    const bool diag = k == l;
    // shuffle sources: E:g (transposed lane, or the two other diagonal lanes) and the two
    // rounds of the reduce over the l-lanes
    const int src1 = active ? (diag ? fb + 4 * ((k + 1) % 3) : fb + 3 * l + k) : lane;
    const int src2 = active ? (diag ? fb + 4 * ((k + 2) % 3) : lane) : lane;
    const int srr1 = active ? fb + 3 * k + (l + 1) % 3 : lane;
    const int srr2 = active ? fb + 3 * k + (l + 2) % 3 : lane;
    float Sm[NG][NG];   // scale * S, slot j = time node (l + j) % 3
#pragma unroll
    for (int j = 0; j < NG; ++j)
#pragma unroll
        for (int b = 0; b < NG; ++b) Sm[j][b] = scale * (float)rtp->S[((l + j) % 3) * NG + b];
    const int64_t n_grp = (n_face + FPW - 1) / FPW;
    const int64_t stride = (int64_t)gridDim.x * wpb;
    constexpr long kPollLimit = 1L << 24;

    auto load_ids = [&](int64_t pp, int (&el)[FPW], int (&er)[FPW]) {
#pragma unroll
        for (int i = 0; i < FPW; ++i) {
            const int64_t f = FPW * pp + i;
            const bool ok = pp < n_grp && f < n_face;
            el[i] = ok ? fl[f] : -1;
            er[i] = ok ? fr[f] : -1;
        }
    };
    auto issue = [&](int64_t p, int st, const int (&el)[FPW], const int (&er)[FPW]) {   // every lane
        float* sg = base + st * F::STAGE;
        if (lane == 0) {
            const uint32_t bar = st ? bar1 : bar0;
            uint32_t bytes = 0;
#pragma unroll
            for (int i = 0; i < FPW; ++i)
                if (el[i] >= 0) bytes += F::DT * sizeof(float);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_expect_tx(bar, bytes);
#pragma unroll
            for (int i = 0; i < FPW; ++i)
                if (el[i] >= 0) bulk_g2s(smem_u32(sg + i * F::FACE_SEG), Dt + (FPW * p + i) * (int64_t)F::DT,
                                         F::DT * sizeof(float), bar);
        }
        // element rows: FPW faces x 2 sides x 45 pieces of 8 bytes
#pragma unroll
        for (int u = 0; u < (FPW * 2 * NVS / 2 + 31) / 32; ++u) {
            const int ci = lane + 32 * u;
            if (ci < FPW * 2 * NVS / 2) {
                const int i = ci / NVS, side = (ci % NVS) / (NVS / 2), j = ci % (NVS / 2);
                static_assert(FPW == 3, "face selection below");
                const int eli = i == 0 ? el[0] : (i == 1 ? el[1] : el[2]);   // selects, not a local array
                const int eri = i == 0 ? er[0] : (i == 1 ? er[1] : er[2]);
                const int e = side ? eri : eli;
                const bool ok = eli >= 0 && e >= 0;
                cp_async8(sg + i * F::FACE_SEG + F::XOFF + side * F::XR + 2 * j,
                          ok ? x + (int64_t)e * NVS + 2 * j : x, ok);
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto fetch = [&](int64_t pp, int& a, int& b, float& lm, float& m) {
        const int64_t ff = FPW * pp + fq;
        const bool ok = active && pp < n_grp && ff < n_face;
        a = ok ? fl[ff] : -1;
        b = ok ? fr[ff] : -1;
        lm = ok ? lamf[ff] : 0.f;
        m = ok ? muf[ff] : 0.f;
    };

    int64_t p = blockIdx.x * (int64_t)wpb + warp;
    int idl[FPW], idr[FPW];
    load_ids(p, idl, idr);
    if (p < n_grp) issue(p, 0, idl, idr);
    load_ids(p + stride, idl, idr);
    int el, er;
    float lam, mu;
    fetch(p, el, er, lam, mu);
    uint32_t ph0 = 0, ph1 = 0;
    int st = 0;
    for (; p < n_grp; p += stride) {
        const int64_t pn = p + stride;
        if (pn < n_grp) issue(pn, st ^ 1, idl, idr);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        int nidl[FPW], nidr[FPW];
        load_ids(pn + stride, nidl, nidr);
        int el_n, er_n;
        float lam_n, mu_n;
        fetch(pn, el_n, er_n, lam_n, mu_n);
        if (!__all_sync(FULL, mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0, kPollLimit))) {
            if (lane == 0) atomicExch(err, 1);
            bool drained = mbar_wait(st ? bar1 : bar0, st ? ph1 : ph0, kPollLimit);
            if (pn < n_grp) drained = mbar_wait(st ? bar0 : bar1, st ? ph0 : ph1, kPollLimit) && drained;
            if (!drained && lane == 0) atomicExch(err, 2);
            break;
        }
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncwarp();
        if (st) ph1 ^= 1u; else ph0 ^= 1u;
        const float* seg = base + st * F::STAGE + fq * F::FACE_SEG;
        // ---- gather: rows (k, b), columns (l, m), m = 0..9
        float2 acc[NG][10];
#pragma unroll
        for (int b = 0; b < NG; ++b)
#pragma unroll
            for (int c = 0; c < 10; ++c) acc[b][c] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int Rg = 0; Rg < 4; ++Rg) {   // one tile live at a time (rolled loop)
            const int s = Rg >> 1, h = Rg & 1;
            {
                float T[TS];   // the tile, read once for the three time nodes
                {
                    const float4* tp = reinterpret_cast<const float4*>(seg + TS * (3 * Rg + l));
#pragma unroll
                    for (int j = 0; j < TS / 4; ++j) {
                        const float4 q = tp[j];
                        T[4 * j] = q.x; T[4 * j + 1] = q.y; T[4 * j + 2] = q.z; T[4 * j + 3] = q.w;
                    }
                }
#pragma unroll
                for (int b = 0; b < NG; ++b) {
                    const float2* vr = reinterpret_cast<const float2*>(seg + F::XOFF + s * F::XR + (3 * k + b) * F::NP);
                    const float2 pa = vr[h ? 3 : 0], pb = vr[h ? 4 : 1], m2 = vr[2];
                    const float sg = h ? m2.y : m2.x;
#pragma unroll
                    for (int c = 0; c < 10; ++c) {
                        acc[b][c] = ffma2(make_float2(T[2 * c], T[2 * c + 1]), pa, acc[b][c]);
                        acc[b][c] = ffma2(make_float2(T[20 + 2 * c], T[21 + 2 * c]), pb, acc[b][c]);
                        acc[b][c].x = fmaf(T[40 + c], sg, acc[b][c].x);
                    }
                }
            }
        }
        // ---- t = E_j : g (two shuffles per value), h = scale S t in the lane's slot order
        float tv[NG][10];
#pragma unroll
        for (int b = 0; b < NG; ++b)
#pragma unroll
            for (int c = 0; c < 10; ++c) {
                const float gv = acc[b][c].x + acc[b][c].y;
                const float x1 = __shfl_sync(FULL, gv, src1);
                const float x2 = __shfl_sync(FULL, gv, src2);
                tv[b][c] = diag ? fmaf(2.f * mu, gv, lam * (gv + x1 + x2)) : mu * (gv + x1);
            }
        float hv[NG][10];
#pragma unroll
        for (int j = 0; j < NG; ++j)
#pragma unroll
            for (int c = 0; c < 10; ++c) {
                float a = 0.f;
#pragma unroll
                for (int b2 = 0; b2 < NG; ++b2) a = fmaf(Sm[j][b2], tv[b2][c], a);
                hv[j][c] = a;
            }
        // ---- scatter: partial sums over this lane's columns, reduced over the three l-lanes
#pragma unroll 1
        for (int Rg = 0; Rg < 4; ++Rg) {
            float T[TS];
            {
                const float4* tp = reinterpret_cast<const float4*>(seg + TS * (3 * Rg + l));
#pragma unroll
                for (int j = 0; j < TS / 4; ++j) {
                    const float4 q = tp[j];
                    T[4 * j] = q.x; T[4 * j + 1] = q.y; T[4 * j + 2] = q.z; T[4 * j + 3] = q.w;
                }
            }
            float R[NG][5];
#pragma unroll
            for (int j = 0; j < NG; ++j) {
                float2 oA = make_float2(0.f, 0.f), oB = oA;
                float oS = 0.f;
#pragma unroll
                for (int c = 0; c < 10; ++c) {
                    const float hc = hv[j][c];
                    oA = ffma2(make_float2(T[2 * c], T[2 * c + 1]), make_float2(hc, hc), oA);
                    oB = ffma2(make_float2(T[20 + 2 * c], T[21 + 2 * c]), make_float2(hc, hc), oB);
                    oS = fmaf(T[40 + c], hc, oS);
                }
                R[j][0] = oA.x; R[j][1] = oA.y; R[j][2] = oB.x; R[j][3] = oB.y; R[j][4] = oS;
            }
            float Y[5];
#pragma unroll
            for (int v = 0; v < 5; ++v)
                Y[v] = R[0][v] + __shfl_sync(FULL, R[2][v], srr1) + __shfl_sync(FULL, R[1][v], srr2);
            const int es = (Rg >> 1) == 0 ? el : er, odd = Rg & 1;
            if (es >= 0) {
                float* yr = y + (int64_t)es * NVS + (3 * k + l) * F::NP + 5 * odd;
                red_add2(yr + odd, Y[0], Y[1]);
                red_add2(yr + 2 + odd, Y[2], Y[3]);
                red_add1(yr + (odd ? 0 : 4), Y[4]);
            }
        }
        __syncwarp();   // stage st is free for the next group
        st ^= 1;
        el = el_n; er = er_n; lam = lam_n; mu = mu_n;
#pragma unroll
        for (int i = 0; i < FPW; ++i) { idl[i] = nidl[i]; idr[i] = nidr[i]; }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------------
// Multi-shot FP32 kernel for 2D, p = 2 (d = 2, N_phi = 6, N_gamma = 3): one lane per shot.
// A warp takes a face and 32 shots of a stacked vector at a time.  Each lane keeps its shot's
// two element rows (72 values) and its 72 outputs in registers; the face's D~ block is read
// from shared memory by all lanes at once, one column m at a time (24 values, each used in 12
// products).  S acts on the time nodes only and commutes with D~ and E, so it is applied to v
// first: per column m the gather g[k][l][b] = sum_(s,n) D~_s[l][n][m] v'_s[k][b][n], the stress
// map h = E_j : g and the scatter y_s[k][b][n] += sum_l D~_s[l][n][m] h[(k,l)][b] need no other
// column.  The rows of the next (face, 32 shots) item are copied by cp.async while the current
// one is computed; the outputs go back through the same shared rows so that the atomic
// additions are 16-byte vectors along one shot's element row.
// ---------------------------------------------------------------------------------
struct FaceShots {
    static constexpr int NP = 6, NG = 3, NVS = 2 * NG * NP;   // 36 values per element
    static constexpr int DFACE = 2 * 2 * NP * NP;             // 144
    static constexpr int ROW = 76;                             // 72 values + 4: 19 x 16 bytes (odd)
    static constexpr int VBUF = 32 * ROW;
    static constexpr int PER_WARP = 2 * VBUF + 2 * DFACE;
    static_assert(2 * NVS <= ROW && (ROW / 4) % 2 == 1 && (NVS * 4) % 16 == 0 && (DFACE * 4) % 16 == 0, "layout");
};

__device__ __forceinline__ void cp_async16(float* dst, const float* src, bool on) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(on ? 16u : 0u)
                 : "memory");
}
__device__ __forceinline__ void red_add4(float* y, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(y), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

__global__ void __launch_bounds__(128) face_apply_shots_kernel(int64_t n_face, const int32_t* __restrict__ fl,
                                                               const int32_t* __restrict__ fr, const float* __restrict__ D,
                                                               const float* __restrict__ lamf, const float* __restrict__ muf,
                                                               const RefTables* __restrict__ rtp, const float* __restrict__ x,
                                                               const int* __restrict__ xidx, int64_t ld,
                                                               float* __restrict__ y0, float scale, int nshots, int64_t nvec) {
    using F = FaceShots;
    constexpr int NP = F::NP, NG = F::NG, NVS = F::NVS;
    extern __shared__ __align__(16) unsigned char smraw[];
    if (xidx) x += (int64_t)(*xidx) * ld;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    float* vbuf = reinterpret_cast<float*>(smraw) + warp * F::PER_WARP;   // two buffers of 32 rows
    float* dbuf = vbuf + 2 * F::VBUF;                                      // two D~ blocks
    float Sm[NG][NG];   // scale * S
#pragma unroll
    for (int a = 0; a < NG; ++a)
#pragma unroll
        for (int b = 0; b < NG; ++b) Sm[a][b] = scale * (float)rtp->S[a * NG + b];
    const int nc = (nshots + 31) >> 5;            // 32-shot chunks
    const int64_t gw = blockIdx.x * (int64_t)wpb + warp, W = (int64_t)gridDim.x * wpb;
    const int64_t n_mine = gw < n_face ? (n_face - 1 - gw) / W + 1 : 0;
    const int64_t n_items = n_mine * nc;         // item t: face gw + (t / nc) W, chunk t % nc
    struct Info { int el, er; float lam, mu; };
    auto info = [&](int64_t t) {
        Info r{-1, -1, 0.f, 0.f};
        if (t < n_items) {
            const int64_t f = gw + (t / nc) * W;
            r.el = fl[f]; r.er = fr[f]; r.lam = lamf[f]; r.mu = muf[f];
        }
        return r;
    };
    // the 32 shots' rows of an item are 32 x 18 chunks of 16 bytes, copied in order by the warp
    // (one instruction covers 2-3 shot rows: the shots lie a whole vector apart in memory, and 32
    // of them per instruction would fall on the same memory partitions)
    constexpr int CPR = 2 * NVS / 4;   // chunks per shot row
    auto issue = [&](int64_t t, const Info& I) {   // every lane: a share of the rows, and of the D~ block
        if (t < n_items) {
            const int64_t f = gw + (t / nc) * W;
            const int c0 = (int)(t % nc) * 32;
            float* buf = vbuf + (t & 1) * F::VBUF;
#pragma unroll
            for (int u = 0; u < CPR; ++u) {
                const int ci = lane + 32 * u, sl = ci / CPR, part = ci % CPR;
                const int side = part >= NVS / 4, j = side ? part - NVS / 4 : part;
                const bool ok = c0 + sl < nshots && (side == 0 || I.er >= 0);
                const int e = side ? I.er : I.el;
                const float* src = x + (ok ? (int64_t)(c0 + sl) * nvec + (int64_t)e * NVS + 4 * j : 0);
                cp_async16(buf + sl * F::ROW + side * NVS + 4 * j, src, ok);
            }
            float* db = dbuf + (t & 1) * F::DFACE;
            const float* src = D + f * (int64_t)F::DFACE;
            for (int j = lane; j < F::DFACE / 4; j += 32) cp_async16(db + 4 * j, src + 4 * j, true);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    Info I0 = info(0), I1 = info(1);
    issue(0, I0);
    for (int64_t t = 0; t < n_items; ++t) {
        issue(t + 1, I1);
        const Info I2 = info(t + 2);
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncwarp();
        float* row = vbuf + (t & 1) * F::VBUF + lane * F::ROW;
        const float* sD = dbuf + (t & 1) * F::DFACE;
        // ---- v' = scale S v over the time nodes, rows (s, k, b), N_phi values each
        float v[2][2][NG][NP];
#pragma unroll
        for (int j = 0; j < 2 * NVS / 4; ++j) {
            const float4 q = reinterpret_cast<const float4*>(row)[j];
            const float e4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = 4 * j + u, s = e / NVS, r = e % NVS;
                v[s][r / (NG * NP)][(r / NP) % NG][r % NP] = e4[u];
            }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int n = 0; n < NP; ++n) {
                    float w[NG];
#pragma unroll
                    for (int b = 0; b < NG; ++b) {
                        float a = 0.f;
#pragma unroll
                        for (int b2 = 0; b2 < NG; ++b2) a = fmaf(Sm[b][b2], v[s][k][b2][n], a);
                        w[b] = a;
                    }
#pragma unroll
                    for (int b = 0; b < NG; ++b) v[s][k][b][n] = w[b];
                }
        const float lam = I0.lam, mu = I0.mu, dg = 2.f * mu + lam;
        float yv[2][2][NG][NP];
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int b = 0; b < NG; ++b)
#pragma unroll
                    for (int n = 0; n < NP; ++n) yv[s][k][b][n] = 0.f;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            float Dc[2][2][NP];   // D~_s[l][n][m]
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int l = 0; l < 2; ++l)
#pragma unroll
                    for (int n = 0; n < NP; ++n) Dc[s][l][n] = sD[((s * 2 + l) * NP + n) * NP + m];
            float h[3][NG];
#pragma unroll
            for (int b = 0; b < NG; ++b) {
                float g[2][2];
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int l = 0; l < 2; ++l) {
                        float a = 0.f;
#pragma unroll
                        for (int s = 0; s < 2; ++s)
#pragma unroll
                            for (int n = 0; n < NP; ++n) a = fmaf(Dc[s][l][n], v[s][k][b][n], a);
                        g[k][l] = a;
                    }
                h[0][b] = dg * g[0][0] + lam * g[1][1];
                h[1][b] = lam * g[0][0] + dg * g[1][1];
                h[2][b] = mu * (g[0][1] + g[1][0]);
            }
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int b = 0; b < NG; ++b)
#pragma unroll
                    for (int n = 0; n < NP; ++n) {
                        // k = 0: components (xx, xy) with l = 0, 1; k = 1: (xy, yy)
                        yv[s][0][b][n] = fmaf(Dc[s][0][n], h[0][b], fmaf(Dc[s][1][n], h[2][b], yv[s][0][b][n]));
                        yv[s][1][b][n] = fmaf(Dc[s][0][n], h[2][b], fmaf(Dc[s][1][n], h[1][b], yv[s][1][b][n]));
                    }
        }
        // ---- outputs back through the lane's row, then vector additions along each shot's rows
#pragma unroll
        for (int j = 0; j < 2 * NVS / 4; ++j) {
            float e4[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int e = 4 * j + u, s = e / NVS, r = e % NVS;
                e4[u] = yv[s][r / (NG * NP)][(r / NP) % NG][r % NP];
            }
            reinterpret_cast<float4*>(row)[j] = make_float4(e4[0], e4[1], e4[2], e4[3]);
        }
        __syncwarp();
        const int c0 = (int)(t % nc) * 32;
        const float* rows = vbuf + (t & 1) * F::VBUF;
        if (lane < 2 * NVS / 4) {
            const bool right = lane >= NVS / 4;
            const int es = right ? I0.er : I0.el, q = right ? lane - NVS / 4 : lane;
            if (es >= 0) {
                for (int j = 0; j < 32 && c0 + j < nshots; ++j) {
                    const float4 val = reinterpret_cast<const float4*>(rows + j * F::ROW)[lane];
                    red_add4(y0 + (int64_t)(c0 + j) * nvec + (int64_t)es * NVS + 4 * q, val);
                }
            }
        }
        __syncwarp();   // the rows and the D~ block are free for the item after next
        I0 = I1;
        I1 = I2;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int DIM, int NP, int NG, typename R>
static cudaError_t launch_fast(stdg_ctx* c, const R* D, const R* lamf, const R* muf, const R* x, const int* xidx,
                               int64_t ld, R* y, double scale, int nshots) {
    using T = FaceTma<DIM, NP, NG, R>;
    const bool aligned = (reinterpret_cast<uintptr_t>(D) % 16 == 0) && (reinterpret_cast<uintptr_t>(x) % 16 == 0) &&
                         ((ld * (int64_t)sizeof(R)) % 16 == 0);
    if constexpr (DIM == 2 && NP == 10 && NG == 4 && std::is_same<R, float>::value) {
        // the tiled kernel, on the tiled copy of D~ made with the FP32 copy
        if (nshots == 1 && aligned && c->d_err && c->d_Dt32 && D == c->d_D32 &&
            reinterpret_cast<uintptr_t>(y) % 8 == 0) {
            using TF = FaceTile;
            const int wpb = c->tune.face_wpb;   // <= 4: the kernel's launch bounds and its per-warp barriers
            const size_t smem = sizeof(float) * (size_t)wpb * TF::PER_WARP;
            const int64_t n_grp = (c->n_face + TF::FPW - 1) / TF::FPW;
            const int64_t blocks = std::min<int64_t>((n_grp + wpb - 1) / wpb, (int64_t)c->n_sm * c->tune.face_bpsm);
            auto go = [&](auto kern) {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                kern<<<(unsigned)blocks, 32 * wpb, smem, c->stream>>>(c->n_face, c->d_face_l, c->d_face_r, c->d_Dt32, lamf,
                                                                     muf, c->d_rt, x, xidx, ld, y, (float)scale, c->d_err);
            };
            // capped: the registers of 11 resident warps per SM, the most that the shared memory of
            // the bulk-copy stages admits
            if (c->tune.face_cap) go(face_apply_tile_kernel<184>);
            else go(face_apply_tile_kernel<255>);
            note_launch(c);
            return cudaGetLastError();
        }
    }
    if constexpr (DIM == 3 && NP == 10 && NG == 3 && std::is_same<R, float>::value) {
        // the 3D tiled kernel, on the tiled copy of D~ made with the FP32 copy
        if (nshots == 1 && c->d_err && c->d_Dt32 && D == c->d_D32 && reinterpret_cast<uintptr_t>(x) % 8 == 0 &&
            reinterpret_cast<uintptr_t>(y) % 8 == 0 && (ld * (int64_t)sizeof(R)) % 8 == 0) {
            using TF = FaceTile3;
            const int wpb = c->tune.face_wpb;   // <= 4: the kernel's per-warp barriers
            const size_t smem = sizeof(float) * (size_t)wpb * TF::PER_WARP;
            const int64_t n_grp = (c->n_face + TF::FPW - 1) / TF::FPW;
            const int64_t blocks = std::min<int64_t>((n_grp + wpb - 1) / wpb, (int64_t)c->n_sm * c->tune.face_bpsm);
            auto go = [&](auto kern) {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                kern<<<(unsigned)blocks, 32 * wpb, smem, c->stream>>>(c->n_face, c->d_face_l, c->d_face_r, c->d_Dt32, lamf,
                                                                     muf, c->d_rt, x, xidx, ld, y, (float)scale, c->d_err);
            };
            if (c->tune.face_cap) go(face_apply_tile3_kernel<168>);
            else go(face_apply_tile3_kernel<255>);
            note_launch(c);
            return cudaGetLastError();
        }
    }
    if (nshots == 1 && aligned && c->d_err) {
        const int wpb = c->tune.face_wpb;   // <= 4: the kernel's launch bounds and its per-warp barriers
        const size_t smem = sizeof(R) * (size_t)wpb * T::PER_WARP;
        const int64_t blocks = std::min<int64_t>((c->n_face + wpb - 1) / wpb, (int64_t)c->n_sm * c->tune.face_bpsm);
        auto go = [&](auto kern) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            kern<<<(unsigned)blocks, 32 * wpb, smem, c->stream>>>(c->n_face, c->d_face_l, c->d_face_r, D, lamf, muf,
                                                                 c->d_rt, x, xidx, ld, y, (R)scale, c->d_err);
        };
        if (c->tune.face_cap) go(face_apply_tma_kernel<DIM, NP, NG, R, T::MIN_BLOCKS>);
        else go(face_apply_tma_kernel<DIM, NP, NG, R, 1>);
        note_launch(c);
        return cudaGetLastError();
    }
    if constexpr (DIM == 2 && NP == 6 && NG == 3 && std::is_same<R, float>::value) {
        // batches of 16 shots or more: one lane per shot
        if (nshots >= 16 && (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (reinterpret_cast<uintptr_t>(D) % 16 == 0) &&
            (reinterpret_cast<uintptr_t>(y) % 16 == 0) && (ld * (int64_t)sizeof(R)) % 16 == 0 &&
            (c->nvel * (int64_t)sizeof(R)) % 16 == 0) {
            using SF = FaceShots;
            const int wpb = c->tune.face_wpb;
            const size_t smem = sizeof(float) * (size_t)wpb * SF::PER_WARP;
            const int64_t blocks = std::min<int64_t>((c->n_face + wpb - 1) / wpb, (int64_t)c->n_sm * c->tune.face_bpsm);
            cudaFuncSetAttribute(face_apply_shots_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            face_apply_shots_kernel<<<(unsigned)blocks, 32 * wpb, smem, c->stream>>>(
                c->n_face, c->d_face_l, c->d_face_r, D, lamf, muf, c->d_rt, x, xidx, ld, y, (float)scale, nshots, c->nvel);
            note_launch(c);
            return cudaGetLastError();
        }
    }
    using F = FaceReg<DIM, NP, NG, R>;
    const int wpb = c->tune.face_wpb;
    const int64_t blocks = std::min<int64_t>((c->n_face + wpb - 1) / wpb, 1 << 30);
    if (F::HALVES == 2 && nshots >= 2) {
        constexpr int H = F::HALVES;
        const size_t smem = sizeof(R) * (size_t)wpb * H * F::PER_WARP;
        cudaFuncSetAttribute(face_apply_fast_kernel<DIM, NP, NG, R, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        face_apply_fast_kernel<DIM, NP, NG, R, H><<<(unsigned)blocks, 32 * wpb, smem, c->stream>>>(
            c->n_face, c->d_face_l, c->d_face_r, D, lamf, muf, c->d_rt, x, xidx, ld, y, (R)scale, nshots, c->nvel);
    } else {
        const size_t smem = sizeof(R) * (size_t)wpb * F::PER_WARP;
        cudaFuncSetAttribute(face_apply_fast_kernel<DIM, NP, NG, R, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        face_apply_fast_kernel<DIM, NP, NG, R, 1><<<(unsigned)blocks, 32 * wpb, smem, c->stream>>>(
            c->n_face, c->d_face_l, c->d_face_r, D, lamf, muf, c->d_rt, x, xidx, ld, y, (R)scale, nshots, c->nvel);
    }
    note_launch(c);
    return cudaGetLastError();
}

// FP32 tiles of D~ for the tiled (2,10,4) kernel; false for other shapes
static bool tiled2(const stdg_ctx* c) { return c->dim == 2 && c->Nphi == 10 && c->Ng == 4; }
static bool tiled3(const stdg_ctx* c) { return c->dim == 3 && c->Nphi == 10 && c->Ng == 3; }
bool face_tiled_shape(const stdg_ctx* c) { return tiled2(c) || tiled3(c); }
int64_t face_tiled_floats(const stdg_ctx* c) {
    return tiled2(c) ? c->n_face * FaceTile::DT : tiled3(c) ? c->n_face * FaceTile3::DT : 0;
}
cudaError_t launch_tile_d32(stdg_ctx* c) {
    if (tiled2(c)) tile_d32_kernel<<<(unsigned)(c->n_sm * 8), 256, 0, c->stream>>>(c->n_face, c->d_D, c->d_Dt32);
    else tile3_d32_kernel<<<(unsigned)(c->n_sm * 8), 256, 0, c->stream>>>(c->n_face, c->d_D, c->d_Dt32);
    note_launch(c);
    return cudaGetLastError();
}

// Specialised shapes: (2,10,4) space-time p = 3 in 2D, (2,6,3) p = 2 in 2D, (3,10,3) p = 2 in
// 3D, (2,3,1) Crank-Nicolson p = 1 in 2D.  Returns false when no specialisation exists.
template <typename R>
bool launch_face_fast(stdg_ctx* c, const R* D, const R* lamf, const R* muf, const R* x, const int* xidx, int64_t ld, R* y,
                      double scale, cudaError_t* err, int nshots) {
    const int d = c->dim, np = c->Nphi, ng = c->Ng;
    // FP64 stays on the shared-memory kernel: at 1/64 of the FP32 rate the FP64 pipe, not
    // issue, bounds it, and the register-blocked variant's occupancy is lower.
    if (sizeof(R) == 8) return false;
    if (d == 2 && np == 10 && ng == 4) { *err = launch_fast<2, 10, 4, R>(c, D, lamf, muf, x, xidx, ld, y, scale, nshots); return true; }
    if (d == 2 && np == 6 && ng == 3) { *err = launch_fast<2, 6, 3, R>(c, D, lamf, muf, x, xidx, ld, y, scale, nshots); return true; }
    if (d == 3 && np == 10 && ng == 3) { *err = launch_fast<3, 10, 3, R>(c, D, lamf, muf, x, xidx, ld, y, scale, nshots); return true; }
    if (d == 2 && np == 3 && ng == 1) { *err = launch_fast<2, 3, 1, R>(c, D, lamf, muf, x, xidx, ld, y, scale, nshots); return true; }
    return false;
}

template bool launch_face_fast<float>(stdg_ctx*, const float*, const float*, const float*, const float*, const int*, int64_t,
                                      float*, double, cudaError_t*, int);
template bool launch_face_fast<double>(stdg_ctx*, const double*, const double*, const double*, const double*, const int*,
                                       int64_t, double*, double, cudaError_t*, int);

}  // namespace stdg
