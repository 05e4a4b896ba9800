// Element-local step of the stencil preconditioner "Pre2" (Appendix A, Eqs. APPRE1 -
// APPRE2) for a batch of shots, on the 5th-generation tensor cores (tcgen05, TMEM
// accumulators).  For every element e and every shot s of the stacked vectors
//   z_e,s = S_e^{-1} (2 r_e,s - w_e,s)          (w = A P_1 r, see precond2.cu)
// which, for a batch of shots, is the dense product Z_e = S_e^{-1} T_e with T_e = [t_e,s]
// of N x n_shots values: a real GEMM once the shots are many.  It is evaluated transposed,
// D = A B with
//   A = T^T  (rows: shots, K: the N entries of t_e,s -- the shot-major vectors as they lie),
//   B = S_e^{-T} (K: columns c of S_e^{-1}, N_mma: its rows r),
//   D = Z^T  (TMEM lane = shot, column = r), written back to the shot-major z.
// Each element's product is its own MMA chain with M = 64 (up to 64 shots per group), N = the
// rows of S^{-1} rounded up to 8, K = N (in steps of 8): for M = 64 the accumulator row r lies in
// TMEM lane 32 (r / 16) + r % 16 (lanes 16..31 of each 32-lane sub-partition stay unused, as
// measured on the GPU).  A CTA handles two consecutive elements per iteration (their S^{-1}
// images are adjacent, one bulk copy), their accumulators in TMEM columns 0.. and 64..; each
// thread stages the r and w rows of its (element, shot) for the next iteration with cp.async
// while the current iteration's MMAs and epilogue run.  The kernel is bound by HBM (the
// vectors of all shots plus one S^{-1} block per element), which is read once for all shots
// instead of once per small group of shots.
//
// Precision (kind::tf32, FP32 accumulation): S^{-1} is stored rounded to TF32 (a fixed,
// linear perturbation of the preconditioner of relative size 2^-11, like any change of
// preconditioner), while t is split into t_hi = tf32(t) and t_lo = t - t_hi and both are
// multiplied (two MMAs per K step), so the map t -> z stays linear to FP32 rounding as
// right-preconditioned GMRES requires.
//
// Shared-memory operands use the canonical K-major layout without swizzling: 8-row x
// 16-byte core matrices (8 rows x 4 FP32), described to the MMA by the byte distance of
// K-adjacent cores (LBO) and of M/N-adjacent cores (SBO).  S^{-1} is pre-tiled in global
// memory as that image (S_img, one per element, KC x NI cores, K-core major), so one bulk
// copy (cp.async.bulk, mbarrier completion) per element pair lands it ready for the MMA.
//
// Every wait (bulk copy, MMA completion) is bounded; on timeout the kernel records the error,
// drains what it issued (bounded too) and frees its TMEM columns before it returns.
#include <algorithm>
#include <cstdint>

#include "stdg_internal.h"
#include "tma.h"

namespace stdg {

namespace {

template <int N>
struct MmaShape {
    static_assert(N % 4 == 0, "element block order must be a multiple of 4");
    static constexpr int NI = (N + 7) / 8;              // row cores of S^{-T} (MMA N side)
    static constexpr int KC = N / 4;                    // K cores per element
    static constexpr int KCP = (KC + 1) / 2 * 2;        // ... rounded up to whole K steps (8 = 2 cores)
    static constexpr int IMG = KC * NI * 32;            // floats per element image
    static constexpr int NMMA = NI * 8;                 // MMA N (multiple of 8 for M = 64)
    static constexpr int M = 64, MI = 8;                // MMA rows: up to 64 shots of one element
    static constexpr int A_BYTES = KCP * MI * 128;      // one A operand of one element (K-core major)
    // two images; an element's last K step may read one K-core column past the pair's images
    static constexpr int B_BYTES = 2 * IMG * 4 + NI * 128 * (KCP - KC) + 16;
    static constexpr int DCOL = 64;                     // TMEM column offset of the second element
    static constexpr int TMEM_COLS = 128;
    // staging of one item's vectors, per shot row: r of both elements, then w of both (4N floats
    // + 4 of padding: rows 16-byte aligned and spread over the banks)
    static constexpr int ROW = 4 * N + 4;
    static constexpr int STAGE = 64 * ROW * 4;
    static constexpr int ZROW = 2 * N + 4;              // z staging row (both elements), in the A area
    static constexpr int SMEM = 4 * A_BYTES + 2 * B_BYTES + STAGE;   // A_hi, A_lo of two elements; two B stages
    static_assert(64 * ZROW * 4 <= 4 * A_BYTES, "z staging fits in the A operands");
    static_assert(NMMA <= 64 && NMMA % 8 == 0, "MMA N");
    static_assert((ROW * 4) % 16 == 0 && (ZROW * 4) % 16 == 0, "staging rows of whole 16-byte chunks");
    static_assert(((long)MI * 128 / 16) < (1 << 14) && (NI * 128 / 16) < (1 << 14), "descriptor offsets");
};

// shared-memory matrix descriptor: K-major, no swizzle (sm_100 descriptor version 1)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// 32 consecutive TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t u[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
          "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15]), "=r"(u[16]),
          "=r"(u[17]), "=r"(u[18]), "=r"(u[19]), "=r"(u[20]), "=r"(u[21]), "=r"(u[22]), "=r"(u[23]), "=r"(u[24]),
          "=r"(u[25]), "=r"(u[26]), "=r"(u[27]), "=r"(u[28]), "=r"(u[29]), "=r"(u[30]), "=r"(u[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(u[i]);
}
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t u[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3])
                 : "r"(taddr)
                 : "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(u[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

constexpr long kPoll = 1L << 24;

// 16-byte asynchronous global -> shared copy (L2 only), zero-filled when `bytes` is 0
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

}  // namespace

// S^{-1} (column-major FP32, blocks `stride` floats apart) -> the MMA image: per element,
// core (kc, ni) at float offset (kc * NI + ni) * 32 holds S^{-1}[8 ni + i][4 kc + j] at
// i * 4 + j (rows beyond N zero), rounded to TF32.
template <int N>
__global__ void pre2_mma_image_kernel(int64_t n_elem, const float* __restrict__ sinv, int64_t stride,
                                      float* __restrict__ img) {
    using Sh = MmaShape<N>;
    const int64_t total = n_elem * (int64_t)Sh::IMG;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = q / Sh::IMG;
        const int o = (int)(q % Sh::IMG);
        const int core = o / 32, within = o % 32;
        const int kc = core / Sh::NI, ni = core % Sh::NI;
        const int row = ni * 8 + within / 4, col = kc * 4 + within % 4;
        img[q] = row < N ? tf32_round(sinv[e * stride + (int64_t)col * N + row]) : 0.0f;
    }
}

template <int N>
__global__ void __launch_bounds__(128, 2) pre2_local_mma_kernel(int64_t n_elem, const float* __restrict__ img,
                                                                const float* __restrict__ r, const int* __restrict__ ridx,
                                                                int64_t ld, const float* __restrict__ w,
                                                                float* __restrict__ z, int nshots, int64_t nvec,
                                                                int* __restrict__ err) {
    using Sh = MmaShape<N>;
    constexpr int NI = Sh::NI, KC = Sh::KC, KCP = Sh::KCP, IMG = Sh::IMG, MI = Sh::MI;
    constexpr uint32_t LBO_A = MI * 128, SBO_A = 128, LBO_B = NI * 128, SBO_B = 128;
    constexpr uint32_t IDESC = idesc_tf32(Sh::M, Sh::NMMA);
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bars[3];      // B stage 0, B stage 1, MMA done
    __shared__ uint32_t tmem_slot;
    if (ridx) r += (int64_t)(*ridx) * ld;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // A operands: [element 0 hi, element 0 lo, element 1 hi, element 1 lo]
    auto A_of = [&](int ek, int lo) { return smraw + (2 * ek + lo) * Sh::A_BYTES; };
    unsigned char* B0 = smraw + 4 * Sh::A_BYTES;   // stage 0; stage 1 follows at + B_BYTES
    // zero the A operands and both B stages (the slack past the images stays zero)
    for (int i = tid; i < Sh::SMEM / 16; i += blockDim.x) reinterpret_cast<float4*>(smraw)[i] = make_float4(0, 0, 0, 0);
    const uint32_t bar_b0 = smem_u32(&bars[0]), bar_b1 = smem_u32(&bars[1]), bar_m = smem_u32(&bars[2]);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)Sh::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(bar_b0, 1);
        mbar_init(bar_b1, 1);
        mbar_init(bar_m, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_slot;

    const int64_t npairs = (n_elem + 1) / 2;
    const int ngroups = (nshots + 63) / 64;
    auto issue_b = [&](int64_t pair, int st) {   // thread 0: both elements' images of a pair
        const int64_t e0 = 2 * pair;
        const uint32_t bytes = (uint32_t)((e0 + 1 < n_elem ? 2 : 1) * IMG * 4);
        const uint32_t bar = st ? bar_b1 : bar_b0;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, bytes);
        bulk_g2s(smem_u32(B0 + st * Sh::B_BYTES), img + e0 * IMG, bytes, bar);
    };
    // the row of A this thread fills: element ek of the pair, shot slot sl of the group
    const int ek = tid >> 6, sl = tid & 63;
    // per stage: phase bit (bit 0 / bit 1 of ph_b) and whether a copy is in flight (pend_b)
    uint32_t ph_b = 0, pend_b = 0, ph_m = 0;
    bool ok = true, mma_pending = false;
    int st = 0;
    int64_t pair = blockIdx.x;
    if (pair < npairs) {
        if (tid == 0) issue_b(pair, 0);
        pend_b = 1u;
    }
    // The vectors of an item -- for each of up to 64 shots, the 2 x N contiguous values of the
    // pair's two elements in r and in w -- are copied with cp.async into the staging rows,
    // warp-coalesced (consecutive threads take consecutive 16-byte chunks of a row), one item
    // ahead: the copies of the next item overlap the MMA and the epilogue of the current one.
    float* stage = reinterpret_cast<float*>(B0 + 2 * Sh::B_BYTES);
    constexpr int CH = 2 * N / 4;                       // 16-byte chunks per row and vector
    auto prefetch = [&](int64_t pp, int g) {
        const int64_t e0 = 2 * pp;
        const int nch = pp < npairs ? (e0 + 1 < n_elem ? CH : CH / 2) : 0;   // valid chunks of a row
        for (int c = tid; c < 64 * 2 * CH; c += blockDim.x) {
            const int row = c / (2 * CH), q = c % (2 * CH), vec = q / CH, part = q % CH;
            const int s = g * 64 + row;
            const bool valid = part < nch && s < nshots;
            const float* src = valid ? (vec ? w : r) + (int64_t)s * nvec + e0 * N + 4 * part : r;
            cp_async16(smem_u32(stage + row * Sh::ROW + vec * 2 * N + 4 * part), src, valid ? 16u : 0u);
        }
        cp_async_commit();
    };
    float* zst = reinterpret_cast<float*>(smraw);       // z staging, aliasing the A operands after the MMA
    prefetch(pair, 0);
    for (; pair < npairs && ok; pair += gridDim.x) {
        const int64_t nxt = pair + gridDim.x;
        if (nxt < npairs) {
            if (tid == 0) issue_b(nxt, st ^ 1);
            pend_b |= 1u << (st ^ 1);
        }
        const bool got = mbar_wait(st ? bar_b1 : bar_b0, (ph_b >> st) & 1u, kPoll);
        if (__syncthreads_and(got) == 0) { ok = false; break; }
        ph_b ^= 1u << st;
        pend_b &= ~(1u << st);
        for (int g = 0; g < ngroups; ++g) {
            cp_async_wait_all();
            __syncthreads();   // every thread's copies of this item have landed
            // ---- A: t = 2 r - w of (element ek, shot sl), split hi / lo, into row sl of its operands
            {
                const float4* rr = reinterpret_cast<const float4*>(stage + sl * Sh::ROW + ek * N);
                const float4* wr = reinterpret_cast<const float4*>(stage + sl * Sh::ROW + 2 * N + ek * N);
                const uint32_t row_off = (uint32_t)((sl >> 3) * 128 + (sl & 7) * 16);
#pragma unroll
                for (int k = 0; k < KC; ++k) {
                    const float4 a = rr[k], b = wr[k];
                    const float4 t = make_float4(2.f * a.x - b.x, 2.f * a.y - b.y, 2.f * a.z - b.z, 2.f * a.w - b.w);
                    const float4 hi = make_float4(tf32_round(t.x), tf32_round(t.y), tf32_round(t.z), tf32_round(t.w));
                    const float4 lo = make_float4(t.x - hi.x, t.y - hi.y, t.z - hi.z, t.w - hi.w);
                    const uint32_t off = (uint32_t)k * LBO_A + row_off;
                    *reinterpret_cast<float4*>(A_of(ek, 0) + off) = hi;
                    *reinterpret_cast<float4*>(A_of(ek, 1) + off) = lo;
                }
#pragma unroll
                for (int k = KC; k < KCP; ++k) {   // the padding K-core (the z staging used this area)
                    const uint32_t off = (uint32_t)k * LBO_A + row_off;
                    *reinterpret_cast<float4*>(A_of(ek, 0) + off) = make_float4(0, 0, 0, 0);
                    *reinterpret_cast<float4*>(A_of(ek, 1) + off) = make_float4(0, 0, 0, 0);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before();
            __syncthreads();   // A complete; the staging rows are free for the next item
            if (g + 1 < ngroups) prefetch(pair, g + 1);
            else prefetch(pair + gridDim.x, 0);
            // ---- MMA per element: D_k = A_hi B_k + A_lo B_k over KCP / 2 K-steps of 2 cores
            if (tid == 0) {
                fence_after();
                const uint32_t bb = smem_u32(B0 + st * Sh::B_BYTES);
#pragma unroll 1
                for (int k2 = 0; k2 < 2; ++k2) {
                    const uint32_t ah = smem_u32(A_of(k2, 0)), al = smem_u32(A_of(k2, 1));
                    const uint32_t dt = tmem + (uint32_t)(k2 * Sh::DCOL);
#pragma unroll 1
                    for (int k = 0; k < KCP / 2; ++k) {
                        const uint64_t db = smem_desc(bb + (k2 * KC + 2 * k) * LBO_B, LBO_B, SBO_B);
                        mma_tf32(dt, smem_desc(ah + 2 * k * LBO_A, LBO_A, SBO_A), db, IDESC, k > 0);
                        mma_tf32(dt, smem_desc(al + 2 * k * LBO_A, LBO_A, SBO_A), db, IDESC, 1);
                    }
                }
                mma_commit(bar_m);
            }
            const bool done = mbar_wait(bar_m, ph_m, kPoll);
            if (__syncthreads_and(done) == 0) { ok = false; mma_pending = true; break; }
            ph_m ^= 1u;
            fence_after();
            // ---- epilogue: lane 32 w + t (t < 16) of the accumulators holds shot 16 w + t of the
            // group; both elements' rows (TMEM columns 0.. and 64..) go to the z staging rows ...
            {
                const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
                float* zr = zst + (warp * 16 + (lane & 15)) * Sh::ZROW;
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2) {
                    static_assert(N <= 36, "epilogue loads 32 + 4 columns");
                    float v[36];
                    tmem_ld32(tl + k2 * Sh::DCOL, v);
                    if constexpr (N > 32) {
                        float v4[4];
                        tmem_ld4(tl + k2 * Sh::DCOL + 32, v4);
                        tmem_wait_ld();
#pragma unroll
                        for (int i = 0; i < 4; ++i) v[32 + i] = v4[i];
                    } else {
                        tmem_wait_ld();
                    }
                    if (lane < 16) {
#pragma unroll
                        for (int q = 0; q < N / 4; ++q)
                            reinterpret_cast<float4*>(zr + k2 * N)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                }
            }
            __syncthreads();
            // ... and from there to z, warp-coalesced (2 N contiguous values per shot row)
            {
                const int64_t e0 = 2 * pair;
                const int nch = e0 + 1 < n_elem ? CH : CH / 2;
                for (int c = tid; c < 64 * CH; c += blockDim.x) {
                    const int row = c / CH, part = c % CH;
                    const int s = g * 64 + row;
                    if (part < nch && s < nshots)
                        *reinterpret_cast<float4*>(z + (int64_t)s * nvec + e0 * N + 4 * part) =
                            *reinterpret_cast<const float4*>(zst + row * Sh::ZROW + 4 * part);
                }
            }
            fence_before();
            __syncthreads();   // TMEM and the A area are free for the next group
        }
        st ^= 1;
    }
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
        // drain: the MMA committed last and the bulk copies still in flight (bounded)
        bool drained = true;
        if (tid == 0) {
            if (pend_b & 1u) drained = mbar_wait(bar_b0, ph_b & 1u, kPoll) && drained;
            if (pend_b & 2u) drained = mbar_wait(bar_b1, (ph_b >> 1) & 1u, kPoll) && drained;
            if (mma_pending) drained = mbar_wait(bar_m, ph_m, kPoll) && drained;
            if (!drained) atomicExch(err, 2);
        }
    }
    cp_async_wait_all();   // no copy into shared memory outlives the CTA
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Sh::TMEM_COLS)
                     : "memory");
    }
}

bool pre2_mma_supported(const stdg_ctx* c) { return c->dim * c->Nphi * c->Ng == 36; }

int64_t pre2_mma_image_floats(const stdg_ctx* c) { return c->n_elem * (int64_t)MmaShape<36>::IMG; }

cudaError_t launch_pre2_mma_image(stdg_ctx* c) {
    if (!pre2_mma_supported(c) || !c->d_pre2_mma || !c->d_pre2_32) return cudaErrorInvalidValue;
    pre2_mma_image_kernel<36><<<c->n_sm * 8, 256, 0, c->stream>>>(c->n_elem, c->d_pre2_32, pre2_stride32(c), c->d_pre2_mma);
    note_launch(c);
    return cudaGetLastError();
}

// false when the shape, the buffers or the alignment do not allow the tensor-core kernel
bool launch_pre2_local_mma(stdg_ctx* c, const float* r, const int* ridx, int64_t ld, const float* w, float* z,
                           int nshots, cudaError_t* e) {
    using Sh = MmaShape<36>;
    if (!pre2_mma_supported(c) || !c->d_pre2_mma || nshots < 2 || !c->d_err) return false;
    const bool aligned = (reinterpret_cast<uintptr_t>(r) % 16 == 0) && (reinterpret_cast<uintptr_t>(w) % 16 == 0) &&
                         (reinterpret_cast<uintptr_t>(z) % 16 == 0) && (ld % 4 == 0) && (c->nvel % 4 == 0);
    if (!aligned) return false;
    cudaFuncSetAttribute(pre2_local_mma_kernel<36>, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
    const int64_t npairs = (c->n_elem + 1) / 2;
    const int64_t grid = std::min<int64_t>(npairs, (int64_t)c->n_sm * c->tune.mma_cps);
    pre2_local_mma_kernel<36><<<(unsigned)grid, 128, Sh::SMEM, c->stream>>>(c->n_elem, c->d_pre2_mma, r, ridx, ld, w, z,
                                                                           nshots, c->nvel, c->d_err);
    note_launch(c);
    *e = cudaGetLastError();
    return true;
}

}  // namespace stdg
