// C ABI of the library (declared in include/stdg.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "stdg_internal.h"

namespace stdg {
void solver_invalidate_graph(stdg_ctx* c);
double* solver_dparams(stdg_ctx* c);

int dev_alloc(stdg_ctx* c, void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? STDG_ENOMEM : STDG_ECUDA;
    }
    c->allocs.push_back(*p);
    c->alloc_bytes.push_back(bytes);
    c->bytes += bytes;
    return STDG_OK;
}

void dev_release(stdg_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) {
        const size_t k = (size_t)(it - c->allocs.begin());
        c->bytes -= c->alloc_bytes[k];
        c->allocs.erase(it);
        c->alloc_bytes.erase(c->alloc_bytes.begin() + (int64_t)k);
    }
    cudaFree(p);
}

static void dev_free(stdg_ctx* c, void* p) { dev_release(c, p); }

void dev_free_all(stdg_ctx* c) {
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    c->alloc_bytes.clear();
    c->bytes = 0;
}

static bool all_finite(const double* a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

// phi_k at a point given in the element's frame (host evaluation for sources/receivers)
static void eval_phi_host(const stdg_ctx* c, int64_t e, const double* x, double* phi) {
    const int d = c->dim, NP = c->Nphi, nv = d + 1;
    double xi[3] = {0, 0, 0};
    for (int r = 0; r < d; ++r)
        for (int a = 0; a < d; ++a) xi[r] += c->hm.Jinv[(e * d + r) * d + a] * (x[a] - c->hm.X[(e * nv) * d + a]);
    double mono[kMaxNP];
    for (int a = 0; a < NP; ++a) {
        double v = 1.0;
        for (int r = 0; r < d; ++r)
            for (int q = 0; q < c->rt.exps[a][r]; ++q) v *= xi[r];
        mono[a] = v;
    }
    for (int k = 0; k < NP; ++k) {
        double v = 0;
        for (int a = 0; a < NP; ++a) v += c->rt.coef[a * NP + k] * mono[a];
        phi[k] = v;
    }
}

// phi(x_s) and grad phi(x_s) (physical coordinates, [NP][dim]) for source q, the source's
// element held fixed (host; for the source-term gradient of the misfit)
void source_basis_host(const stdg_ctx* c, int64_t q, double* phi, double* dphi) {
    const int d = c->dim, NP = c->Nphi, nv = d + 1;
    double y[3];
    const int64_t e = c->src_elem[q];
    locate_point(c->hm, c->src_xs.data() + q * d, y);
    double xi[3] = {0, 0, 0};
    for (int r = 0; r < d; ++r)
        for (int a = 0; a < d; ++a) xi[r] += c->hm.Jinv[(e * d + r) * d + a] * (y[a] - c->hm.X[(e * nv) * d + a]);
    for (int k = 0; k < NP; ++k) {
        phi[k] = 0.0;
        for (int m = 0; m < d; ++m) dphi[k * d + m] = 0.0;
    }
    for (int a = 0; a < NP; ++a) {
        double v = 1.0, g[3];
        for (int r = 0; r < d; ++r)
            for (int t = 0; t < c->rt.exps[a][r]; ++t) v *= xi[r];
        for (int r = 0; r < d; ++r) {   // d xi^a / d xi_r
            const int er = c->rt.exps[a][r];
            double w = er == 0 ? 0.0 : (double)er;
            for (int s2 = 0; s2 < d; ++s2)
                for (int t = 0; t < c->rt.exps[a][s2] - (s2 == r ? 1 : 0); ++t) w *= xi[s2];
            g[r] = w;
        }
        for (int k = 0; k < NP; ++k) {
            const double ck = c->rt.coef[a * NP + k];
            phi[k] += ck * v;
            for (int m = 0; m < d; ++m) {   // d/dx_m = sum_r d/dxi_r Jinv[r][m]
                double s = 0.0;
                for (int r = 0; r < d; ++r) s += g[r] * c->hm.Jinv[(e * d + r) * d + m];
                dphi[k * d + m] += ck * s;
            }
        }
    }
}

static int alloc_state(stdg_ctx* c, int n_shots) {
    dev_free(c, c->d_vtr);
    dev_free(c, c->d_sigtr);
    dev_free(c, c->d_energy);
    c->d_vtr = c->d_sigtr = c->d_energy = nullptr;
    int rc;
    if ((rc = dev_alloc(c, (void**)&c->d_vtr, sizeof(double) * c->ntr * n_shots)) != STDG_OK) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_sigtr, sizeof(double) * c->nsig * n_shots)) != STDG_OK) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_energy, sizeof(double) * std::max(1, n_shots))) != STDG_OK) return rc;
    STDG_CUDA(c, cudaMemsetAsync(c->d_vtr, 0, sizeof(double) * c->ntr * n_shots, c->stream));
    STDG_CUDA(c, cudaMemsetAsync(c->d_sigtr, 0, sizeof(double) * c->nsig * n_shots, c->stream));
    if (c->opt.preconditioner == 2) {   // stencil preconditioner scratch: two stacked vectors
        dev_free(c, c->d_p2y);
        dev_free(c, c->d_p2t);
        c->d_p2y = c->d_p2t = nullptr;
        if ((rc = dev_alloc(c, &c->d_p2y, sizeof(double) * c->nvel * n_shots)) != STDG_OK) return rc;
        if ((rc = dev_alloc(c, &c->d_p2t, sizeof(double) * c->nvel * n_shots)) != STDG_OK) return rc;
    }
    // the receiver records are laid out per shot: start them over for the new shot count
    dev_free(c, c->d_records);
    c->d_records = nullptr;
    c->rec_cap_steps = 0;
    c->n_shots = n_shots;
    c->rec_steps = 0;
    solver_invalidate_graph(c);
    return solver_setup(c);   // stacked Krylov workspace sized for n_shots
}

static int ensure_fp32(stdg_ctx* c) {
    if (c->d_D32) return STDG_OK;
    int rc;
    const int64_t nD = c->n_face * 2 * c->dim * c->Nphi * c->Nphi;
    if ((rc = dev_alloc(c, (void**)&c->d_D32, sizeof(float) * nD)) != STDG_OK) return rc;
    STDG_CUDA(c, launch_to_fp32(c));
    if (face_tiled_shape(c)) {   // the single-shot face kernel of this shape reads D~ in tiles
        if ((rc = dev_alloc(c, (void**)&c->d_Dt32, sizeof(float) * face_tiled_floats(c))) != STDG_OK) return rc;
        STDG_CUDA(c, launch_tile_d32(c));
    }
    return STDG_OK;
}

static int upload_material32(stdg_ctx* c) {
    if (!c->have_material || !c->d_D32) return STDG_OK;
    std::vector<float> lf(c->n_face), mf(c->n_face), rj(c->n_elem);
    std::vector<double> l(c->n_face), m(c->n_face), r(c->n_elem);
    STDG_CUDA(c, cudaMemcpy(l.data(), c->d_lamf, sizeof(double) * c->n_face, cudaMemcpyDeviceToHost));
    STDG_CUDA(c, cudaMemcpy(m.data(), c->d_muf, sizeof(double) * c->n_face, cudaMemcpyDeviceToHost));
    STDG_CUDA(c, cudaMemcpy(r.data(), c->d_rhoJ, sizeof(double) * c->n_elem, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < c->n_face; ++i) { lf[i] = (float)l[i]; mf[i] = (float)m[i]; }
    for (int64_t i = 0; i < c->n_elem; ++i) rj[i] = (float)r[i];
    STDG_CUDA(c, cudaMemcpy(c->d_lamf32, lf.data(), sizeof(float) * c->n_face, cudaMemcpyHostToDevice));
    STDG_CUDA(c, cudaMemcpy(c->d_muf32, mf.data(), sizeof(float) * c->n_face, cudaMemcpyHostToDevice));
    STDG_CUDA(c, cudaMemcpy(c->d_rhoJ32, rj.data(), sizeof(float) * c->n_elem, cudaMemcpyHostToDevice));
    return STDG_OK;
}

// Block-Jacobi preconditioner set-up: per-element eigen-decomposition (dt-independent).
static int setup_pre1(stdg_ctx* c) {
    const int n = c->dim * c->Nphi;
    const int64_t ne = c->n_elem;
    int rc;
    if (!c->d_preV) {
        if ((rc = dev_alloc(c, (void**)&c->d_preV, sizeof(double) * ne * n * n)) != STDG_OK) return rc;
        if ((rc = dev_alloc(c, (void**)&c->d_preLam, sizeof(double) * ne * n)) != STDG_OK) return rc;
        if ((rc = dev_alloc(c, (void**)&c->d_preB, sizeof(double) * ne * n * c->Ng * c->Ng)) != STDG_OK) return rc;
        if (c->opt.precision != STDG_FP64) {
            if ((rc = dev_alloc(c, (void**)&c->d_preV32, sizeof(float) * ne * n * n)) != STDG_OK) return rc;
            if ((rc = dev_alloc(c, (void**)&c->d_preB32, sizeof(float) * ne * n * c->Ng * c->Ng)) != STDG_OK) return rc;
            if (c->dim == 2 && c->Nphi == 10 && c->Ng == 4 &&   // the single-shot apply's lane order
                (rc = dev_alloc(c, (void**)&c->d_preB32t, sizeof(float) * ne * n * c->Ng * c->Ng)) != STDG_OK) return rc;
        }
    }
    double* d_Rinv = nullptr;
    int* d_status = nullptr;
    if ((rc = dev_alloc(c, (void**)&d_Rinv, sizeof(double) * c->Nphi * c->Nphi)) != STDG_OK) return rc;
    if ((rc = dev_alloc(c, (void**)&d_status, sizeof(int))) != STDG_OK) return rc;
    std::vector<double> Ri(c->Nphi * c->Nphi);
    for (int i = 0; i < c->Nphi * c->Nphi; ++i) Ri[i] = c->rt.MrefLinv[i];
    STDG_CUDA(c, cudaMemcpy(d_Rinv, Ri.data(), sizeof(double) * Ri.size(), cudaMemcpyHostToDevice));
    STDG_CUDA(c, cudaMemset(d_status, 0, sizeof(int)));
    STDG_CUDA(c, launch_pre1_setup(c, d_Rinv, c->d_elem_face, d_status));
    int status = 0;
    STDG_CUDA(c, cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, d_Rinv);
    dev_free(c, d_status);
    if (status) STDG_FAIL(c, STDG_ECUDA, "block-Jacobi eigen-decomposition did not converge");
    if (c->d_preV32) {
        const int64_t nv = ne * n * n;
        extern cudaError_t launch_cast32(stdg_ctx*, const double*, float*, int64_t);
        STDG_CUDA(c, launch_cast32(c, c->d_preV, c->d_preV32, nv));
    }
    if (c->opt.preconditioner == 2) {
        if (!pre2_supported(c)) STDG_FAIL(c, STDG_EINVAL, "stencil preconditioner: element block too large for this shape");
        const int N = c->dim * c->Nphi * c->Ng;
        const int64_t nS = ne * (int64_t)N * N;
        if (!c->d_pre2 && !c->d_pre2_32) {
            // the FP64 solver keeps FP64 blocks; the mixed path keeps only the FP32 ones its inner
            // solve applies (its FP64 refinement residual needs no preconditioner)
            if (c->opt.precision == STDG_FP64 &&
                (rc = dev_alloc(c, (void**)&c->d_pre2, sizeof(double) * nS)) != STDG_OK) return rc;
            if (c->opt.precision != STDG_FP64 &&
                (rc = dev_alloc(c, (void**)&c->d_pre2_32, sizeof(float) * ne * pre2_stride32(c))) != STDG_OK) return rc;
            // tensor-core image of the FP32 blocks for batches of shots
            if (c->opt.precision != STDG_FP64 && pre2_mma_supported(c) &&
                (rc = dev_alloc(c, (void**)&c->d_pre2_mma, sizeof(float) * pre2_mma_image_floats(c))) != STDG_OK) return rc;
            // FP16 balanced copy for one shot (the dominant stream at half the bytes)
            if (c->opt.precision != STDG_FP64 && pre2_half_supported(c)) {
                if ((rc = dev_alloc(c, &c->d_pre2_16, 2 * (size_t)ne * N * N)) != STDG_OK) return rc;
                if ((rc = dev_alloc(c, (void**)&c->d_pre2_scl, sizeof(float) * 2 * (size_t)ne * N)) != STDG_OK) return rc;
            }
            if ((rc = dev_alloc(c, (void**)&c->d_p2status, sizeof(int))) != STDG_OK) return rc;
        }
    }
    c->pre_dt = -1.0;
    return STDG_OK;
}

// Time blocks of the block-Jacobi preconditioner and, for the stencil preconditioner, the
// local Schur-complement inverses, for slab size dt (rebuilt only when dt changes).
int precond_for_dt(stdg_ctx* c, double dt) {
    if (!c->opt.preconditioner || c->pre_dt == dt) return STDG_OK;
    STDG_CUDA(c, launch_pre1_time(c, dt));
    c->pre_dt = dt;
    if (c->opt.preconditioner == 2) {
        STDG_CUDA(c, cudaMemsetAsync(c->d_p2status, 0, sizeof(int), c->stream));
        STDG_CUDA(c, launch_pre2_setup(c, dt, c->d_p2status));
        if (c->d_pre2_mma) STDG_CUDA(c, launch_pre2_mma_image(c));
        if (c->d_pre2_16) STDG_CUDA(c, launch_pre2_half(c));
        int status = 0;
        STDG_CUDA(c, cudaMemcpyAsync(&status, c->d_p2status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        STDG_CUDA(c, cudaStreamSynchronize(c->stream));
        if (status) {
            c->pre_dt = -1.0;
            STDG_FAIL(c, STDG_ECUDA, "stencil preconditioner: a local Schur complement is singular");
        }
    }
    return STDG_OK;
}

}  // namespace stdg

using namespace stdg;

namespace stdg {
int take_device_error(stdg_ctx* c) {
    c->wait_gave_up = false;
    if (!c->d_err) return STDG_OK;
    int e = 0;
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    STDG_CUDA(c, cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!e) return STDG_OK;
    STDG_CUDA(c, cudaMemset(c->d_err, 0, sizeof(int)));
    c->wait_gave_up = true;
    STDG_FAIL(c, STDG_ECUDA, e == 1 ? "a device-side wait gave up (bounded mbarrier wait); results of this call are invalid"
                                    : "a device-side wait gave up and a copy in flight could not be drained; results of "
                                      "this call are invalid");
}
}  // namespace stdg

#define CHECK_CTX(c) do { if (!(c)) return STDG_EINVAL; } while (0)
#define NEED_MESH(c) do { if (!(c)->have_mesh) STDG_FAIL(c, STDG_ESTATE, "call stdg_set_mesh first"); } while (0)
#define NEED_ALL(c) do { NEED_MESH(c); if (!(c)->have_material) STDG_FAIL(c, STDG_ESTATE, "call stdg_set_material first"); } while (0)

extern "C" {

int stdg_create(stdg_ctx** out, int dim, const stdg_options* opt, void* cuda_stream) {
    if (!out || !opt) return STDG_EINVAL;
    *out = nullptr;
    if (dim != 2 && dim != 3) return STDG_EINVAL;
    if (opt->p < 1 || opt->p > (dim == 2 ? 4 : 3)) return STDG_EINVAL;
    if (opt->p_gamma < 0 || opt->p_gamma > 4) return STDG_EINVAL;
    if (opt->scheme != STDG_SCHEME_CN && opt->scheme != STDG_SCHEME_STDG) return STDG_EINVAL;
    if (opt->scheme == STDG_SCHEME_CN && opt->p_gamma != 0) return STDG_EINVAL;
    if (opt->precision != STDG_FP64 && opt->precision != STDG_MIXED_FP32) return STDG_EINVAL;
    if (opt->preconditioner < 0 || opt->preconditioner > 2) return STDG_EINVAL;
    if (!(opt->rel_tol > 0.0) || opt->max_iters < 1) return STDG_EINVAL;
    stdg_ctx* c = new stdg_ctx();
    c->dim = dim;
    c->opt = *opt;
    if (!(c->opt.inner_tol > 0.0)) c->opt.inner_tol = 1e-4;
    if (c->opt.gmres_restart <= 0) c->opt.gmres_restart = 30;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreate(&c->stream);   // blocking: ordered with the legacy stream
        if (e != cudaSuccess) { delete c; return STDG_ECUDA; }
        c->own_stream = true;
    }
    {
        int dev = 0, nsm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
            if (c->own_stream) cudaStreamDestroy(c->stream);
            delete c;
            return STDG_ECUDA;
        }
        c->n_sm = nsm;
    }
    build_ref_tables(dim, opt->p, opt->p_gamma, &c->rt);
    c->Nphi = c->rt.Nphi;
    c->Npsi = c->rt.Npsi;
    c->Ng = c->rt.Ng;
    c->s = c->rt.s;
    if (dev_alloc(c, (void**)&c->d_rt, sizeof(RefTables)) != STDG_OK ||
        cudaMemcpy(c->d_rt, &c->rt, sizeof(RefTables), cudaMemcpyHostToDevice) != cudaSuccess) {
        stdg_destroy(c);
        return STDG_ECUDA;
    }
    if (dev_alloc(c, (void**)&c->d_err, sizeof(int)) != STDG_OK || cudaMemset(c->d_err, 0, sizeof(int)) != cudaSuccess) {
        stdg_destroy(c);
        return STDG_ECUDA;
    }
    double gl[16];
    gauss_legendre01(8, gl, gl + 8);
    if (dev_alloc(c, (void**)&c->d_gl8, sizeof(gl)) != STDG_OK ||
        cudaMemcpy(c->d_gl8, gl, sizeof(gl), cudaMemcpyHostToDevice) != cudaSuccess) {
        stdg_destroy(c);
        return STDG_ECUDA;
    }
    *out = c;
    return STDG_OK;
}

void stdg_destroy(stdg_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    solver_free(c);
    dev_free_all(c);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* stdg_last_error(const stdg_ctx* c) { return c ? c->err.c_str() : "null context"; }

int stdg_set_mesh(stdg_ctx* c, int64_t n_vert, const double* xyz, int64_t n_elem, const int32_t* elem_vert,
                  const double* period) {
    CHECK_CTX(c);
    if (!xyz || !elem_vert || n_vert < c->dim + 1 || n_elem < 1 || n_elem > (int64_t)INT32_MAX / 8)
        STDG_FAIL(c, STDG_EINVAL, "bad mesh arguments");
    if (period && !all_finite(period, c->dim)) STDG_FAIL(c, STDG_EINVAL, "non-finite period");
    // release everything mesh-dependent
    solver_free(c);
    void* keep_rt = c->d_rt;
    void* keep_gl = c->d_gl8;
    void* keep_err = c->d_err;
    {
        std::vector<void*> keep_p;
        std::vector<size_t> keep_b;
        c->bytes = 0;
        for (size_t k = 0; k < c->allocs.size(); ++k) {
            void* p = c->allocs[k];
            if (p == keep_rt || p == keep_gl || p == keep_err) {
                keep_p.push_back(p);
                keep_b.push_back(c->alloc_bytes[k]);
                c->bytes += c->alloc_bytes[k];
            } else {
                cudaFree(p);
            }
        }
        c->allocs.swap(keep_p);
        c->alloc_bytes.swap(keep_b);
    }
    c->d_face_l = c->d_face_r = nullptr;
    c->d_elem_face = nullptr;
    c->d_preV = c->d_preLam = c->d_preB = nullptr;
    c->d_preV32 = c->d_preB32 = nullptr;
    c->d_preB32t = nullptr;
    c->d_pre2 = nullptr;
    c->d_pre2_32 = nullptr;
    c->d_pre2_mma = nullptr;
    c->d_pre2_16 = nullptr;
    c->d_pre2_scl = nullptr;
    c->d_p2y = c->d_p2t = nullptr;
    c->d_p2status = nullptr;
    c->pre_dt = -1.0;
    c->rec_cap_steps = 0;
    c->rec_steps = 0;
    c->d_X = c->d_Jinv = c->d_detJ = c->d_faceX = c->d_shift = c->d_normal = c->d_xc = c->d_hj = nullptr;
    c->d_frame = nullptr;
    c->d_D = c->d_L = c->d_Mdual = nullptr;
    c->d_D32 = c->d_Dt32 = nullptr;
    c->d_lamf = c->d_muf = c->d_rhoJ = nullptr;
    c->d_lamf_ph = c->d_muf_ph = c->d_rhoJ_ph = nullptr;
    c->alpha_e.clear();
    c->src_alpha.clear();
    c->d_lamf32 = c->d_muf32 = c->d_rhoJ32 = nullptr;
    c->d_vtr = c->d_sigtr = c->d_b = c->d_x = c->d_energy = c->d_sigtmp = nullptr;
    c->d_src = nullptr;
    c->d_rec_elem = nullptr;
    c->d_rec_phi = c->d_records = nullptr;
    c->have_mesh = c->have_material = false;
    c->have_sources = 0;
    c->n_rec = 0;
    c->t = 0.0;

    int rc = build_host_mesh(c->dim, n_vert, xyz, n_elem, elem_vert, period, &c->hm, &c->err);
    if (rc != STDG_OK) return rc;
    const int d = c->dim, NP = c->Nphi, nv = d + 1;
    c->n_elem = n_elem;
    c->n_face = c->hm.n_face;
    c->nvel = n_elem * d * c->Ng * NP;
    c->ntr = n_elem * d * NP;
    c->nsig = c->n_face * c->s * c->Npsi;
    const int64_t nf = c->n_face;
#define ALLOC(ptr, bytes) do { if ((rc = dev_alloc(c, (void**)&(ptr), (bytes))) != STDG_OK) return rc; } while (0)
#define UP(dst, src, bytes) STDG_CUDA(c, cudaMemcpy((dst), (src), (bytes), cudaMemcpyHostToDevice))
    ALLOC(c->d_face_l, sizeof(int32_t) * nf);
    ALLOC(c->d_elem_face, sizeof(int32_t) * n_elem * nv);
    ALLOC(c->d_face_r, sizeof(int32_t) * nf);
    ALLOC(c->d_X, sizeof(double) * n_elem * nv * d);
    ALLOC(c->d_Jinv, sizeof(double) * n_elem * d * d);
    ALLOC(c->d_detJ, sizeof(double) * n_elem);
    ALLOC(c->d_faceX, sizeof(double) * nf * d * d);
    ALLOC(c->d_shift, sizeof(double) * nf * d);
    ALLOC(c->d_normal, sizeof(double) * nf * d);
    ALLOC(c->d_xc, sizeof(double) * nf * d);
    ALLOC(c->d_hj, sizeof(double) * nf);
    ALLOC(c->d_frame, sizeof(double) * nf * d * d);
    ALLOC(c->d_D, sizeof(double) * nf * 2 * d * NP * NP);
    ALLOC(c->d_L, sizeof(double) * nf * NP * NP);
    ALLOC(c->d_Mdual, sizeof(double) * nf * NP * NP);
    ALLOC(c->d_lamf, sizeof(double) * nf);
    ALLOC(c->d_muf, sizeof(double) * nf);
    ALLOC(c->d_rhoJ, sizeof(double) * n_elem);
    ALLOC(c->d_lamf32, sizeof(float) * nf);
    ALLOC(c->d_muf32, sizeof(float) * nf);
    ALLOC(c->d_rhoJ32, sizeof(float) * n_elem);
    ALLOC(c->d_sigtmp, sizeof(double) * c->nsig);
    UP(c->d_face_l, c->hm.face_l.data(), sizeof(int32_t) * nf);
    UP(c->d_elem_face, c->hm.elem_face.data(), sizeof(int32_t) * n_elem * nv);
    UP(c->d_face_r, c->hm.face_r.data(), sizeof(int32_t) * nf);
    UP(c->d_X, c->hm.X.data(), sizeof(double) * n_elem * nv * d);
    UP(c->d_Jinv, c->hm.Jinv.data(), sizeof(double) * n_elem * d * d);
    UP(c->d_detJ, c->hm.detJ.data(), sizeof(double) * n_elem);
    UP(c->d_faceX, c->hm.face_X.data(), sizeof(double) * nf * d * d);
    UP(c->d_shift, c->hm.shift.data(), sizeof(double) * nf * d);
    UP(c->d_normal, c->hm.normal.data(), sizeof(double) * nf * d);
    UP(c->d_xc, c->hm.xc.data(), sizeof(double) * nf * d);
    UP(c->d_hj, c->hm.hj.data(), sizeof(double) * nf);
    UP(c->d_frame, c->hm.frame.data(), sizeof(double) * nf * d * d);
    // blocks D_{i,j} and dual mass matrices, exact for degree 2p + 1 on every sub-cell
    Rule rv = simplex_rule(d, c->rt.p + 2), rf = simplex_rule(d - 1, c->rt.p + 2);
    std::vector<double> pv, pf;
    for (int q = 0; q < rv.n(); ++q) {
        for (int a = 0; a < d; ++a) pv.push_back(rv.pts[q * d + a]);
        pv.push_back(rv.wts[q]);
    }
    for (int q = 0; q < rf.n(); ++q) {
        for (int a = 0; a < d - 1; ++a) pf.push_back(rf.pts[q * (d - 1) + a]);
        pf.push_back(rf.wts[q]);
    }
    double *d_rv = nullptr, *d_rf = nullptr;
    ALLOC(d_rv, sizeof(double) * pv.size());
    ALLOC(d_rf, sizeof(double) * pf.size());
    UP(d_rv, pv.data(), sizeof(double) * pv.size());
    UP(d_rf, pf.data(), sizeof(double) * pf.size());
    STDG_CUDA(c, launch_precompute(c, d_rv, d_rf, rv.n(), rf.n()));
    cudaError_t e = launch_orthonormalize(c);
    if (e == cudaErrorInvalidValue) STDG_FAIL(c, STDG_EMESH, "dual mass matrix not positive definite");
    STDG_CUDA(c, e);
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, d_rv);
    dev_free(c, d_rf);
    dev_free(c, c->d_Mdual);   // only the Cholesky factors are kept
    c->d_Mdual = nullptr;
#undef ALLOC
#undef UP
    c->have_mesh = true;
    if ((rc = alloc_state(c, 1)) != STDG_OK) return rc;
    if (c->opt.precision != STDG_FP64 && (rc = ensure_fp32(c)) != STDG_OK) return rc;
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    return STDG_OK;
}

static int upload_material(stdg_ctx* c);

int stdg_set_material(stdg_ctx* c, const double* lambda, const double* mu, const double* rho) {
    CHECK_CTX(c);
    NEED_MESH(c);
    const int64_t ne = c->n_elem, nf = c->n_face;
    if (!lambda || !mu || !rho) STDG_FAIL(c, STDG_EINVAL, "null material array");
    for (int64_t i = 0; i < ne; ++i)
        if (!std::isfinite(lambda[i]) || !std::isfinite(mu[i]) || !std::isfinite(rho[i]) || !(mu[i] > 0) ||
            !(rho[i] > 0) || lambda[i] < 0)
            STDG_FAIL(c, STDG_EINVAL, "material must be finite with lambda >= 0, mu > 0, rho > 0");
    c->lam_e.assign(lambda, lambda + ne);
    c->mu_e.assign(mu, mu + ne);
    c->rho_e.assign(rho, rho + ne);
    (void)nf;
    return upload_material(c);
}

// Device material from the host copies: E_j as the sub-cell-measure-weighted mean over the
// dual cell (|T_{i,j}| = |T_i| / (d+1)), rho_i |J_i| per element; with a time scale alpha
// the device holds alpha lambda, alpha mu, rho / alpha (physical copies kept for the energy).
// Sets up the preconditioner.
static int upload_material(stdg_ctx* c) {
    const int64_t ne = c->n_elem, nf = c->n_face;
    const bool ts = !c->alpha_e.empty();
    int rc;
    std::vector<double> lf(nf), mf(nf), rj(ne);
    for (int64_t f = 0; f < nf; ++f) {
        const int64_t l = c->hm.face_l[f], r = c->hm.face_r[f];
        double wl = c->hm.detJ[l], wr = r >= 0 ? c->hm.detJ[r] : 0.0;
        lf[f] = (wl * c->lam_e[l] + (r >= 0 ? wr * c->lam_e[r] : 0.0)) / (wl + wr);
        mf[f] = (wl * c->mu_e[l] + (r >= 0 ? wr * c->mu_e[r] : 0.0)) / (wl + wr);
    }
    for (int64_t i = 0; i < ne; ++i) rj[i] = c->rho_e[i] * c->hm.detJ[i];
    if (ts) {
        if (!c->d_lamf_ph) {
            if ((rc = dev_alloc(c, (void**)&c->d_lamf_ph, sizeof(double) * nf)) != STDG_OK) return rc;
            if ((rc = dev_alloc(c, (void**)&c->d_muf_ph, sizeof(double) * nf)) != STDG_OK) return rc;
            if ((rc = dev_alloc(c, (void**)&c->d_rhoJ_ph, sizeof(double) * ne)) != STDG_OK) return rc;
        }
        STDG_CUDA(c, cudaMemcpy(c->d_lamf_ph, lf.data(), sizeof(double) * nf, cudaMemcpyHostToDevice));
        STDG_CUDA(c, cudaMemcpy(c->d_muf_ph, mf.data(), sizeof(double) * nf, cudaMemcpyHostToDevice));
        STDG_CUDA(c, cudaMemcpy(c->d_rhoJ_ph, rj.data(), sizeof(double) * ne, cudaMemcpyHostToDevice));
        for (int64_t f = 0; f < nf; ++f) {   // both elements of a face have the same scale
            const double a = c->alpha_e[c->hm.face_l[f]];
            lf[f] *= a;
            mf[f] *= a;
        }
        for (int64_t i = 0; i < ne; ++i) rj[i] /= c->alpha_e[i];
    } else if (c->d_lamf_ph) {
        dev_free(c, c->d_lamf_ph);
        dev_free(c, c->d_muf_ph);
        dev_free(c, c->d_rhoJ_ph);
        c->d_lamf_ph = c->d_muf_ph = c->d_rhoJ_ph = nullptr;
    }
    STDG_CUDA(c, cudaMemcpy(c->d_lamf, lf.data(), sizeof(double) * nf, cudaMemcpyHostToDevice));
    STDG_CUDA(c, cudaMemcpy(c->d_muf, mf.data(), sizeof(double) * nf, cudaMemcpyHostToDevice));
    STDG_CUDA(c, cudaMemcpy(c->d_rhoJ, rj.data(), sizeof(double) * ne, cudaMemcpyHostToDevice));
    c->have_material = true;
    rc = upload_material32(c);
    if (rc != STDG_OK) return rc;
    if (c->opt.preconditioner) return setup_pre1(c);
    return STDG_OK;
}

// time scale of each point source: that of its element
static void set_source_alpha(stdg_ctx* c) {
    c->src_alpha.clear();
    if (c->alpha_e.empty()) return;
    c->src_alpha.resize(c->src_elem.size());
    for (size_t q = 0; q < c->src_elem.size(); ++q) c->src_alpha[q] = c->alpha_e[c->src_elem[q]];
}

int stdg_set_time_scale(stdg_ctx* c, const double* alpha) {
    CHECK_CTX(c);
    NEED_MESH(c);
    const int64_t ne = c->n_elem;
    if (!alpha) {
        c->alpha_e.clear();
    } else {
        bool ones = true;
        for (int64_t i = 0; i < ne; ++i) {
            if (!std::isfinite(alpha[i]) || !(alpha[i] > 0)) STDG_FAIL(c, STDG_EINVAL, "time scale must be finite and > 0");
            ones = ones && alpha[i] == 1.0;
        }
        for (int64_t f = 0; f < c->n_face; ++f) {
            const int64_t r = c->hm.face_r[f];
            if (r >= 0 && alpha[c->hm.face_l[f]] != alpha[r])
                STDG_FAIL(c, STDG_EINVAL, "time scale differs across a face");
        }
        if (ones) c->alpha_e.clear();
        else c->alpha_e.assign(alpha, alpha + ne);
    }
    int rc;
    if (c->have_material && (rc = upload_material(c)) != STDG_OK) return rc;
    if (c->have_sources) set_source_alpha(c);
    solver_invalidate_graph(c);   // the source wavelets are launch arguments of captured graphs
    return STDG_OK;
}

int stdg_set_shots(stdg_ctx* c, int n_shots) {
    CHECK_CTX(c);
    NEED_MESH(c);
    if (n_shots < 1) STDG_FAIL(c, STDG_EINVAL, "n_shots must be >= 1");
    c->have_sources = 0;
    return alloc_state(c, n_shots);
}

int stdg_set_state(stdg_ctx* c, int shot, const double* v_tr, const double* sig_tr) {
    CHECK_CTX(c);
    NEED_MESH(c);
    if (shot < 0 || shot >= c->n_shots || !v_tr || !sig_tr) STDG_FAIL(c, STDG_EINVAL, "bad shot or null state");
    if (!all_finite(v_tr, c->ntr) || !all_finite(sig_tr, c->nsig)) STDG_FAIL(c, STDG_EINVAL, "non-finite state");
    STDG_CUDA(c, cudaMemcpyAsync(c->d_vtr + shot * c->ntr, v_tr, sizeof(double) * c->ntr, cudaMemcpyHostToDevice, c->stream));
    // stress arrives in the Taylor-monomial basis; the state is kept in orthonormal coordinates
    STDG_CUDA(c, cudaMemcpyAsync(c->d_sigtmp, sig_tr, sizeof(double) * c->nsig, cudaMemcpyHostToDevice, c->stream));
    STDG_CUDA(c, launch_sig_convert(c, c->d_sigtmp, c->d_sigtr + shot * c->nsig, 0));
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    return STDG_OK;
}

int stdg_get_state(stdg_ctx* c, int shot, double* v_tr, double* sig_tr) {
    CHECK_CTX(c);
    NEED_MESH(c);
    if (shot < 0 || shot >= c->n_shots) STDG_FAIL(c, STDG_EINVAL, "bad shot");
    if (v_tr) STDG_CUDA(c, cudaMemcpyAsync(v_tr, c->d_vtr + shot * c->ntr, sizeof(double) * c->ntr, cudaMemcpyDeviceToHost, c->stream));
    if (sig_tr) {
        STDG_CUDA(c, launch_sig_convert(c, c->d_sigtr + shot * c->nsig, c->d_sigtmp, 1));
        STDG_CUDA(c, cudaMemcpyAsync(sig_tr, c->d_sigtmp, sizeof(double) * c->nsig, cudaMemcpyDeviceToHost, c->stream));
    }
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    return STDG_OK;
}

int stdg_set_plane_wave(stdg_ctx* c, int shot, int kind, const double* n, const double* pol, double amp, double t) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (shot < 0 || shot >= c->n_shots || !n || (kind != 0 && kind != 1)) STDG_FAIL(c, STDG_EINVAL, "bad plane-wave arguments");
    if (!all_finite(n, c->dim) || (pol && !all_finite(pol, c->dim)) || !std::isfinite(amp) || !std::isfinite(t))
        STDG_FAIL(c, STDG_EINVAL, "non-finite plane-wave argument");
    double nn = 0;
    for (int a = 0; a < c->dim; ++a) nn += n[a] * n[a];
    if (!(nn > 0)) STDG_FAIL(c, STDG_EINVAL, "zero wave vector");
    if (kind == 1 && c->dim == 3 && !pol) STDG_FAIL(c, STDG_EINVAL, "3D S wave needs a polarisation");
    Rule r = simplex_rule(c->dim, 2 * c->rt.p + 8);
    std::vector<double> pr;
    for (int q = 0; q < r.n(); ++q) {
        for (int a = 0; a < c->dim; ++a) pr.push_back(r.pts[q * c->dim + a]);
        pr.push_back(r.wts[q]);
    }
    double* d_r = nullptr;
    int rc = dev_alloc(c, (void**)&d_r, sizeof(double) * pr.size());
    if (rc != STDG_OK) return rc;
    STDG_CUDA(c, cudaMemcpy(d_r, pr.data(), sizeof(double) * pr.size(), cudaMemcpyHostToDevice));
    STDG_CUDA(c, launch_project_plane_wave(c, shot, kind, n, pol, amp, t, d_r, r.n()));
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, d_r);
    c->t = t;
    return STDG_OK;
}

int stdg_set_point_sources(stdg_ctx* c, int n_shots, int per_shot, const double* xs, const double* dir, double f0,
                           double t_delay, double a1) {
    CHECK_CTX(c);
    NEED_ALL(c);
    const int d = c->dim, NP = c->Nphi;
    if (n_shots < 1 || per_shot < 1 || !xs || !dir) STDG_FAIL(c, STDG_EINVAL, "bad source arguments");
    const int64_t ns = (int64_t)n_shots * per_shot;
    if (!all_finite(xs, ns * d) || !all_finite(dir, ns * d) || !std::isfinite(f0) || !std::isfinite(t_delay) ||
        !std::isfinite(a1))
        STDG_FAIL(c, STDG_EINVAL, "non-finite source argument");
    int rc = alloc_state(c, n_shots);
    if (rc != STDG_OK) return rc;
    std::vector<double> host((size_t)ns * (d + NP));
    c->src_elem.assign(ns, 0);
    for (int64_t s = 0; s < ns; ++s) {
        double y[3];
        int64_t e = locate_point(c->hm, xs + s * d, y);
        if (e < 0) STDG_FAIL(c, STDG_EINVAL, "source outside the mesh");
        c->src_elem[s] = e;
        for (int a = 0; a < d; ++a) host[s * (d + NP) + a] = dir[s * d + a];
        eval_phi_host(c, e, y, &host[s * (d + NP) + d]);
    }
    dev_free(c, c->d_src);
    c->d_src = nullptr;
    if ((rc = dev_alloc(c, (void**)&c->d_src, sizeof(double) * host.size())) != STDG_OK) return rc;
    STDG_CUDA(c, cudaMemcpy(c->d_src, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice));
    c->src_per_shot = per_shot;
    c->src_xs.assign(xs, xs + ns * d);
    c->src_dir.assign(dir, dir + ns * d);
    c->src_f0 = f0;
    c->src_td = t_delay;
    c->src_a1 = a1;
    c->have_sources = 1;
    set_source_alpha(c);
    solver_invalidate_graph(c);
    return STDG_OK;
}

int stdg_set_sources(stdg_ctx* c, int n_shots, const double* xs, const double* dir, double f0, double t_delay, double a1) {
    return stdg_set_point_sources(c, n_shots, 1, xs, dir, f0, t_delay, a1);
}

int stdg_set_receivers(stdg_ctx* c, int n_rec, const double* xr) {
    CHECK_CTX(c);
    NEED_MESH(c);
    const int d = c->dim, NP = c->Nphi;
    if (n_rec < 0 || (n_rec > 0 && !xr)) STDG_FAIL(c, STDG_EINVAL, "bad receiver arguments");
    if (n_rec > 0 && !all_finite(xr, (int64_t)n_rec * d)) STDG_FAIL(c, STDG_EINVAL, "non-finite receiver position");
    std::vector<int32_t> el(n_rec);
    std::vector<double> phi((size_t)n_rec * NP);
    for (int r = 0; r < n_rec; ++r) {
        double y[3];
        int64_t e = locate_point(c->hm, xr + r * d, y);
        if (e < 0) STDG_FAIL(c, STDG_EINVAL, "receiver outside the mesh");
        el[r] = (int32_t)e;
        eval_phi_host(c, e, y, &phi[r * NP]);
    }
    dev_free(c, c->d_rec_elem);
    dev_free(c, c->d_rec_phi);
    dev_free(c, c->d_records);
    c->d_rec_elem = nullptr;
    c->d_rec_phi = c->d_records = nullptr;
    c->n_rec = n_rec;
    c->rec_steps = 0;
    c->rec_cap_steps = 0;
    solver_invalidate_graph(c);
    if (n_rec == 0) return STDG_OK;
    int rc;
    if ((rc = dev_alloc(c, (void**)&c->d_rec_elem, sizeof(int32_t) * n_rec)) != STDG_OK) return rc;
    if ((rc = dev_alloc(c, (void**)&c->d_rec_phi, sizeof(double) * n_rec * NP)) != STDG_OK) return rc;
    STDG_CUDA(c, cudaMemcpy(c->d_rec_elem, el.data(), sizeof(int32_t) * n_rec, cudaMemcpyHostToDevice));
    STDG_CUDA(c, cudaMemcpy(c->d_rec_phi, phi.data(), sizeof(double) * n_rec * NP, cudaMemcpyHostToDevice));
    return STDG_OK;
}

static int ensure_records(stdg_ctx* c, int n_steps) {
    if (c->n_rec == 0) return STDG_OK;
    const int64_t need = c->rec_steps + n_steps;
    if (need <= c->rec_cap_steps) return STDG_OK;
    int64_t cap = std::max<int64_t>(need, std::max<int64_t>(256, 2 * c->rec_cap_steps));
    const int64_t per = (int64_t)c->n_rec * c->dim;
    double* nb = nullptr;
    int rc = dev_alloc(c, (void**)&nb, sizeof(double) * per * cap * c->n_shots);
    if (rc != STDG_OK) return rc;
    if (c->d_records && c->rec_steps > 0)
        for (int s = 0; s < c->n_shots; ++s)
            STDG_CUDA(c, cudaMemcpy(nb + s * cap * per, c->d_records + s * c->rec_cap_steps * per,
                                    sizeof(double) * per * c->rec_steps, cudaMemcpyDeviceToDevice));
    dev_free(c, c->d_records);
    c->d_records = nb;
    c->rec_cap_steps = cap;
    solver_invalidate_graph(c);
    return STDG_OK;
}

int stdg_step(stdg_ctx* c, double dt, int n_steps, stdg_stats* out) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (!(dt > 0) || !std::isfinite(dt) || n_steps < 0) STDG_FAIL(c, STDG_EINVAL, "dt must be > 0 and n_steps >= 0");
    if (out) std::memset(out, 0, sizeof(*out));
    if (n_steps == 0) return STDG_OK;
    int rc = ensure_records(c, n_steps);
    if (rc != STDG_OK) return rc;
    // Theorem 4 bounds the energy only without sources
    const bool check = c->echeck_on && !(c->have_sources && c->src_a1 != 0.0);
    std::vector<double> e0, e1;
    if (check) {
        e0.resize(c->n_shots);
        if ((rc = stdg_energy(c, e0.data())) != STDG_OK) return rc;
    }
    rc = solver_step(c, dt, n_steps, out);
    if (check && rc == STDG_OK) {
        e1.resize(c->n_shots);
        if ((rc = stdg_energy(c, e1.data())) != STDG_OK) return rc;
        for (int s = 0; s < c->n_shots; ++s)
            if (!(e1[s] <= (1.0 + c->echeck_tol) * e0[s])) {   // also catches a non-finite energy
                char msg[160];
                std::snprintf(msg, sizeof msg, "energy of shot %d grew over a source-free step: %.17g -> %.17g", s,
                              e0[s], e1[s]);
                STDG_FAIL(c, STDG_EENERGY, msg);
            }
    }
    return rc;
}

int stdg_set_energy_check(stdg_ctx* c, int enable, double rel_tol) {
    CHECK_CTX(c);
    if (!std::isfinite(rel_tol) || rel_tol <= -1.0) STDG_FAIL(c, STDG_EINVAL, "rel_tol must be finite and > -1");
    c->echeck_on = enable != 0;
    c->echeck_tol = rel_tol;
    return STDG_OK;
}

int stdg_misfit_grad(stdg_ctx* c, double dt, int n_steps, const double* data, int checkpoint_every, double* loss,
                     double* g_lambda, double* g_mu, double* g_rho, double* g_src, stdg_stats* out) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (!(dt > 0) || !std::isfinite(dt) || n_steps < 1 || !data || !loss)
        STDG_FAIL(c, STDG_EINVAL, "bad misfit arguments");
    if (c->opt.scheme != STDG_SCHEME_STDG) STDG_FAIL(c, STDG_EINVAL, "the adjoint covers the space-time DG scheme only");
    if (!c->alpha_e.empty()) STDG_FAIL(c, STDG_ESTATE, "the adjoint needs a time scale of 1 everywhere");
    if (c->n_rec < 1) STDG_FAIL(c, STDG_ESTATE, "the misfit needs receivers (stdg_set_receivers)");
    if (!c->d_vtr) STDG_FAIL(c, STDG_ESTATE, "no state: set sources, shots or a state first");
    const int64_t nd = (int64_t)c->n_shots * n_steps * c->n_rec * c->dim;
    if (!all_finite(data, nd)) STDG_FAIL(c, STDG_EINVAL, "non-finite data");
    const int K = checkpoint_every > 0 ? std::min(checkpoint_every, n_steps) : std::min(20, n_steps);
    int rc = ensure_records(c, n_steps);
    if (rc != STDG_OK) return rc;
    stdg_stats st;
    rc = misfit_grad_impl(c, dt, n_steps, data, K, loss, g_lambda, g_mu, g_rho, g_src, &st);
    if (out) *out = st;
    return rc;
}

int stdg_get_time(stdg_ctx* c, double* t) {
    CHECK_CTX(c);
    if (!t) return STDG_EINVAL;
    *t = c->t;
    return STDG_OK;
}

int stdg_set_time(stdg_ctx* c, double t) {
    CHECK_CTX(c);
    if (!std::isfinite(t)) STDG_FAIL(c, STDG_EINVAL, "non-finite time");
    c->t = t;
    return STDG_OK;
}

int stdg_energy(stdg_ctx* c, double* out) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (!out) return STDG_EINVAL;
    for (int s = 0; s < c->n_shots; ++s) {
        STDG_CUDA(c, launch_energy(c, s, c->d_energy + s));
    }
    STDG_CUDA(c, cudaMemcpyAsync(out, c->d_energy, sizeof(double) * c->n_shots, cudaMemcpyDeviceToHost, c->stream));
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    return STDG_OK;
}

int stdg_read_receivers(stdg_ctx* c, double* out, int64_t cap) {
    CHECK_CTX(c);
    if (c->n_rec == 0 || c->rec_steps == 0) return 0;
    const int64_t per = (int64_t)c->n_rec * c->dim;
    if (!out || cap < per * c->rec_steps * c->n_shots) STDG_FAIL(c, STDG_EINVAL, "receiver buffer too small");
    for (int s = 0; s < c->n_shots; ++s)
        STDG_CUDA(c, cudaMemcpyAsync(out + s * c->rec_steps * per, c->d_records + s * c->rec_cap_steps * per,
                                     sizeof(double) * per * c->rec_steps, cudaMemcpyDeviceToHost, c->stream));
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    return (int)c->rec_steps;
}

int stdg_apply_operator(stdg_ctx* c, double dt, const double* x, double* y) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (!x || !y || !(dt > 0)) STDG_FAIL(c, STDG_EINVAL, "bad operator arguments");
    double *dx = nullptr, *dy = nullptr;
    int rc;
    if ((rc = dev_alloc(c, (void**)&dx, sizeof(double) * c->nvel)) != STDG_OK) return rc;
    if ((rc = dev_alloc(c, (void**)&dy, sizeof(double) * c->nvel)) != STDG_OK) { dev_free(c, dx); return rc; }
    STDG_CUDA(c, cudaMemcpyAsync(dx, x, sizeof(double) * c->nvel, cudaMemcpyHostToDevice, c->stream));
    STDG_CUDA(c, launch_apply(c, dt, dx, dy, 1.0));
    STDG_CUDA(c, cudaMemcpyAsync(y, dy, sizeof(double) * c->nvel, cudaMemcpyDeviceToHost, c->stream));
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, dx);
    dev_free(c, dy);
    return STDG_OK;
}

int stdg_apply_operator_device(stdg_ctx* c, double dt, const void* x_dev, void* y_dev, int fp32) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (!x_dev || !y_dev || !(dt > 0)) STDG_FAIL(c, STDG_EINVAL, "bad operator arguments");
    if (fp32) {
        int rc = ensure_fp32(c);
        if (rc != STDG_OK) return rc;
        if ((rc = upload_material32(c)) != STDG_OK) return rc;
        STDG_CUDA(c, launch_apply32(c, dt, (const float*)x_dev, (float*)y_dev, 1.0));
        return take_device_error(c);   // the FP32 face kernel's bounded waits
    } else {
        STDG_CUDA(c, launch_apply(c, dt, (const double*)x_dev, (double*)y_dev, 1.0));
    }
    return STDG_OK;
}

int stdg_query(stdg_ctx* c, int what, int64_t* out) {
    CHECK_CTX(c);
    if (!out) return STDG_EINVAL;
    switch (what) {
        case 0: *out = c->n_elem; break;
        case 1: *out = c->n_face; break;
        case 2: *out = c->Nphi; break;
        case 3: *out = c->Npsi; break;
        case 4: *out = c->Ng; break;
        case 5: *out = c->s; break;
        case 6: *out = c->n_shots; break;
        case 7: *out = c->nvel; break;
        case 8: *out = c->n_rec; break;
        case 9: *out = c->hm.n_bnd; break;
        case 10: *out = (int64_t)c->bytes; break;
        case 11: *out = c->last_launches; break;
        case 12: *out = c->d_pre2_32 ? (c->d_pre2_16 && c->pre2_bits == 16 ? 16 : 32) : 0; break;
        default: STDG_FAIL(c, STDG_EINVAL, "unknown query");
    }
    return STDG_OK;
}

int stdg_set_pre2_storage(stdg_ctx* c, int bits) {
    CHECK_CTX(c);
    if (bits != 16 && bits != 32) STDG_FAIL(c, STDG_EINVAL, "bits must be 16 or 32");
    c->pre2_bits = bits;
    solver_invalidate_graph(c);   // graphs keep the kernel they were captured with
    return STDG_OK;
}

int stdg_get_faces(stdg_ctx* c, int32_t* face_l, int32_t* face_r) {
    CHECK_CTX(c);
    NEED_MESH(c);
    if (face_l) std::memcpy(face_l, c->hm.face_l.data(), sizeof(int32_t) * c->n_face);
    if (face_r) std::memcpy(face_r, c->hm.face_r.data(), sizeof(int32_t) * c->n_face);
    return STDG_OK;
}

int stdg_mesh_faces(int dim, int64_t n_vert, const double* xyz, int64_t n_elem, const int32_t* elem_vert,
                    const double* period, int64_t* n_face, int32_t* face_l, int32_t* face_r) {
    if (dim != 2 && dim != 3) return STDG_EINVAL;
    if (!n_face || !xyz || !elem_vert || n_vert < dim + 1 || n_elem < 1 || n_elem > (int64_t)INT32_MAX / 8)
        return STDG_EINVAL;
    if (period && !all_finite(period, dim)) return STDG_EINVAL;
    const int64_t cap = *n_face;
    HostMesh hm;
    std::string err;
    const int rc = build_host_mesh(dim, n_vert, xyz, n_elem, elem_vert, period, &hm, &err);
    if (rc != STDG_OK) return rc;
    *n_face = hm.n_face;
    if (!face_l && !face_r) return STDG_OK;
    if (cap < hm.n_face) return STDG_EINVAL;
    if (face_l) std::memcpy(face_l, hm.face_l.data(), sizeof(int32_t) * hm.n_face);
    if (face_r) std::memcpy(face_r, hm.face_r.data(), sizeof(int32_t) * hm.n_face);
    return STDG_OK;
}

int stdg_locate_points(int dim, int64_t n_vert, const double* xyz, int64_t n_elem, const int32_t* elem_vert,
                       const double* period, int64_t n_pts, const double* pts, int64_t* elem_out) {
    if (dim != 2 && dim != 3) return STDG_EINVAL;
    if (!xyz || !elem_vert || n_vert < dim + 1 || n_elem < 1 || n_elem > (int64_t)INT32_MAX / 8 || n_pts < 0 ||
        (n_pts > 0 && (!pts || !elem_out)))
        return STDG_EINVAL;
    if (period && !all_finite(period, dim)) return STDG_EINVAL;
    if (n_pts > 0 && !all_finite(pts, n_pts * dim)) return STDG_EINVAL;
    HostMesh hm;
    std::string err;
    const int rc = build_host_mesh(dim, n_vert, xyz, n_elem, elem_vert, period, &hm, &err);
    if (rc != STDG_OK) return rc;
    for (int64_t k = 0; k < n_pts; ++k) {
        double y[3];
        elem_out[k] = locate_point(hm, pts + k * dim, y);
    }
    return STDG_OK;
}

int stdg_reference_tables(int dim, int p, int p_gamma, double* Mref, double* W, double* T, double* S, double* kappa,
                          double* u) {
    if (dim != 2 && dim != 3) return STDG_EINVAL;
    if (p < 1 || p > (dim == 2 ? 4 : 3) || p_gamma < 0 || p_gamma > 4) return STDG_EINVAL;
    RefTables rt;
    build_ref_tables(dim, p, p_gamma, &rt);
    const int n = rt.Nphi, g = rt.Ng;
    if (Mref) std::memcpy(Mref, rt.Mref, sizeof(double) * n * n);
    if (W) std::memcpy(W, rt.W, sizeof(double) * g);
    if (T) std::memcpy(T, rt.T, sizeof(double) * g * g);
    if (S) std::memcpy(S, rt.S, sizeof(double) * g * g);
    if (kappa) *kappa = rt.kappa;
    if (u) std::memcpy(u, rt.u_tr, sizeof(double) * g);
    return STDG_OK;
}

int stdg_apply_preconditioner(stdg_ctx* c, double dt, const double* r, double* z) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (!c->opt.preconditioner || !c->d_preV) STDG_FAIL(c, STDG_ESTATE, "context created without a preconditioner");
    if (!r || !z || !(dt > 0)) STDG_FAIL(c, STDG_EINVAL, "bad preconditioner arguments");
    int rc = precond_for_dt(c, dt);
    if (rc != STDG_OK) return rc;
    if (c->opt.preconditioner == 2 && !c->d_p2y) STDG_FAIL(c, STDG_ESTATE, "call stdg_set_shots (or set a state) first");
    if (c->opt.preconditioner == 2 && !c->d_pre2)
        STDG_FAIL(c, STDG_ESTATE, "FP64 stencil blocks exist only in FP64 contexts (mixed precision keeps FP32 blocks)");
    double *dr = nullptr, *dz = nullptr;
    if ((rc = dev_alloc(c, (void**)&dr, sizeof(double) * c->nvel)) != STDG_OK) return rc;
    if ((rc = dev_alloc(c, (void**)&dz, sizeof(double) * c->nvel)) != STDG_OK) { dev_free(c, dr); return rc; }
    STDG_CUDA(c, cudaMemcpyAsync(dr, r, sizeof(double) * c->nvel, cudaMemcpyHostToDevice, c->stream));
    if (c->opt.preconditioner == 2) STDG_CUDA(c, launch_pre2_apply(c, dr, dz, nullptr, 0, 1));
    else STDG_CUDA(c, launch_pre1_apply(c, dr, dz, nullptr, 0));
    STDG_CUDA(c, cudaMemcpyAsync(z, dz, sizeof(double) * c->nvel, cudaMemcpyDeviceToHost, c->stream));
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    dev_free(c, dr);
    dev_free(c, dz);
    return STDG_OK;
}

int stdg_apply_preconditioner_device(stdg_ctx* c, double dt, const void* r_dev, void* z_dev, int fp32) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (!c->opt.preconditioner || !c->d_preV) STDG_FAIL(c, STDG_ESTATE, "context created without a preconditioner");
    if (!r_dev || !z_dev || r_dev == z_dev || !(dt > 0)) STDG_FAIL(c, STDG_EINVAL, "bad preconditioner arguments");
    if (fp32 && c->opt.precision == STDG_FP64) STDG_FAIL(c, STDG_ESTATE, "FP32 preconditioner blocks exist only in mixed precision");
    int rc = precond_for_dt(c, dt);
    if (rc != STDG_OK) return rc;
    if (c->opt.preconditioner == 2 && !c->d_p2y) STDG_FAIL(c, STDG_ESTATE, "call stdg_set_shots (or set a state) first");
    if (!fp32 && c->opt.preconditioner == 2 && !c->d_pre2)
        STDG_FAIL(c, STDG_ESTATE, "FP64 stencil blocks exist only in FP64 contexts (mixed precision keeps FP32 blocks)");
    if (fp32 && (rc = ensure_fp32(c)) != STDG_OK) return rc;
    if (fp32 && (rc = upload_material32(c)) != STDG_OK) return rc;
    const int ns = c->n_shots;
    if (c->opt.preconditioner == 2)
        STDG_CUDA(c, fp32 ? launch_pre2_apply32(c, (const float*)r_dev, (float*)z_dev, nullptr, 0, ns)
                          : launch_pre2_apply(c, (const double*)r_dev, (double*)z_dev, nullptr, 0, ns));
    else
        STDG_CUDA(c, fp32 ? launch_pre1_apply32(c, (const float*)r_dev, (float*)z_dev, nullptr, 0, ns)
                          : launch_pre1_apply(c, (const double*)r_dev, (double*)z_dev, nullptr, 0, ns));
    return take_device_error(c);
}

int stdg_time_kernel(stdg_ctx* c, double dt, int which, int fp32, int n, double* ms_out) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (n < 1 || !ms_out || which < 0 || which > 4) STDG_FAIL(c, STDG_EINVAL, "bad timing arguments");
    if (which == 4 && (c->opt.preconditioner != 2 || !fp32))
        STDG_FAIL(c, STDG_ESTATE, "the batched local step is timed for the FP32 stencil preconditioner");
    if (which == 1 && !c->opt.preconditioner) STDG_FAIL(c, STDG_ESTATE, "context created without a preconditioner");
    if (which == 2 && c->opt.preconditioner != 2) STDG_FAIL(c, STDG_ESTATE, "context created without the stencil preconditioner");
    if (which == 2 && fp32 && !c->d_pre2_32) STDG_FAIL(c, STDG_ESTATE, "FP32 stencil blocks exist only in mixed precision");
    if (which == 2 && !fp32 && !c->d_pre2) STDG_FAIL(c, STDG_ESTATE, "FP64 stencil blocks exist only in FP64 contexts");
    if (which == 1 && fp32 && !c->d_preV32) STDG_FAIL(c, STDG_ESTATE, "FP32 block-Jacobi blocks exist only in mixed precision");
    int rc;
    if (fp32 && (rc = ensure_fp32(c)) != STDG_OK) return rc;
    if (fp32 && (rc = upload_material32(c)) != STDG_OK) return rc;
    if (which == 1 || which == 2 || which == 4) {
        if ((rc = precond_for_dt(c, dt)) != STDG_OK) return rc;
    }
    void *dx = nullptr, *dy = nullptr, *dw = nullptr;
    const size_t bytes = (fp32 ? sizeof(float) : sizeof(double)) * c->nvel * (which == 4 ? c->n_shots : 1);
    if ((rc = dev_alloc(c, &dx, bytes)) != STDG_OK) return rc;
    if ((rc = dev_alloc(c, &dy, bytes)) != STDG_OK) { dev_free(c, dx); return rc; }
    if ((rc = dev_alloc(c, &dw, bytes)) != STDG_OK) { dev_free(c, dx); dev_free(c, dy); return rc; }
    STDG_CUDA(c, cudaMemsetAsync(dx, 0, bytes, c->stream));
    STDG_CUDA(c, cudaMemsetAsync(dy, 0, bytes, c->stream));
    STDG_CUDA(c, cudaMemsetAsync(dw, 0, bytes, c->stream));
    auto launch = [&]() -> cudaError_t {
        switch (which) {
            case 0: return launch_face_only(c, dt, dx, dy, 1.0, fp32);
            case 1: return fp32 ? launch_pre1_apply32(c, (const float*)dx, (float*)dy, nullptr, 0)
                                : launch_pre1_apply(c, (const double*)dx, (double*)dy, nullptr, 0);
            case 2: return launch_pre2_local(c, fp32, dx, dw, dy);
            case 4: return launch_pre2_local_batch(c, (const float*)dx, (const float*)dw, (float*)dy);
            default: return fp32 ? launch_apply32(c, dt, (const float*)dx, (float*)dy, 1.0, nullptr, 0, 1)
                                 : launch_apply(c, dt, (const double*)dx, (double*)dy, 1.0, nullptr, 0, 1);
        }
    };
    STDG_CUDA(c, launch());   // warm-up
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, c->stream);
    for (int i = 0; i < n; ++i) STDG_CUDA(c, launch());
    cudaEventRecord(e1, c->stream);
    STDG_CUDA(c, cudaEventSynchronize(e1));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms / n;
    dev_free(c, dx);
    dev_free(c, dy);
    dev_free(c, dw);
    return take_device_error(c);
}

// Times each candidate launch shape of the kernels this context runs (zero vectors, n
// back-to-back launches, CUDA events) and keeps the fastest; graphs captured before are dropped.
int stdg_autotune(stdg_ctx* c, double dt, stdg_tuning* out) {
    CHECK_CTX(c);
    NEED_ALL(c);
    if (!(dt > 0) || !std::isfinite(dt)) STDG_FAIL(c, STDG_EINVAL, "dt must be > 0");
    int rc;
    const bool mixed = c->opt.precision != STDG_FP64;
    const int ns = c->n_shots;
    if (mixed && (rc = ensure_fp32(c)) != STDG_OK) return rc;
    if (mixed && (rc = upload_material32(c)) != STDG_OK) return rc;
    if (c->opt.preconditioner && (rc = precond_for_dt(c, dt)) != STDG_OK) return rc;
    const size_t w = mixed ? sizeof(float) : sizeof(double);
    const size_t bytes = w * c->nvel * ns;
    void *dx = nullptr, *dy = nullptr, *dw = nullptr;
    if ((rc = dev_alloc(c, &dx, bytes)) != STDG_OK) return rc;
    if ((rc = dev_alloc(c, &dy, bytes)) != STDG_OK) { dev_free(c, dx); return rc; }
    if ((rc = dev_alloc(c, &dw, bytes)) != STDG_OK) { dev_free(c, dx); dev_free(c, dy); return rc; }
    STDG_CUDA(c, cudaMemsetAsync(dx, 0, bytes, c->stream));
    STDG_CUDA(c, cudaMemsetAsync(dy, 0, bytes, c->stream));
    STDG_CUDA(c, cudaMemsetAsync(dw, 0, bytes, c->stream));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int tried = 0;
    auto time = [&](auto launch) -> double {   // ms per launch, or a huge value if a launch fails
        const int n = 10;
        if (launch() != cudaSuccess) { cudaGetLastError(); return 1e30; }
        cudaEventRecord(e0, c->stream);
        for (int i = 0; i < n; ++i)
            if (launch() != cudaSuccess) { cudaGetLastError(); return 1e30; }
        cudaEventRecord(e1, c->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ++tried;
        return ms / n;
    };
    stdg_tuning res{};
    // the face kernel of the Krylov operator: FP32 in mixed precision (the bulk-copy kernel for one
    // shot, the register kernel for a batch), FP64 otherwise (its generic kernel has fixed shapes)
    if (mixed) {
        double best = 1e30;
        Tuning bt = c->tune;
        for (int cap : (ns == 1 ? std::vector<int>{1, 0} : std::vector<int>{1}))
            for (int wpb : {1, 2, 4})
                for (int bpsm : (ns == 1 ? std::vector<int>{8, 16, 32, 64} : std::vector<int>{16})) {
                    c->tune.face_cap = cap;
                    c->tune.face_wpb = wpb;
                    c->tune.face_bpsm = bpsm;
                    const double ms = time([&]() {
                        return launch_apply32(c, dt, (const float*)dx, (float*)dy, 1.0, nullptr, 0, ns);
                    });
                    if (ms < best) { best = ms; bt = c->tune; }
                }
        c->tune = bt;
        res.face_ms = best;
    }
    if (c->opt.preconditioner == 2) {
        double best = 1e30;
        Tuning bt = c->tune;
        const bool mma = mixed && ns > 1 && c->d_pre2_mma;
        for (int k : (mma ? std::vector<int>{1, 2} : std::vector<int>{1, 2, 4})) {
            if (mma) c->tune.mma_cps = k; else c->tune.pre2_wpb = k;
            const double ms = time([&]() -> cudaError_t {
                if (mixed) return launch_pre2_local_batch(c, (const float*)dx, (const float*)dw, (float*)dy);
                return launch_pre2_local(c, 0, dx, dw, dy);
            });
            if (ms < best) { best = ms; bt = c->tune; }
        }
        c->tune = bt;
        res.pre2_ms = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(c, dx);
    dev_free(c, dy);
    dev_free(c, dw);
    if ((rc = take_device_error(c)) != STDG_OK) return rc;
    solver_invalidate_graph(c);   // graphs keep the launch shapes they were captured with
    res.face_warps_per_block = c->tune.face_wpb;
    res.face_blocks_per_sm = c->tune.face_bpsm;
    res.face_register_cap = c->tune.face_cap;
    res.pre2_warps_per_block = c->tune.pre2_wpb;
    res.mma_ctas_per_sm = c->tune.mma_cps;
    res.candidates = tried;
    if (out) *out = res;
    return STDG_OK;
}

int stdg_inject_wait_error(stdg_ctx* c) {
    CHECK_CTX(c);
    if (!c->d_err) STDG_FAIL(c, STDG_ESTATE, "no device error word");
    const int one = 1;
    STDG_CUDA(c, cudaMemcpyAsync(c->d_err, &one, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    STDG_CUDA(c, cudaStreamSynchronize(c->stream));
    return STDG_OK;
}

int stdg_time_operator(stdg_ctx* c, double dt, int fp32, int n, double* ms_out) {
    return stdg_time_kernel(c, dt, 0, fp32, n, ms_out);
}

}  // extern "C"
