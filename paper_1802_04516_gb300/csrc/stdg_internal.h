// Internal declarations of the stdg library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "stdg.h"

namespace stdg {

constexpr int kMaxNP = 20;   // N_phi = N_psi <= 20 (3D p=3, 2D p=4: 15)
constexpr int kMaxNG = 5;    // N_gamma <= 5

// Reference-element and time-basis tables, built on the host (host_setup.cpp) and
// copied to the device once per context.
struct RefTables {
    int dim, p, pg, Nphi, Npsi, Ng, s;
    int exps[kMaxNP][3];          // monomial exponents, graded-lex (dual basis and Vandermonde)
    int succ[kMaxNP][3];          // index of exps[b] + unit exponent s (-1 beyond degree p)
    double coef[kMaxNP * kMaxNP]; // phi_k(xi) = sum_a coef[a*Nphi + k] xi^a
    double Mref[kMaxNP * kMaxNP]; // int_{ref simplex} phi_k phi_m
    double MrefInv[kMaxNP * kMaxNP];
    double MrefLinv[kMaxNP * kMaxNP];   // R^{-1} with M_ref = R R^T (R lower triangular)
    double tnodes[kMaxNG], W[kMaxNG], g0[kMaxNG], g1[kMaxNG];
    double T[kMaxNG * kMaxNG];    // gamma(1) gamma(1)^T - K
    double Tinv[kMaxNG * kMaxNG];
    double S[kMaxNG * kMaxNG];    // W T^{-1} W  (time factor of the Schur term)
    double Tinv_g0[kMaxNG];       // T^{-1} gamma(0)
    double u_tr[kMaxNG];          // gamma(1)^T T^{-1} W  (stress trace weights)
    double kappa;                 // gamma(1)^T T^{-1} gamma(0)
};

// A quadrature rule on a reference simplex: points (n x dim, barycentric-free
// reference coordinates) and weights summing to 1/dim!.
struct Rule {
    int dim = 0;
    std::vector<double> pts, wts;
    int n() const { return (int)wts.size(); }
};

void build_ref_tables(int dim, int p, int pg, RefTables* out);
Rule simplex_rule(int dim, int n_per_dir);
void gauss_legendre01(int n, double* x, double* w);
void lagrange_time(const RefTables& rt, double tau, double* val);

// Host-side mesh connectivity (Sec. 3): faces, l(j), r(j), normals, dual cells.
struct HostMesh {
    int dim = 0;
    int64_t n_elem = 0, n_face = 0, n_bnd = 0;
    std::vector<double> X;        // unwrapped element vertices [e][dim+1][dim]
    std::vector<double> Jinv;     // [e][dim][dim]  xi = Jinv (x - X0)
    std::vector<double> detJ;     // [e]
    std::vector<int32_t> face_l, face_r;   // r = -1 on the boundary
    std::vector<int8_t> face_fl, face_fr;  // local face index (opposite local vertex)
    std::vector<int32_t> elem_face;        // [e][dim+1]
    std::vector<double> face_X;   // face vertices in the frame of l(j) [f][dim][dim]
    std::vector<double> shift;    // r-frame -> l-frame translation [f][dim]
    std::vector<double> normal;   // unit, from l to r [f][dim]
    std::vector<double> xc, hj;   // dual-cell centre (l frame) and scale
    std::vector<double> frame;    // [f][dim][dim] B_j: principal-axis coordinates y' = B_j (x - x_j) of R_j
    std::vector<double> period;   // dim entries (0 = not periodic), empty if none
};

// Returns STDG_OK or STDG_EMESH (message in err).
int build_host_mesh(int dim, int64_t n_vert, const double* xyz, int64_t n_elem, const int32_t* ev,
                    const double* period, HostMesh* m, std::string* err);
// Element containing x (lowest index wins); writes the point in that element's frame.
int64_t locate_point(const HostMesh& m, const double* x, double* x_local);

// Krylov workspace and step graph state live in the context.
struct Scalars;   // device-side solver scalars (defined in solver.cu)

}  // namespace stdg

namespace stdg {
// Launch shapes of the hot kernels, chosen by stdg_autotune (defaults until it runs)
struct Tuning {
    int face_wpb = 4;     // face kernels: warps per block (1, 2, 4)
    int face_bpsm = 16;   // single-shot bulk-copy face kernel: grid cap, blocks per SM
    int face_cap = 1;     // single-shot bulk-copy face kernel: register cap for occupancy (1) or none (0)
    int pre2_wpb = 4;     // CUDA-core stencil local step: warps per block (1, 2, 4)
    int mma_cps = 2;      // tensor-core stencil local step: CTAs per SM (1, 2)
};
}  // namespace stdg

struct stdg_ctx {
    int dim = 0;
    stdg_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    bool have_mesh = false, have_material = false;

    stdg::RefTables rt{};
    stdg::HostMesh hm;
    int Nphi = 0, Npsi = 0, Ng = 0, s = 0;
    int64_t n_elem = 0, n_face = 0;
    int64_t nvel = 0;      // velocity values per shot per slab: n_elem*dim*Ng*Nphi
    int64_t ntr = 0;       // velocity trace values per shot: n_elem*dim*Nphi
    int64_t nsig = 0;      // stress trace values per shot: n_face*s*Npsi
    int n_shots = 1;
    double t = 0.0;

    // ---- device: tables and geometry
    stdg::RefTables* d_rt = nullptr;
    int32_t *d_face_l = nullptr, *d_face_r = nullptr;
    double *d_X = nullptr, *d_Jinv = nullptr, *d_detJ = nullptr;
    double *d_faceX = nullptr, *d_shift = nullptr, *d_normal = nullptr, *d_xc = nullptr, *d_hj = nullptr;
    double* d_frame = nullptr;  // principal-axis frames B_j of the dual cells [face][dim][dim]
    double *d_D = nullptr;      // orthonormalised blocks D~_{i,j} [face][side][l][n][m] (FP64)
    double *d_L = nullptr;      // Cholesky factors of the dual mass matrices (lower, [face][m][m'])
    double *d_Mdual = nullptr;  // dual mass matrices (set-up workspace)
    float *d_D32 = nullptr;     // FP32 copy of D~
    float *d_Dt32 = nullptr;    // FP32 D~ in tiles (2D p = 3 and 3D p = 2 only: the tiled face kernels)
    double *d_lamf = nullptr, *d_muf = nullptr, *d_rhoJ = nullptr;    // per face / element (time-scaled)
    // physical copies for the energy when a time scale other than 1 is set (else null)
    double *d_lamf_ph = nullptr, *d_muf_ph = nullptr, *d_rhoJ_ph = nullptr;
    std::vector<double> alpha_e;       // per-element time scale; empty: 1 everywhere
    float *d_lamf32 = nullptr, *d_muf32 = nullptr, *d_rhoJ32 = nullptr;

    // ---- device: state (shot-major)
    double *d_vtr = nullptr, *d_sigtr = nullptr;
    double *d_b = nullptr, *d_x = nullptr;      // per shot slab RHS and solution
    double *d_sigtmp = nullptr;                  // one shot's stress trace (basis conversions)
    double *d_energy = nullptr;

    // ---- sources / receivers
    int have_sources = 0;
    std::vector<int64_t> src_elem;     // [shot][source of the shot]
    int src_per_shot = 1;
    double *d_src = nullptr;           // [shot][source]: [dim dir][Nphi phi(x_s)]
    int32_t *d_src_elem = nullptr;
    double src_f0 = 0, src_td = 0, src_a1 = 0;
    std::vector<double> src_alpha;     // time scale of each source's element (empty: 1)
    std::vector<double> src_xs, src_dir;   // host copies: [shot][source of the shot][dim]
    double* d_gl8 = nullptr;           // 8-point Gauss-Legendre rule on [0,1]: nodes, weights
    std::vector<double> lam_e, mu_e, rho_e;   // host copies of the material
    int n_rec = 0;
    int32_t *d_rec_elem = nullptr;
    double *d_rec_phi = nullptr;       // [rec][Nphi]
    double *d_records = nullptr;       // [shot][cap_steps][rec][dim]
    int64_t rec_cap_steps = 0, rec_steps = 0;

    // ---- block-Jacobi preconditioner (precond.cu)
    double *d_preV = nullptr, *d_preLam = nullptr, *d_preB = nullptr;
    float *d_preV32 = nullptr, *d_preB32 = nullptr;
    float *d_preB32t = nullptr;   // B in the lane order of the single-shot 2D p = 3 apply ([qi][a][g][b])
    int32_t* d_elem_face = nullptr;
    double pre_dt = -1.0;    // slab size the time blocks d_preB were built for
    // ---- stencil preconditioner (precond2.cu): S_i^{-1} per element, column-major
    double* d_pre2 = nullptr;
    float* d_pre2_32 = nullptr;                // FP32 copy for the FP32 solver, pre2_stride32 apart
    float* d_pre2_mma = nullptr;               // TF32-rounded tensor-core operand image (multi-shot, pre2_mma.cu)
    void* d_pre2_16 = nullptr;                 // FP16 balanced blocks H (S^-1 = diag(r) H diag(c)), single shot
    float* d_pre2_scl = nullptr;               // per element: row scales r then column scales c
    int pre2_bits = 16;                        // storage of the FP32 path's local blocks: 16 or 32
    void *d_p2y = nullptr, *d_p2t = nullptr;   // P_1 r and A P_1 r, stacked over shots (FP64-sized)
    int* d_p2status = nullptr;

    // ---- device error word: set by kernels whose bounded waits ran out (1: a copy did not
    // arrive in time; 2: a copy still in flight could not be drained).  Read and cleared by
    // take_device_error after every call that can launch such a kernel.
    int* d_err = nullptr;
    bool wait_gave_up = false;   // the last take_device_error found the word set
    bool echeck_on = false;      // energy-growth sentinel around stdg_step
    double echeck_tol = 0.0;

    int n_sm = 152;              // multiprocessors of the context's device (grid sizing)
    stdg::Tuning tune;

    // ---- solver workspace (solver.cu)
    void* ws = nullptr;

    // bookkeeping
    std::vector<long> scopes;
    int64_t last_launches = 0;   // kernel executions of the last stdg_step call    // kernels recorded per open loop-body scope (launch counting)
    size_t bytes = 0;
    std::vector<void*> allocs;
    std::vector<size_t> alloc_bytes;   // size of each entry of allocs
};

// Launch counting: every kernel launch of the library adds one to the innermost open
// scope; a loop body ends with a kernel that adds its scope's count to a device counter,
// so the total number of kernel executions is known even inside CUDA-graph while loops.
inline void note_launch(stdg_ctx* c, long k = 1) {
    if (!c->scopes.empty()) c->scopes.back() += k;
}

// Error helpers
#define STDG_FAIL(ctx, code, msg) do { (ctx)->err = (msg); return (code); } while (0)
#define STDG_CUDA(ctx, call) do { cudaError_t e_ = (call); if (e_ != cudaSuccess) { \
    (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e_); \
    return e_ == cudaErrorMemoryAllocation ? STDG_ENOMEM : STDG_ECUDA; } } while (0)

namespace stdg {
// Synchronises the context stream, reads the device error word and clears it.  Returns
// STDG_OK, or STDG_ECUDA with a message when a bounded wait gave up (the results of the
// launches since the last check are then invalid; the context stays usable).
int take_device_error(stdg_ctx* c);
int dev_alloc(stdg_ctx* c, void** p, size_t bytes);
void dev_release(stdg_ctx* c, void* p);   // frees one allocation made by dev_alloc
void dev_free_all(stdg_ctx* c);

// kernels.cu -- launchers (all on c->stream); return cudaGetLastError()
cudaError_t launch_precompute(stdg_ctx* c, const double* d_rule_v, const double* d_rule_f, int nq_v, int nq_f);
cudaError_t launch_orthonormalize(stdg_ctx* c);
cudaError_t launch_sig_convert(stdg_ctx* c, const double* in, double* out, int dir);
cudaError_t launch_to_fp32(stdg_ctx* c);
bool face_tiled_shape(const stdg_ctx* c);
int64_t face_tiled_floats(const stdg_ctx* c);
cudaError_t launch_tile_d32(stdg_ctx* c);
// y = A x (cfac scales the Schur part; 1 for the operator).  With xidx != null the input is
// x + (*xidx) * ld, the index read on the device (Krylov basis column j).
// nshots > 1: x and y hold nshots consecutive (shot-major) velocity vectors of c->nvel values.
cudaError_t launch_apply(stdg_ctx* c, double dt, const double* x, double* y, double cfac,
                         const int* xidx = nullptr, int64_t ld = 0, int nshots = 1);
cudaError_t launch_apply32(stdg_ctx* c, double dt, const float* x, float* y, double cfac,
                           const int* xidx = nullptr, int64_t ld = 0, int nshots = 1);
cudaError_t launch_face_only(stdg_ctx* c, double dt, const void* x, void* y, double cfac, int fp32);
cudaError_t launch_rhs(stdg_ctx* c, double dt, const double* dparams, int shot, double* b);
cudaError_t launch_stress_update(stdg_ctx* c, double dt, int shot, const double* x);
cudaError_t launch_traces(stdg_ctx* c, int shot, const double* x);
cudaError_t launch_receivers(stdg_ctx* c, const double* dparams, int shot);
cudaError_t launch_energy(stdg_ctx* c, int shot, double* d_out);
cudaError_t launch_project_plane_wave(stdg_ctx* c, int shot, int kind, const double* n, const double* pol,
                                      double amp, double t, const double* d_rule, int nq);
cudaError_t launch_initial_guess(stdg_ctx* c, int shot, double* x);

// operator_fast.cu: compile-time-shape face kernel; false if the shape is not specialised
template <typename R>
bool launch_face_fast(stdg_ctx* c, const R* D, const R* lamf, const R* muf, const R* x, const int* xidx, int64_t ld, R* y,
                      double scale, cudaError_t* err, int nshots = 1);

// precond.cu
cudaError_t launch_pre1_setup(stdg_ctx* c, const double* d_Rinv, const int32_t* d_elem_face, int* d_status);
cudaError_t launch_pre1_time(stdg_ctx* c, double dt);
cudaError_t launch_pre1_apply(stdg_ctx* c, const double* r, double* z, const int* ridx, int64_t ld, int nshots = 1);
cudaError_t launch_pre1_apply32(stdg_ctx* c, const float* r, float* z, const int* ridx, int64_t ld, int nshots = 1);

// precond2.cu
bool pre2_supported(const stdg_ctx* c);
// entries between consecutive FP32 blocks: (d N_phi N_gamma)^2 rounded up to 16 bytes
inline int64_t pre2_stride32(const stdg_ctx* c) {
    const int64_t N = (int64_t)c->dim * c->Nphi * c->Ng;
    return (N * N + 3) / 4 * 4;
}
cudaError_t launch_pre2_setup(stdg_ctx* c, double dt, int* d_status);
bool pre2_half_supported(const stdg_ctx* c);
cudaError_t launch_pre2_half(stdg_ctx* c);
cudaError_t launch_pre2_apply(stdg_ctx* c, const double* r, double* z, const int* ridx, int64_t ld, int nshots = 1);
cudaError_t launch_pre2_apply32(stdg_ctx* c, const float* r, float* z, const int* ridx, int64_t ld, int nshots = 1);
cudaError_t launch_pre2_local(stdg_ctx* c, int fp32, const void* r, const void* w, void* z);
cudaError_t launch_pre2_local_batch(stdg_ctx* c, const float* r, const float* w, float* z);
// pre2_mma.cu: the element-local step for a batch of shots on the tensor cores (tcgen05)
bool pre2_mma_supported(const stdg_ctx* c);
int64_t pre2_mma_image_floats(const stdg_ctx* c);
cudaError_t launch_pre2_mma_image(stdg_ctx* c);
bool launch_pre2_local_mma(stdg_ctx* c, const float* r, const int* ridx, int64_t ld, const float* w, float* z,
                           int nshots, cudaError_t* e);
// (re)build the dt-dependent preconditioner blocks when dt changes (capi.cu)
int precond_for_dt(stdg_ctx* c, double dt);

// solver.cu
int solver_setup(stdg_ctx* c);
void solver_free(stdg_ctx* c);
int solver_step(stdg_ctx* c, double dt, int n_steps, stdg_stats* st);
int solver_solve(stdg_ctx* c, double dt, stdg_stats* st);   // A x = b on the stacked d_b / d_x

// adjoint.cu
int misfit_grad_impl(stdg_ctx* c, double dt, int n_steps, const double* data, int checkpoint_every, double* loss,
                     double* g_lam, double* g_mu, double* g_rho, double* g_src, stdg_stats* stats);
// capi.cu: phi(x_s) and its physical gradient [NP][dim] for source q (host copies of the sources)
void source_basis_host(const stdg_ctx* c, int64_t q, double* phi, double* dphi);
}  // namespace stdg
