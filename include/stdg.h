/*
 * stdg.h -- C ABI of the GB300 (sm_103a) library for the staggered space-time
 * discontinuous Galerkin scheme for velocity-stress linear elasticity of
 * Tavelli & Dumbser, arXiv:1802.04516.
 *
 * The library owns all device memory it allocates.  Every pointer argument is a
 * HOST pointer unless its name ends in _dev (a device pointer the caller owns).
 * Host buffers are read or written synchronously: when a call returns, the
 * caller may reuse or free them.  All work is issued on the stream given to
 * stdg_create (NULL = the legacy default stream).
 *
 * Error behaviour: every int-returning call returns STDG_OK (0) or a negative
 * STDG_E* code; a human-readable message is then available from
 * stdg_last_error().  A failed call leaves the context usable unless the code is
 * STDG_ECUDA from a CUDA error proper (the context should then be destroyed).  One kind of
 * STDG_ECUDA leaves it usable: a kernel's bounded wait for a bulk copy that gave up (the
 * message says so); that call's results are invalid and the error is reported once.
 *
 * Layouts (row-major, contiguous):
 *   velocity, one slab      [elem][component d][time node N_gamma][space node N_phi]
 *   velocity trace          [elem][component d][space node N_phi]
 *   stress trace            [face][component s][dual mode N_psi]
 *   stress components       2D: xx, yy, xy      3D: xx, yy, zz, xy, yz, xz
 *   space nodes             equispaced Lagrange nodes of the reference simplex,
 *                           z outer, then y, x fastest
 *   dual modes              Taylor monomials ((x - x_j)/h_j)^a, |a| <= p, graded-
 *                           lexicographic (degree ascending, then x-exponent
 *                           descending, then y-exponent descending)
 *   time nodes              Gauss-Legendre points of [0,1], ascending
 *   faces                   ascending lexicographic order of the sorted global
 *                           vertex-id tuple; l(j) = smaller, r(j) = larger element
 * Multi-shot data is shot-major: [shot][...] with the per-shot layout above.
 */
#ifndef STDG_H
#define STDG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STDG_OK        0
#define STDG_EINVAL   (-1)  /* bad argument, NaN or Inf in an input                */
#define STDG_EMESH    (-2)  /* inverted element, non-manifold or self-adjacent face */
#define STDG_ENOMEM   (-3)  /* device allocation failed                             */
#define STDG_ECUDA    (-4)  /* CUDA runtime error                                   */
#define STDG_ENOTCONV (-5)  /* Krylov hit max_iters; the state is still advanced    */
#define STDG_ESTATE   (-6)  /* call out of order (e.g. step before set_mesh)        */
#define STDG_ENONFINITE (-7) /* a residual norm became NaN or Inf (e.g. an input that
                                overflows); the solve stopped, the state is advanced but
                                holds non-finite values                                 */
#define STDG_EENERGY  (-8)  /* the energy check (stdg_set_energy_check) found a shot whose
                                energy grew over a source-free stdg_step; the state is
                                advanced                                                */

enum stdg_scheme { STDG_SCHEME_CN = 0, STDG_SCHEME_STDG = 1 };
enum stdg_precision { STDG_FP64 = 0, STDG_MIXED_FP32 = 1 };

typedef struct stdg_ctx stdg_ctx;

typedef struct {
    int p;              /* spatial degree, 1..4 in 2D, 1..3 in 3D                      */
    int p_gamma;        /* time degree, 0..4; must be 0 for Crank-Nicolson             */
    int scheme;         /* stdg_scheme                                                   */
    int precision;      /* stdg_precision                                                */
    double rel_tol;     /* Krylov stop: ||b - A x||_2 <= rel_tol ||b||_2                 */
    int max_iters;      /* cap on operator applications per solve                       */
    int gmres_restart;  /* GMRES(m) restart length                                      */
    double inner_tol;   /* relative tolerance of the FP32 inner solve (mixed precision)  */
    int use_graph;      /* 1: one CUDA graph per step with device-side loops; 0: host loop */
    int preconditioner; /* 0: none; 1: block Jacobi "Pre1" (Appendix A, Eq. pre1): exact inverse of
                           every element's diagonal block, applied on the right (GMRES) or as PCG;
                           2: stencil preconditioner "Pre2" (Appendix A, Eqs. APPRE1-APPRE2): first
                           block row of the inverse of the system restricted to the element and its
                           face neighbours.  Pre2 is not symmetric, so Crank-Nicolson then runs
                           GMRES instead of CG.  Needs d N_phi N_gamma <= 128 (else STDG_EINVAL at
                           stdg_set_material); costs (d N_phi N_gamma)^2 values per element, FP64
                           in FP64 contexts and FP32 in mixed-precision ones (which keep no FP64
                           copy: the FP64 stencil apply calls are then STDG_ESTATE) plus a
                           balanced FP16 copy for one shot (stdg_set_pre2_storage).             */
} stdg_options;

typedef struct {
    int iters_total;        /* operator applications summed over the steps            */
    int iters_max;          /* largest per-step count                                 */
    int refinements;        /* FP64 refinement sweeps (mixed precision)               */
    double final_rel_res;   /* ||b - A x|| / ||b|| of the last step (FP64)            */
    int status;             /* STDG_OK, STDG_ENOTCONV or STDG_ENONFINITE              */
} stdg_stats;

/* Context.  `cuda_stream` is a cudaStream_t (may be NULL). */
int  stdg_create(stdg_ctx** out, int dim, const stdg_options* opt, void* cuda_stream);
void stdg_destroy(stdg_ctx* ctx);
const char* stdg_last_error(const stdg_ctx* ctx);

/* Mesh of simplices (Sec. 3): n_vert x dim coordinates, n_elem x (dim+1) vertex ids
 * (0-based, positively oriented after unwrapping).  `period` (dim entries, 0 = not
 * periodic) or NULL.  On a periodic axis vertices are identified, not duplicated.
 * Every boundary face is a free surface (sigma . n = 0).  Builds faces, l(j)/r(j),
 * normals, dual cells R_j and, on the device, the blocks D_{i,j} (Eq. MD_3) and the
 * Cholesky factors L_j of the dual mass matrices M_j = L_j L_j^T (Eq. MD_2); the kernels
 * use the orthonormalised blocks D_{i,j} L_j^{-T} and never form M_j^{-1}.  Replaces any
 * previous mesh (states, sources and receivers are dropped).  Returns STDG_EMESH for an
 * inverted element, a face shared by more than two elements, an element that is its own
 * neighbour or a dual mass matrix that is not positive definite; STDG_EINVAL for a bad
 * size, a vertex index out of range or a non-finite coordinate or period. */
int stdg_set_mesh(stdg_ctx* ctx, int64_t n_vert, const double* xyz, int64_t n_elem,
                  const int32_t* elem_vert, const double* period);

/* Per-element Lame parameters and density (Eq. 5, Eq. NM1), n_elem values each: rho_i
 * constant per element; E_j constant per dual cell, the sub-cell-measure-weighted mean
 * of its two elements.  Requires lambda >= 0, mu > 0, rho > 0, all finite (else
 * STDG_EINVAL); STDG_ESTATE before stdg_set_mesh.  Also sets up the preconditioner. */
int stdg_set_material(stdg_ctx* ctx, const double* lambda, const double* mu, const double* rho);

/* Per-element time scale alpha (n_elem values, > 0, finite), for disconnected parts of one
 * mesh that advance with their own time steps (a ragged batch, each part at its own CFL):
 * a stdg_step(dt) advances element i by alpha_i dt in its own time.  alpha must be the same
 * on the two elements of every face (STDG_EINVAL otherwise: a step that changes across a
 * face is local time stepping, not this scheme).  Implemented without a kernel change: with
 * tau = t / alpha the elastic system of a part is the same system with density rho / alpha
 * and Lame parameters alpha lambda, alpha mu (Eq. 5 rescaled; the slab system of Eq.
 * velocity.sys then scales by 1/alpha on both sides, the stress update of Eq. NM26 is
 * unchanged), and a point source in such a part has the Ricker wavelet of Sec. 6.3 at
 * frequency alpha f0 and delay t_delay / alpha.  States, receivers and stdg_energy stay in
 * physical units; the time of stdg_get_time is the reference time (alpha = 1).  NULL resets
 * to 1 everywhere.  Applies to the material and sources already set and to later ones;
 * STDG_ESTATE before stdg_set_mesh.  stdg_misfit_grad rejects a context with a time scale
 * other than 1 (STDG_ESTATE). */
int stdg_set_time_scale(stdg_ctx* ctx, const double* alpha);

/* Number of shots (right-hand sides).  Resets states to zero.  Default 1. */
int stdg_set_shots(stdg_ctx* ctx, int n_shots);

/* Carried state of one shot: the t^{n,-} traces (Eq. NM13), v_tr n_elem*d*N_phi and
 * sig_tr n_face*s*N_psi values in the layouts above (stress in the Taylor-monomial dual
 * basis; the library converts to its orthonormal coordinates).  STDG_EINVAL for a shot
 * outside 0..n_shots-1 or a non-finite value. */
int stdg_set_state(stdg_ctx* ctx, int shot, const double* v_tr, const double* sig_tr);
int stdg_get_state(stdg_ctx* ctx, int shot, double* v_tr, double* sig_tr);

/* Projects the exact plane wave of Eq. NT2.1/NT2.2 (unit normal n/|n|, wave vector
 * 2 pi n, amplitude amp; kind 0 = P, 1 = S with polarisation pol, NULL in 2D =
 * (-n_y, n_x)) at time t onto the bases, for one shot.  Homogeneous media only
 * (element 0's material is used). */
int stdg_set_plane_wave(stdg_ctx* ctx, int shot, int kind, const double* n, const double* pol,
                        double amp, double t);

/* Point sources (Sec. 6.3): shot k has force direction dir[k] at xs[k] (n_shots x dim
 * each) and the Ricker time function S(t) = a1 (0.5 + a2 tau^2) exp(a2 tau^2),
 * tau = t - t_delay, a2 = -(pi f0)^2.  Sets n_shots (resets states and records).
 * STDG_EINVAL for a source outside the mesh or a non-finite argument. */
int stdg_set_sources(stdg_ctx* ctx, int n_shots, const double* xs, const double* dir,
                     double f0, double t_delay, double a1);

/* Several point sources per shot (same Ricker wavelet): shot k has the sources
 * xs[k*per_shot + q], dir[k*per_shot + q], q < per_shot.  stdg_set_sources is the case
 * per_shot = 1.  A disconnected mesh with one source per part advances independent
 * problems (a ragged batch) in one shot.  Sets n_shots (resets states). */
int stdg_set_point_sources(stdg_ctx* ctx, int n_shots, int per_shot, const double* xs, const double* dir,
                           double f0, double t_delay, double a1);

/* Receivers (n_rec x dim positions): velocity v_h(x_r, t^{n+1,-}) is recorded after
 * every step; earlier records are dropped.  STDG_EINVAL for a position outside the mesh
 * (located as by stdg_locate_points) or a non-finite one. */
int stdg_set_receivers(stdg_ctx* ctx, int n_rec, const double* xr);

/* Advances every shot by n_steps slabs of size dt (Eq. velocity.sys + NM26, or the
 * Crank-Nicolson Eqs. velocity.sys.cn + NM26.cn).  `out` may be NULL.  Returns
 * STDG_ENOTCONV if some solve hit max_iters (the state is still advanced, stats filled),
 * STDG_ENONFINITE if a residual norm became NaN or Inf (the solve stops at once instead
 * of running to max_iters). */
int stdg_step(stdg_ctx* ctx, double dt, int n_steps, stdg_stats* out);

/* Simulation time of the carried state. */
int stdg_get_time(stdg_ctx* ctx, double* t);
int stdg_set_time(stdg_ctx* ctx, double t);

/* Total energy of each shot's carried state (Eq. SP3F): out[n_shots]. */
int stdg_energy(stdg_ctx* ctx, double* out);

/* Energy-growth sentinel (Sec. 5, Theorem 4: without sources the discrete energy of the
 * space-time scheme never increases from one slab to the next, and Crank-Nicolson keeps it).
 * With enable != 0, every stdg_step on a context without point sources (none set, or
 * amplitude a1 = 0) evaluates each shot's energy before and after the call and returns
 * STDG_EENERGY when E_after > (1 + rel_tol) E_before for some shot, or E_after is not finite;
 * the state, time and receiver records are advanced as for STDG_OK, and a status of the solve
 * itself (STDG_ENOTCONV, STDG_ENONFINITE, ...) takes precedence.  rel_tol > -1: 0 or a small
 * positive value allows rounding (FP64 about 1e-12, mixed precision the inner tolerance);
 * a negative value demands a decrease by that fraction.  Off by default (two energy
 * evaluations per call).  Returns STDG_OK or STDG_EINVAL (rel_tol <= -1 or not finite). */
int stdg_set_energy_check(stdg_ctx* ctx, int enable, double rel_tol);

/* Receiver records since the last stdg_set_receivers / stdg_set_sources:
 * out[n_shots][n_recorded_steps][n_rec][dim]; `cap` = capacity in doubles.
 * Returns the number of recorded steps (>= 0) or an error code. */
int stdg_read_receivers(stdg_ctx* ctx, double* out, int64_t cap);

/* y = A x for one slab of size dt (Eq. velocity.sys, or Eq. velocity.sys.cn for CN),
 * canonical velocity layout, one shot, FP64.  Host pointers. */
int stdg_apply_operator(stdg_ctx* ctx, double dt, const double* x, double* y);

/* Same on device buffers owned by the caller (FP64; or FP32 when fp32 != 0, using
 * the FP32 copy of the blocks).  Asynchronous on the context stream in FP64; the FP32
 * path synchronises the stream to check the bounded waits of its face kernel and returns
 * STDG_ECUDA if one gave up (y is then invalid; the context stays usable). */
int stdg_apply_operator_device(stdg_ctx* ctx, double dt, const void* x_dev, void* y_dev, int fp32);

/* Sizes: what = 0 n_elem, 1 n_face, 2 N_phi, 3 N_psi, 4 N_gamma, 5 stress comps s,
 * 6 n_shots, 7 velocity values per shot and slab, 8 n_rec, 9 n_boundary_faces,
 * 10 device bytes held, 11 kernel executions of the library during the last stdg_step
 * call (counted on the device, including every iteration of the device-side loops),
 * 12 bits per stored entry of the stencil preconditioner's local blocks in the FP32 inner
 * solve of one shot (16 or 32; 0 without such blocks). */
int stdg_query(stdg_ctx* ctx, int what, int64_t* out);

/* Storage of the stencil preconditioner's local blocks S_e^{-1} (Appendix A, Eq. APPRE2)
 * applied by the FP32 inner solve of a single shot: bits = 16 (default for mixed precision)
 * keeps each block balanced, S^{-1} = diag(r) H diag(c) with r_i = max_j |S_ij|,
 * c_j = max_i |S_ij| / r_i, and H in FP16 (11-bit significand, as the TF32 rounding of the
 * multi-shot tensor-core path), FP32 arithmetic: half the bytes of the slab's dominant
 * stream; bits = 32 applies the FP32 blocks.  The preconditioner only steers the Krylov
 * iteration, so the solution meets the same residual bar either way.  Shapes with an odd
 * d N_phi N_gamma or above 128 keep FP32.  Returns STDG_OK or STDG_EINVAL (bits not 16/32). */
int stdg_set_pre2_storage(stdg_ctx* ctx, int bits);

/* Face table as built by stdg_set_mesh: l(j), r(j) (-1 on the boundary). */
int stdg_get_faces(stdg_ctx* ctx, int32_t* face_l, int32_t* face_r);

/* The same face table built on the host alone, with no context and no GPU (the mesh
 * connectivity of Sec. 3: faces by sorted vertex tuples, periodic faces through the
 * period, l(j) the smaller and r(j) the larger element index, -1 on the boundary).
 * Arguments as for stdg_set_mesh (dim 2 or 3).  On entry *n_face holds the capacity of
 * face_l / face_r (0 with NULL arrays asks for the count only); on return it holds the
 * number of faces, also when the capacity was too small (then STDG_EINVAL and nothing
 * written).  Returns STDG_OK, STDG_EINVAL (bad argument, vertex index out of range,
 * non-finite coordinate) or STDG_EMESH (inverted element, a face shared by more than two
 * elements, an element adjacent to itself).  The caller owns every array. */
int stdg_mesh_faces(int dim, int64_t n_vert, const double* xyz, int64_t n_elem, const int32_t* elem_vert,
                    const double* period, int64_t* n_face, int32_t* face_l, int32_t* face_r);

/* Elements containing n_pts points (n_pts x dim, row-major), located on the host with no
 * context and no GPU by the code that places sources and receivers: the element whose
 * barycentric coordinates are all >= -1e-12, the lowest index on ties (edges, vertices),
 * periodic images folded into the element's frame; -1 for a point outside the mesh.
 * Mesh arguments as for stdg_set_mesh; elem_out (n_pts entries) is owned by the caller.
 * Returns STDG_OK, STDG_EINVAL (bad argument, non-finite point) or STDG_EMESH. */
int stdg_locate_points(int dim, int64_t n_vert, const double* xyz, int64_t n_elem, const int32_t* elem_vert,
                       const double* period, int64_t n_pts, const double* pts, int64_t* elem_out);

/* The reference tables every kernel uses, computed on the host with no context (Sec. 3
 * bases, Eqs. MD_2 - MD_2_3 time factors): Mref (N_phi x N_phi, row-major) =
 * int over the reference simplex of phi_k phi_m for the nodal P_p basis; for the
 * Lagrange time basis on the N_gamma = p_gamma + 1 Gauss-Legendre points of [0, 1]:
 * W (N_gamma, the diagonal of int gamma_a gamma_b), T (N_gamma x N_gamma) =
 * gamma(1) gamma(1)^T - K with K_ab = int gamma_a' gamma_b, S = W T^{-1} W (the time factor
 * of the Schur term), kappa = gamma(1)^T T^{-1} gamma(0) and u = gamma(1)^T T^{-1} W
 * (N_gamma; the stress-trace update sigma <- kappa sigma - dt sum_b u_b (E:g)_b).  Any
 * output may be NULL.  Returns STDG_OK or STDG_EINVAL (dim not 2 or 3, p outside 1..4 in
 * 2D or 1..3 in 3D, p_gamma outside 0..4). */
int stdg_reference_tables(int dim, int p, int p_gamma, double* Mref, double* W, double* T, double* S, double* kappa,
                          double* u);

/* z = P^{-1} r with the context's preconditioner (Pre1 or Pre2) for slab size dt
 * (canonical velocity layout, one shot, FP64, host pointers).  Requires preconditioner
 * 1 or 2; with 2, the shots must be set (stdg_set_shots or a source / state call). */
int stdg_apply_preconditioner(stdg_ctx* ctx, double dt, const double* r, double* z);

/* z_dev = P^{-1} r_dev for every shot of the context at once (stacked shot-major, n_shots x
 * velocity values per slab, canonical layout), on device buffers owned by the caller (r_dev
 * and z_dev distinct), slab size dt.  fp32 = 0: the FP64 preconditioner of the FP64 solver;
 * fp32 != 0 (mixed-precision contexts only): the FP32 one of the inner solve -- for the stencil
 * preconditioner with several shots and d N_phi N_gamma = 36, its element-local step runs on
 * the tensor cores (kind::tf32 with S^{-1} rounded to TF32 and the vector split into two TF32
 * terms).  Appendix A, Eq. pre1 (Pre1) or Eqs. APPRE1-APPRE2 (Pre2).  Synchronises the stream;
 * STDG_ESTATE without a preconditioner or shots, STDG_ECUDA if a bounded wait gave up. */
int stdg_apply_preconditioner_device(stdg_ctx* ctx, double dt, const void* r_dev, void* z_dev, int fp32);

/* Residual of the velocity system without allocating: r_dev = b_dev - A x_dev for slab
 * size dt (A as in stdg_apply_operator, FP64, one shot, canonical layout) and
 * out_dev[0] = ||r|| / ||b|| (||r|| when b = 0), out_dev[1] = ||r||.  All four pointers
 * are device memory owned by the caller.  The paper has no counterpart: this exists for
 * callers that cannot call cudaMalloc -- code running while a stream is captured into a
 * CUDA graph, pipelines that cannot afford the device-wide synchronisation of cudaFree,
 * or processes whose device memory is already reserved by another allocator.  The only
 * other memory used is a 1 MiB scratch array compiled into the library (held by every GPU
 * that loads it until exit); velocity vectors longer than 2^28 values are rejected with
 * STDG_EINVAL.  The first call on a device looks up that array's device address, so make
 * it before any stream capture.  Calls share the array: calls that overlap on the GPU race
 * and must be ordered by the caller.  r_dev must not be x_dev or b_dev (STDG_EINVAL):
 * A x is written into r_dev while x_dev is still being read.  The device address of the
 * array is looked up once per device and kept for the life of the process, so it assumes
 * the device's primary context is not reset (cudaDeviceReset) in between.  Asynchronous
 * on the context stream. */
int stdg_residual_noalloc(stdg_ctx* ctx, double dt, const double* x_dev, const double* b_dev,
                          double* r_dev, double* out_dev);

/* Receiver misfit and its gradient (full-waveform inversion).  From the current state of
 * every shot, advance n_steps slabs of size dt and return
 *   *loss = 1/2 sum_shots sum_{n=1..n_steps} sum_r |v_h(x_r, t^n) - data|^2,
 * data laid out [shot][step][receiver][component] (as stdg_read_receivers returns).  With
 * any of g_lambda, g_mu, g_rho non-NULL (host arrays of n_elem values), also the exact
 * gradient of the discrete misfit with respect to the per-element lambda, mu and rho, by
 * the adjoint of the slab map: the transposed velocity system is solved as the forward
 * system on time-reversed vectors (A^T = J A J for the reversal J of the Gauss-Legendre
 * time nodes), with the context's solver, precision and preconditioner; states are
 * checkpointed every checkpoint_every slabs (<= 0: 20) and each segment is recomputed
 * once in the backward sweep.  g_src (may be NULL): the gradient with respect to the point
 * sources of Sec. 6.3, n_shots x per_shot x (1 + 2 dim) values, for every source q (in the
 * order of stdg_set_point_sources): dL/d(amplitude of source q), dL/d(force direction, dim
 * values), dL/d(position, dim values; the source's element held fixed) -- the source enters the
 * right-hand side only, so these are lam^T ds/dtheta summed over the slabs (zeros when the
 * context has no point sources).  Space-time DG only (STDG_EINVAL for Crank-Nicolson); needs
 * receivers.  The context ends at the final time with the final states, as after
 * stdg_step; stats (may be NULL) sums the Krylov work of all forward and adjoint solves.
 * The paper has no adjoint: this is the gradient of the library's own discrete map. */
int stdg_misfit_grad(stdg_ctx* ctx, double dt, int n_steps, const double* data, int checkpoint_every,
                     double* loss, double* g_lambda, double* g_mu, double* g_rho, double* g_src, stdg_stats* stats);

/* Average device time of `n` launches of the operator's face kernel (fp32 != 0: the
 * FP32 one) on the context stream, measured with CUDA events: *ms_out. */
int stdg_time_operator(stdg_ctx* ctx, double dt, int fp32, int n, double* ms_out);

/* Average device time of one launch of a single kernel, over n back-to-back launches on
 * the context's stream (CUDA events), for roofline figures.  which: 0 face term of the
 * operator (as stdg_time_operator), 1 block-Jacobi apply, 2 the element-local step of the
 * stencil preconditioner (z = S^{-1} (2 r - w)), 3 the whole operator (mass + face), 4 the
 * element-local step for all the context's shots at once (FP32 only; the tensor-core kernel
 * where it applies).
 * fp32 selects the FP32 blocks (mixed-precision contexts only for 1 and 2).  Timing only:
 * the kernels run on zero vectors in buffers allocated for the call.  No counterpart in
 * the paper. */
int stdg_time_kernel(stdg_ctx* ctx, double dt, int which, int fp32, int n, double* ms_out);

/* Launch shapes chosen by the library's autotuner (no counterpart in the paper). */
typedef struct {
    int face_warps_per_block;   /* face kernels of the operator: warps per block (1, 2, 4)            */
    int face_blocks_per_sm;     /* single-shot bulk-copy face kernel: grid cap, blocks per SM         */
    int face_register_cap;      /* single-shot bulk-copy face kernel: 1 register cap for occupancy, 0 none */
    int pre2_warps_per_block;   /* CUDA-core element-local step of the stencil preconditioner         */
    int mma_ctas_per_sm;        /* tensor-core element-local step (a batch of shots): CTAs per SM (1, 2) */
    double face_ms, pre2_ms;    /* best time per launch of the tuned face kernel / local step (0: not tuned) */
    int candidates;             /* configurations timed                                               */
} stdg_tuning;

/* Autotuner: times every candidate launch shape of the hot kernels this context runs for slab
 * size dt -- the FP32 face kernel (mixed precision; warps per block 1/2/4 and, for one shot, the
 * grid cap 8/16/32/64 blocks per SM and the kernel compiled with or without a register cap) and the element-local step of the stencil preconditioner
 * (warps per block, or CTAs per SM of the tensor-core kernel) -- on the context's own mesh and
 * shot count (zero vectors, 10 launches each, CUDA events) and keeps the fastest for every later
 * launch; step graphs captured before are dropped and re-captured.  `out` (may be NULL) receives
 * the choices.  Allocates three scratch vectors for the call.  Results do not depend on the
 * choice beyond the order of floating-point atomics. */
int stdg_autotune(stdg_ctx* ctx, double dt, stdg_tuning* out);

/* Arithmetic peak of this GPU (no counterpart in the paper): the FP64 (fp64 != 0) or FP32 FMA
 * rate in TFLOP/s (2 flops per FMA) that the library's own probe kernel sustains -- 8 independent
 * FMA chains per thread, 8 blocks of 256 threads per SM, timed with CUDA events on a private
 * stream -- the denominator of the ALU-bound rooflines.  Needs no context; allocates and frees
 * its own output buffer.  Returns STDG_OK, STDG_EINVAL (null out), STDG_ENOMEM or STDG_ECUDA. */
int stdg_measure_fma_peak(int fp64, double* tflops);

/* Failure-path testing (no counterpart in the paper): sets the context's device error word
 * exactly as a face kernel whose bounded wait for a bulk copy gave up would.  The next call
 * that checks the word (stdg_step, stdg_misfit_grad, the FP32 stdg_apply_operator_device,
 * stdg_time_kernel) returns STDG_ECUDA once and clears it; stdg_step still advances the time
 * and the receiver records, since the graph ran.  No kernel is made to fail. */
int stdg_inject_wait_error(stdg_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* STDG_H */
