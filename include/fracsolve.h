/*
 * fracsolve: GB300 (sm_103a) solve phase of the stabilised 3x3 block
 * Jacobian of frictional contact mechanics with fracture flow
 * (A. Franceschini, L. Gazzola, M. Ferronato, "A scalable preconditioning
 * framework for stabilized contact mechanics with hydraulically active
 * fractures", arXiv 2112.12397).
 *
 *   J = [ A   C1  Q1 ]      unknowns  [u; t; p]           (Eq. JacSys)
 *       [ C2  -H  0  ]      u: 3 per node copy, global frame
 *       [ Q2  0   T  ]      t: 3 per fracture face, local frame (n, t1, t2)
 *                           p: 1 per fracture face
 *
 * The library builds the preconditioners of Alg. 1 (t-p-u) and Alg. 3
 * (t-u-p) on the GPU, applies them as in Alg. 2 and Alg. 4 with inner
 * smoothed-aggregation AMG V-cycles, and solves J x = b by right-preconditioned
 * flexible GMRES with classical Gram-Schmidt applied twice (Sec. 4: zero
 * initial guess, stop on relative residual).
 *
 * Conventions for every entry point:
 *  - Return value: an fc_status code (FC_OK on success).  Nothing throws or
 *    aborts across this boundary.  fc_last_error() gives a message for the
 *    most recent failure of a context.
 *  - Pointers named d_* are DEVICE pointers on the context's device; pointers
 *    named h_* are HOST pointers.  The caller owns every buffer it passes;
 *    the library never frees or keeps caller memory after a call returns.
 *  - Work is issued on the CUDA stream given to fc_create; calls that
 *    return results to the host synchronise that stream.
 *  - Vectors have length n = 3 n_node + 3 n_face + n_face in the order
 *    [u; t; p] (u node-major x,y,z; t face-major N,T1,T2; p per face).
 */
#ifndef FRACSOLVE_H
#define FRACSOLVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FC_OK = 0,
  FC_NOT_CONVERGED = 1,   /* maxit reached; iters and relres are filled */
  FC_BREAKDOWN = 2,       /* Krylov breakdown before reaching tol */
  FC_SINGULAR_BLOCK = 3,  /* a singular H~ block, AMG diagonal block or
                             coarse matrix */
  FC_NAN = 4,             /* NaN or Inf met in the input or an iterate */
  FC_BAD_ARG = 5,         /* invalid sizes, pointers, variant or options */
  FC_CUDA_ERROR = 6,      /* a CUDA runtime call failed */
  FC_OOM = 7,             /* device allocation failed */
  FC_INTERNAL = 8,        /* a capacity limit of a setup kernel was hit */
  FC_NOT_SETUP = 9        /* fc_setup has not built what the call needs */
} fc_status;

/* Variants of the block preconditioner (Sec. 3).  FC_TUP_STAR is the
 * incomplete t-u-p factorisation D2^-1 L2^-1 of Eq. P2 (the remark after
 * Prop. 3.2): one S1 V-cycle per application instead of two.  It uses the
 * t-u-p setup, so bit FC_TUP of fc_options.variants builds it. */
enum { FC_TPU = 0, FC_TUP = 1, FC_TUP_STAR = 2 };

/* Precision modes. FP64: everything in double.  MIXED: the AMG hierarchies,
 * smoothers, H~^-1 and the coupling blocks used inside the preconditioner are
 * stored and applied in float; the outer Krylov method (J z, Arnoldi,
 * Givens, solution update, true residual) and the coarsest dense solve stay
 * in double. */
enum { FC_FP64 = 0, FC_MIXED = 1 };

/* Block sparse row matrix (row-major dense blocks of br x bc), DEVICE
 * pointers.  Columns must be sorted and unique within each block row.  Used
 * for the seven blocks of Eq. block_def:
 *   A  n_node x n_node 3x3;  C1 n_node x n_face 3x3;  Q1 n_node x n_face 3x1;
 *   C2 n_face x n_node 3x3;  H  n_face x n_face 3x3;  Q2 n_face x n_node 1x3;
 *   T  n_face x n_face 1x1. */
typedef struct {
  int32_t n_brows, n_bcols, br, bc;
  int64_t nnzb;
  const int32_t *d_row_ptr;   /* n_brows + 1 */
  const int32_t *d_col_idx;   /* nnzb */
  const double *d_val;        /* nnzb * br * bc */
} fc_bsr;

typedef struct {
  fc_bsr A, C1, Q1, C2, H, Q2, T;
  int32_t n_node, n_face;
} fc_blocks;

/* Solver options.  The AMG settings define the smoothed-aggregation
 * hierarchy (strength threshold theta0 * theta_decay^level on block
 * Frobenius norms, distance-2 maximal independent set roots with SplitMix64
 * priorities drawn from amg_seed, one Jacobi smoothing step of the
 * tentative prolongator with omega = omega_num / lambda, Galerkin coarse
 * operators, dense coarsest solve) and its V(1,1)-cycle with a Chebyshev
 * smoother of degree cheb_degree on [cheb_lo * cheb_hi * lambda,
 * cheb_hi * lambda]. */
typedef struct {
  int32_t precision;        /* FC_FP64 or FC_MIXED */
  int32_t variants;         /* bit FC_TPU and/or bit FC_TUP to build */
  double theta0, theta_decay;
  int32_t coarse_max;       /* block rows of the coarsest elasticity level */
  int32_t coarse_max_p;     /* rows of the coarsest pressure level */
  int32_t max_levels;
  double max_ratio;         /* stop coarsening when n_c > max_ratio * n */
  int32_t power_steps;
  double omega_num;
  int32_t cheb_degree;
  double cheb_hi, cheb_lo;
  uint64_t amg_seed;
  int32_t max_restarts;     /* MIXED: true-residual restarts allowed */
  int32_t verbose;
  int32_t coarse_graphs;    /* 1: the coarse levels (1 ..) of every V-cycle run as one
                             * CUDA graph, captured at the first cycle; 0: launched one
                             * by one.  Same kernels and results either way. */
} fc_options;

typedef struct fc_ctx fc_ctx;

/* Fill *opt with the defaults (FP64, both variants, theta0 0.08, decay 0.5,
 * coarse_max 200, coarse_max_p 200, 12 levels, ratio 0.8, 15 power
 * steps, omega_num 4/3, Chebyshev degree 2 on [0.11, 1.1] * lambda,
 * 3 restarts, coarse_graphs 1). */
void fc_default_options(fc_options *opt);

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *ctx receives the new
 * context; free it with fc_destroy. */
int fc_create(fc_ctx **ctx, const fc_options *opt, void *cuda_stream);

/* Alg. 1 (cpt_tpu) and/or Alg. 3 (cpt_tup): H~ = Bdiag(H,3) and its inverse,
 * S1 = A + C1 H~^-1 C2 (Eq. Schur1_2), S~ = S1 - Q1 diag(T)^-1 Q2
 * (Eq. appSchur_1), S~2 = T - FS(Q2, S1, Q1) (Eq. app_Schur2_2,
 * Eq. FS_algebraic), and the AMG hierarchies of S~ and T (t-p-u) or S1 and
 * S~2 (t-u-p).  The blocks are deep-copied: the caller may free them when
 * this returns.  Calling it again replaces the operator.  Every block's
 * structure is checked on the device before use (row pointers from 0 to
 * nnzb, non-decreasing; columns in range and strictly increasing per row).
 * The contact states take no argument of their own: they are carried by the
 * blocks (the rows of C2 and Q2 and the blocks of H, Eq. block_def).
 * Errors: FC_BAD_ARG (inconsistent sizes, row pointers or columns),
 * FC_SINGULAR_BLOCK, FC_OOM, FC_INTERNAL, FC_CUDA_ERROR. */
int fc_setup(fc_ctx *ctx, const fc_blocks *J);

/* fc_setup with every array of J (row pointers, columns, values of the
 * seven blocks) in HOST memory: the library copies them to the device on the
 * context's stream (asynchronously from pinned memory) and keeps the copies
 * as its own.  The caller guarantees that each host array holds the entries
 * its sizes state.  Same checks, errors and results as fc_setup. */
int fc_setup_host(fc_ctx *ctx, const fc_blocks *J);

/* Replace the algebraic fixed stress of S~2 (Eq. FS_algebraic) by the
 * geometric one (Eq. FS, the cheaper form the paper starts from) at the next
 * fc_setup or fc_update: [S_K]_k = -omega[k] / (kbar[k] dt) on faces whose
 * row of Q2 holds a nonzero entry, 0 elsewhere, S~2 = T - S_K.  omega[k] is
 * the volume of the cells around face k, kbar[k] their bulk modulus, dt the
 * time step of the flow equation (the sign and 1/dt follow Q2 = -Q1^T / dt
 * on open faces).  Device arrays of n_face doubles, copied; call after the
 * first fc_setup (the face count is taken from it).  omega == NULL restores
 * the algebraic form.  Errors: FC_BAD_ARG (kbar NULL, dt <= 0), FC_NOT_SETUP
 * (no fc_setup yet, or no faces); a later fc_setup with another face count
 * fails with FC_BAD_ARG until this is reset. */
int fc_set_geometric_fs(fc_ctx *ctx, const double *d_omega, const double *d_kbar, double dt);

/* Numeric refresh of the last fc_setup for new block values with exactly the
 * same sparsity patterns and sizes (the same mesh and contact states: the
 * next Newton iteration of an active set, or new apertures and pressures
 * that change T and Q2; the paper's outer loop, Sec. 2, recomputes J while
 * A, C1, Q1 stay fixed).  H~^-1, S1, S~ / S~2 and the fixed stress are
 * recomputed as in fc_setup.  Each AMG hierarchy whose level-0 operator
 * changed is rebuilt numerically on its kept aggregates and patterns: no
 * strength graph, no aggregation, no symbolic products; D^-1, lambda, the
 * smoothed prolongator values, R, the Galerkin products, the coarsest
 * inverse and the cycle data are recomputed.  A hierarchy whose operator is
 * bitwise unchanged is kept.  The blocks are read, not kept.
 * Errors: FC_NOT_SETUP before a completed fc_setup; FC_BAD_ARG when a size
 * or a block's pattern differs (call fc_setup instead); FC_SINGULAR_BLOCK,
 * FC_OOM, FC_INTERNAL, FC_CUDA_ERROR as fc_setup (the context then needs a
 * new fc_setup). */
int fc_update(fc_ctx *ctx, const fc_blocks *J);

/* d_y = J d_x (Eq. JacSys), double, device vectors of length n. */
int fc_spmv(fc_ctx *ctx, const double *d_x, double *d_y);

/* d_r = d_b - J d_x (double, device vectors of length n, caller-owned) and
 * *relres = ||d_r|| / ||d_b|| (||d_r|| when b = 0).  The reduction uses
 * partial sums held by the context.  FC_NAN if the norm is not finite. */
int fc_residual(fc_ctx *ctx, const double *d_b, const double *d_x, double *d_r, double *relres);

/* The relative residual ||d_b - J d_x|| / ||d_b|| (||.|| when b = 0) written
 * to *relres, computed without allocating anything: for callers that may not
 * call cudaMalloc at this point (a device-memory budget fixed up front, or
 * stream work that a cudaFree would synchronise).  The paper has no
 * counterpart: it is a no-allocation variant of fc_residual.
 * Scratch: the residual vector and the reduction partials live in file-scope
 * device arrays of the library (8 MiB + 4 KiB, held on every GPU that loads it
 * until the process exits).  Limit: n <= 1048576, else FC_BAD_ARG.  The first
 * call on a device looks up the arrays' device addresses (set-up, once per
 * device), so make that first call before any stream capture.  J x is formed
 * by the same product as fc_spmv.  The call synchronises the context's stream
 * before it returns (the norm is read on the host).  Every call reuses the
 * same arrays and overwrites them; calls that overlap on the GPU (other
 * streams, other contexts of the same device) race on them. */
int fc_residual_noalloc(fc_ctx *ctx, const double *d_b, const double *d_x, double *relres);

/* d_v = M^-1 d_w: app_tpu (Alg. 2) for FC_TPU, app_tup (Alg. 4) for FC_TUP,
 * D2^-1 L2^-1 (Eq. P2 without its first factor) for FC_TUP_STAR; device
 * vectors of length n. */
int fc_apply_prec(fc_ctx *ctx, int variant, const double *d_w, double *d_v);

/* Solve J x = b by right-preconditioned FGMRES-CGS2 with x0 = 0 (Sec. 4).
 * Stops when the recurrence residual drops below tol * ||b||; returns the
 * true relative residual ||b - J x|| / ||b|| in *relres and the number of
 * preconditioner applications in *iters.  d_x is output only.
 * maxit must lie in [1, 4000].  Returns FC_NOT_CONVERGED when maxit is reached
 * (x, iters, relres filled).  In FC_MIXED mode the method restarts from the
 * current x (at most max_restarts times) while the double-precision true
 * residual is above tol. */
int fc_solve(fc_ctx *ctx, int variant, const double *d_b, double *d_x, double tol,
             int maxit, int *iters, double *relres);

/* Same as fc_solve with HOST right-hand side and solution: copies h_b to the
 * device, solves, copies the solution back to h_x.  Pinned host memory makes
 * the copies asynchronous. */
int fc_solve_host(fc_ctx *ctx, int variant, const double *h_b, double *h_x, double tol,
                  int maxit, int *iters, double *relres);

/* ---------------- seeded instances assembled on the device ---------------- */

/* Fracture layouts of the synthetic unit-cube workloads (stand-ins for the
 * paper's test meshes, Sec. 4): one x-plane through the centre; three central
 * planes; n_rect seeded axis-aligned rectangles (extents 0.2-0.8 of the side);
 * full planes every `spacing` cells on all three axes. */
enum { FC_GEN_PLANE_X = 0, FC_GEN_PLANES_XYZ = 1, FC_GEN_RECTS = 2, FC_GEN_NETWORK = 3 };

/* Generator parameters.  Contact state per face: stick with probability
 * p_stick, slip with p_slip, open otherwise.  Young's modulus per cell
 * E0 exp(sigma_E Z) (median 10 GPa); aperture per face 1e-3 exp(aperture_sigma Z)
 * m unless d_aperture is given; current pressure p^l = pl_scale U MPa.
 * beta scales the stabilisation tensor and k = Ebar / (k_scale h)
 * (<= 0: the defaults 1/4 and 8). */
typedef struct {
  int32_t N;                 /* cells per side of the unit cube, [2, 1024] */
  int32_t layout;            /* FC_GEN_* */
  int32_t n_rect;            /* FC_GEN_RECTS: number of rectangles */
  int32_t spacing;           /* FC_GEN_NETWORK: cells between planes */
  double p_stick, p_slip;
  double sigma_E, aperture_sigma, pl_scale;
  double beta, k_scale;
  const double *d_aperture;  /* optional DEVICE array of n_aperture apertures (m),
                                one per fracture face in face order; NULL: drawn */
  int32_t n_aperture;        /* must equal the layout's face count when d_aperture is set */
} fc_gen_config;

/* One assembled instance.  Every pointer is DEVICE memory owned by the
 * instance (free it with fc_instance_free).  J feeds fc_setup directly. */
typedef struct {
  fc_blocks J;               /* the seven blocks of Eq. block_def */
  const double *d_b;         /* right-hand side, U(-1, 1), 0 on roller dofs; length n */
  int64_t n;                 /* 3 n_node + 4 n_face */
  int32_t n_node, n_face, grid_n;
  double h, dt, nu;          /* cell size, flow time step, Poisson ratio */
  const int8_t *d_state;     /* n_face: 0 stick, 1 slip, 2 open */
  const int8_t *d_dirichlet; /* 3 n_node: 1 on roller dofs */
  const double *d_aperture;  /* n_face (m) */
  const double *d_pl;        /* n_face: current pressures p^l (MPa) */
  const double *d_ebar;      /* n_face: mean Young's modulus of the two cells (MPa) */
  const int32_t *d_face_geom;   /* 4 n_face: normal axis, plane, in-plane cell p, q */
  const int32_t *d_face_copies; /* 8 n_face: node copies of the minus side (corners 0-3), then plus */
  const int32_t *d_node_grid;   /* n_node: grid node i + (N+1)(j + (N+1) k) of each copy */
  void *owner;               /* library-internal */
} fc_instance;

/* Defaults of the four workload families for grid size N (the paper's state
 * mix 60/30/10, sigma_E 1, lognormal apertures; one all-stick plane with
 * sigma_E 0.5 and a = 1e-3 m; ten rectangles; planes every 8 cells with
 * 50/40/10). */
void fc_default_gen_config(fc_gen_config *cfg, int layout, int N);

/* Assemble a seeded instance on the device, on `cuda_stream` (NULL: legacy
 * default stream), synchronising it before returning: the unit cube of N^3
 * trilinear hexahedra with rollers on its faces; fracture faces of the
 * layout; grid nodes split across them (one copy per group of cells joined
 * through unfractured faces, Sec. 2.2); the blocks A, C1, Q1, C2, H, Q2, T of
 * Eq. block_def for the drawn contact states (Eq. C2def, Eq. Hdef, Eq. Q2def
 * with Eq. Q2vsQ1, Eq. Tdef); b.  Counter-based draws: the result depends only
 * on (cfg, seed).  *out receives the instance.  Errors: FC_BAD_ARG (sizes,
 * layout, probabilities, n_aperture), FC_OOM, FC_CUDA_ERROR;
 * fc_generate_error() describes the last failure of this thread. */
int fc_generate(const fc_gen_config *cfg, uint64_t seed, void *cuda_stream, fc_instance **out);
const char *fc_generate_error(void);
void fc_instance_free(fc_instance *inst);

/* ---------------- adjoint (transposed system) ---------------- */
/* The adjoint data (transposed blocks, transposed preconditioner blocks and
 * transposed AMG cycles) is built on the first adjoint call after fc_setup. */

/* d_y = J^T d_x (double, device, length n). */
int fc_spmv_adjoint(fc_ctx *ctx, const double *d_x, double *d_y);

/* d_v = M^-T d_w: the transposes of the block factorisations of Eq. P1
 * (FC_TPU), Eq. P2 (FC_TUP) or its incomplete form L2^-T D2^-T
 * (FC_TUP_STAR), factors applied in reverse order, with the
 * transposed V-cycle for S~ / S1 (the V-cycles of the symmetric T and S~2 are
 * symmetric). */
int fc_apply_prec_adjoint(fc_ctx *ctx, int variant, const double *d_w, double *d_v);

/* Solve J^T lambda = g by right-preconditioned FGMRES-CGS2 with M^-T, same
 * stopping rule and return values as fc_solve.  The Krylov basis of the
 * forward solve is not used (it is recomputed, not stored). */
int fc_solve_adjoint(fc_ctx *ctx, int variant, const double *d_g, double *d_lambda, double tol,
                     int maxit, int *iters, double *relres);

/* Aperture gradient of an objective L(x) given the forward solution d_x and
 * the adjoint d_lambda (J^T lambda = dL/dx):
 *   d_grad[f] = -lambda^T (dJ/da_f) x,   f = 0 .. n_face-1,
 * through the transmissibility T and the coupling Q2 (their entries carry
 * the apertures: cubic-law conductivity, TPFA averages, flux derivatives).
 * dJ/da arrives as entries sorted by face, DEVICE arrays: face_ptr (n_face+1,
 * int64) delimits the entries of each face; entry e is d J[row, col]/d a_f =
 * val with block[e] = 0 for T (row, col faces; comp unused) or 1 for Q2 (row a
 * face, (col, comp) = (node copy, component)).  The entry arrays hold
 * face_ptr[n_face] elements, owned by the caller.  Deterministic.
 * Errors: FC_NOT_SETUP before fc_setup; FC_BAD_ARG for NULL arrays, a face_ptr
 * that does not start at 0 or decreases, or an entry whose row, column, block
 * or component lies outside the system (checked on the device; d_grad is then
 * unspecified). */
int fc_aperture_gradient(fc_ctx *ctx, const int64_t *d_face_ptr, const int8_t *d_block,
                         const int32_t *d_row, const int32_t *d_col, const int8_t *d_comp,
                         const double *d_val, const double *d_x, const double *d_lambda, double *d_grad);

/* ---------------- inspection (used by the parity tests) ---------------- */

/* Hierarchies: FC_H_TPU_U = AMG of S~, FC_H_TPU_P = AMG of T,
 * FC_H_TUP_U = AMG of S1, FC_H_TUP_P = AMG of S~2. */
enum { FC_H_TPU_U = 0, FC_H_TPU_P = 1, FC_H_TUP_U = 2, FC_H_TUP_P = 3 };
/* Matrices: level operators of a hierarchy and the setup products. */
enum { FC_M_LEVEL = 0, FC_M_PROLONG = 1, FC_M_S1 = 2, FC_M_STILDE = 3, FC_M_S2TILDE = 4 };

/* Number of levels of hierarchy `hier` (0 if it was not built). */
int fc_num_levels(fc_ctx *ctx, int hier, int *levels);

/* Copy a matrix to HOST buffers.  kind FC_M_LEVEL / FC_M_PROLONG select the
 * operator / prolongator of `level` of `hier` (in double, as built before any
 * cast); FC_M_S1 / FC_M_STILDE / FC_M_S2TILDE ignore hier and level.  Pass
 * NULL buffers to query the sizes only. */
int fc_get_bsr(fc_ctx *ctx, int kind, int hier, int level, int32_t *n_brows,
               int32_t *n_bcols, int32_t *br, int32_t *bc, int64_t *nnzb,
               int32_t *h_row_ptr, int32_t *h_col_idx, double *h_val);

/* Aggregate index of every block row of `level` (-1: no coarse unknown) and
 * the power-iteration estimate lambda of D^-1 S on that level, to HOST. */
int fc_get_aggregates(fc_ctx *ctx, int hier, int level, int32_t *h_agg, double *h_lambda);

/* One V-cycle of hierarchy `hier` applied to the device vector d_f (length =
 * scalar rows of level 0), result in d_x. */
int fc_vcycle(fc_ctx *ctx, int hier, const double *d_f, double *d_x);

/* One transposed V-cycle (B^T) of hierarchy `hier` on device vectors. */
int fc_vcycle_adjoint(fc_ctx *ctx, int hier, const double *d_f, double *d_x);

/* The orthonormal Arnoldi basis V_0 .. V_{nvec-1} left by the last FGMRES
 * cycle of fc_solve / fc_solve_adjoint (Sec. 4), row-major nvec x n doubles,
 * copied to d_V (DEVICE, caller-owned) unless d_V is NULL; *nvec receives
 * the count (0 before any solve). */
int fc_krylov_basis(fc_ctx *ctx, int *nvec, double *d_V);

/* The fixed-stress diagonal [S_K]_k of Eq. FS_algebraic to HOST (n_face). */
int fc_get_fixed_stress(fc_ctx *ctx, double *h_sk);

/* ---------------- measurement ---------------- */

/* Kernels timed with CUDA events on the context's stream while profiling is
 * on: FC_K_SMOOTH0 = one fused Chebyshev step on the finest level of the
 * elasticity hierarchy (S1 or S~); FC_K_JAC = one product J z (all seven
 * blocks); FC_K_CGS = one classical Gram-Schmidt pass (dots + update);
 * FC_K_PREC = one preconditioner application; FC_K_VCYCLE = one V-cycle of
 * the elasticity hierarchy inside t-u-p (first of the two); FC_K_RESID0,
 * FC_K_RESTRICT0 = residual and restriction on the finest level;
 * FC_K_PROLONG0 = the finest level's prolongation fused with its first
 * post-smoothing step (one pass over P and S P); FC_K_COARSE0 = everything
 * below the finest level;
 * FC_K_VCYCLE_P = the pressure V-cycle of t-u-p. */
enum {
  FC_K_SMOOTH0 = 0, FC_K_JAC = 1, FC_K_CGS = 2, FC_K_VCYCLE = 3, FC_K_PREC = 4, FC_K_RESID0 = 5,
  FC_K_RESTRICT0 = 6, FC_K_PROLONG0 = 7, FC_K_COARSE0 = 8, FC_K_VCYCLE_P = 9
};

/* Turn event timing on (enable != 0) or off, clearing what was recorded. */
int fc_profile(fc_ctx *ctx, int enable);

/* Launches recorded for `kernel`, their summed duration in ms, and the sum of
 * their algorithmic bytes (matrix values and indices plus each vector entry
 * read or written once).  Synchronises on the recorded events. */
int fc_kernel_stats(fc_ctx *ctx, int kernel, int64_t *launches, double *total_ms, double *bytes);

/* Number of kernel launches this library has issued in the process. */
unsigned long long fc_launch_count(void);

void fc_destroy(fc_ctx *ctx);
const char *fc_strerror(int status);
const char *fc_last_error(fc_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
