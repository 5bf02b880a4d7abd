/*
 * tobk.h — C-ABI of the GB300 multilevel linearized-buckling solver library (libtobk.so).
 *
 * The library implements, with hand-written CUDA kernels for sm_103a, the solver path of the
 * multilevel buckling method of Ferrari & Sigmund ("Towards solving large-scale topology
 * optimization problems with buckling constraints at the cost of linear analyses",
 * arXiv 1909.13585):
 *   - the linear analysis (LA) K[x] u = f by multigrid-preconditioned CG (Algorithm 1, step 2;
 *     Appendix A "mgPCG"),
 *   - the stress stiffness G[x, u] (Sec. 2),
 *   - the buckling load factors and modes, either exactly on the fine grid (Algorithm 1, EA) or by
 *     the multilevel procedure of Sec. 2.1 (coarse Galerkin eigenproblem, prolongation, one fine
 *     block solve K Phi = G Psi, Rayleigh quotients),
 *   - the adjoint systems K z_i = phi_i^T (grad_u G) phi_i and the sensitivities of the load factors
 *     and of the compliance (Sec. 2, eq. SensitivityLambda / AdjointSystem).
 *
 * Problem model.  A structured grid of nel[0] x nel[1] (x nel[2]) unit elements: bilinear Q4 in plane
 * stress (dim = 2, unit thickness) or trilinear H8 (dim = 3), unit element size, Young's modulus
 * interpolated per element by SIMP (Sec. 2): E_kappa = Emin + x^p (E0 - Emin) for K and
 * E_sigma = x^p E0 for G.
 *
 * Layouts (all arrays FP64 unless stated):
 *   element (i,j,k) has index e = i + nel[0] * (j + nel[1] * k)                       [m elements]
 *   node    (i,j,k) has index a = i + (nel[0]+1) * (j + (nel[1]+1) * k)
 *   DOF c of node a is dim * a + c (node-interleaved)                                   [n DOFs]
 *   blocks of vectors are stored vector after vector ([count][n]).
 * Dirichlet DOFs are given by a byte mask (1 = fixed, u = 0); every vector the library returns is
 * zero at fixed DOFs.
 *
 * Ownership and calling conventions.  The caller owns every buffer it passes; "on_device" flags say
 * whether a pointer is a device pointer (the handle's device) or host memory.  The library owns its
 * internal device memory (one allocation per handle, made by tobk_create).  All work is issued on the
 * CUDA stream given to tobk_create; functions return after their results are available to the caller
 * (host outputs are copied, device outputs are complete on that stream).  No C++ exception crosses
 * this interface.  Every function returns a tobk_status; on failure tobk_last_error() gives a
 * message.  Calls must follow the order of the method: set densities, load and fixed DOFs ->
 * solve_equilibrium -> compute_buckling -> compute_sensitivities; otherwise TOBK_E_STATE.
 * A handle must not be used from two threads at once.
 */
#ifndef TOBK_H_
#define TOBK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TOBK_OK = 0,
  TOBK_E_ARG = 1,            /* invalid argument (sizes, NaN/out-of-range densities, null pointers) */
  TOBK_E_STATE = 2,          /* call out of order (e.g. buckling before equilibrium) */
  TOBK_E_NOMEM = 3,          /* device allocation failed */
  TOBK_E_CUDA = 4,           /* a CUDA call failed; the message names it */
  TOBK_E_NOT_CONVERGED = 5,  /* iteration limit reached; outputs hold the last iterate */
  TOBK_E_BREAKDOWN = 6,      /* CG breakdown (p^T K p <= 0): K not positive definite on the free DOFs */
  TOBK_E_TIMEOUT = 7,        /* a bounded device wait expired (tensor-core inference) */
  TOBK_E_NONFINITE = 8       /* a NaN/Inf appeared in an iterate */
} tobk_status;

typedef enum {
  TOBK_FP64 = 0,             /* every multigrid operation in FP64 (plain mgPCG) */
  TOBK_FP32_VCYCLE = 1       /* V-cycle (smoother, transfers, coarse matvecs) in FP32 storage and
                                arithmetic as the preconditioner of FP64 flexible CG; the coarsest
                                dense solve, residuals, dot products and updates stay FP64 */
} tobk_precision;

typedef enum {
  TOBK_FIELD_U = 0,          /* displacement u [n] */
  TOBK_FIELD_MODES = 1,      /* buckling modes [q][n], phi_i^T K phi_j = delta_ij */
  TOBK_FIELD_ADJOINT = 2,    /* adjoint solutions z_i [q][n] */
  TOBK_FIELD_ADJOINT_RHS = 3, /* adjoint right-hand sides phi_i^T (grad_u G) phi_i [q][n] (with
                                 consistent_sens: the combined right-hand sides g_i, see
                                 tobk_compute_sensitivities) */
  /* consistent sensitivities only (desc.consistent_sens = 1, multilevel path), each [q][n] in the order
   * and on the scale of the modes: */
  TOBK_FIELD_FINE_ADJOINT = 4,   /* w_i, K w_i = (K + lambda_i G) phi_i */
  TOBK_FIELD_COARSE_ADJOINT = 5, /* P c_i, the coarse adjoint prolongated to Omega_1 */
  TOBK_FIELD_PROLONGATED = 6     /* Psi_i = P psi_i with K phi_i = G Psi_i */
} tobk_field;

typedef struct {
  int dim;           /* 2 (Q4 plane stress) or 3 (H8) */
  int nel[3];        /* elements per axis; nel[2] ignored in 2D.  Each axis divisible by 2^(mg_levels-1) */
  double nu;         /* Poisson ratio (0.3 in the paper, Sec. 2) */
  double E0;         /* solid Young's modulus (paper's E_1) */
  double Emin;       /* void modulus of the stiffness interpolation (paper's E_0; E1/E0 = 1e6) */
  double penal;      /* SIMP exponent p */
  int mg_levels;     /* multigrid levels (1 = fine grid only; the coarsest level is solved densely,
                        at most 6000 DOFs) */
  int eig_level;     /* 1-based level of the buckling eigenproblem: 1 = exact LBA on the fine grid
                        (Algorithm 1), l > 1 = multilevel procedure of Sec. 2.1 with Omega_l */
  int num_modes;     /* q, number of buckling modes / load factors (<= 24) */
  int precision;     /* tobk_precision of the V-cycle */
  double rtol;       /* CG stop: ||f - K u||_2 / ||f||_2 <= rtol over free DOFs (e.g. 1e-8) */
  int max_iter;      /* CG iteration limit per solve */
  double omega;      /* damped-Jacobi weight (e.g. 0.6) */
  int nu_pre;        /* pre-smoothing sweeps per level (>= 1) */
  int nu_post;       /* post-smoothing sweeps per level */
  double eig_tol;    /* eigenpair residual ||(K + lam G) phi|| / ||K phi|| target (1e-8, Appendix A) */
  int eig_max_iter;  /* outer iterations of the block eigensolver */
  int max_rhs;       /* largest multi-RHS block the caller will pass to tobk_solve (>= 1) */
  int eig_inner_iters; /* eigensolver preconditioner: 0 = one V-cycle, k > 0 = k mgPCG iterations */
  int fuse_load_adjoint; /* 1: tobk_compute_sensitivities solves K [u, Z] = [f, B] as one (q+1)-RHS
                            block (the load re-solved beside the q adjoint systems, u replaced by the
                            new solution); 0: only the q adjoint systems */
  int smoother;      /* tobk_smoother: damped Jacobi (weight omega) or Chebyshev (degree nu_pre /
                        nu_post in D^{-1} K over [lambda_max / cheb_ratio, lambda_max], lambda_max
                        measured per level and design by power iteration); nu_pre, nu_post <= 8 */
  double cheb_ratio; /* lambda_max / lambda_min of the Chebyshev interval (e.g. 10) */
  /* Algorithm 2 (Appendix A) on the way from Omega_l to Omega_1, after each prolongation
   * Psi^j = I^j_{j+1} Psi^{j+1} (levels l-1 down to 1; multilevel path only): */
  int kaczmarz_sweeps; /* Kaczmarz sweeps on (K^j + sigma G^j) psi = 0 for every mode, sigma the smallest
                          load factor known from the level above; rows in 3^d node-colour order (colour
                          (i mod 3) + 3 (j mod 3) + 9 (k mod 3) ascending, the d rows of a node in turn);
                          0 = none (Sec. 2.1 steps 1-4) */
  int ritz_levels;   /* 1: Rayleigh-Ritz projection of (K^j, G^j) on span Psi^j after the smoothing */
  int fine_steps;    /* inverse-iteration steps K phi_{k+1} = G phi_k on Omega_1 (eq.
                        PInvIt-GeneralInteration with the preconditioner P = K, each solve by mgPCG to
                        rtol), each followed by the Rayleigh quotients; 1 (or 0) = the single fine solve
                        of Sec. 2.1 step 3 */
  int element;       /* tobk_element: the element of the fine grid */
  int eig_gram_tc;   /* 1: the eigensolver's Gram products V^T W run on the tensor cores with FP64
                        accuracy (error-free splitting, see tobk_gram_tc); 0 (default): FP64 CUDA-core
                        products, faster for the eigen levels of the configured workloads */
  int consistent_sens; /* 1: on the multilevel path, tobk_compute_sensitivities returns the exact
                          derivative of the multilevel load factors (eq. consistentSensitivity, with the
                          fine and coarse adjoints; see there); 0 (default): eq. SensitivityLambda applied
                          to the multilevel pairs, as the paper does.  Requires Sec. 2.1 steps 1-4 as they
                          stand (no Kaczmarz sweeps, Ritz projections or extra fine steps) and plain
                          elements; ignored for eig_level = 1, whose pairs are exact */
  int early_fine;    /* 1 (default): on the multilevel path of Sec. 2.1 (no Kaczmarz sweeps, Ritz projections
                        or extra fine steps) and on a stream of the caller's, the fine systems K phi =
                        G P psi of the coarse pairs that meet eig_tol while the eigensolver still iterates
                        on others are solved beside it, in groups on streams of the handle's own, to the
                        same rtol (the handle then holds 2q - 1 RHS columns of work space); 0: all q after
                        the eigensolve.  The load factors agree to the solver tolerances, not bit for bit */
} tobk_desc;

/* Elements (Sec. 2).  TOBK_ELEMENT_INCOMPATIBLE: Wilson's quadrilateral (2D) and the hexahedron with
 * 11 interpolation functions per component (3D): the bilinear / trilinear nodal functions plus d
 * internal modes 1 - xi_k^2 per component, condensed out element by element (the stress stiffness
 * uses the same condensation, its Gauss-point stresses from the enhanced strain).  Batches and the
 * learned warm start take TOBK_ELEMENT_PLAIN only. */
typedef enum { TOBK_ELEMENT_PLAIN = 0, TOBK_ELEMENT_INCOMPATIBLE = 1 } tobk_element;

typedef enum { TOBK_SMOOTHER_JACOBI = 0, TOBK_SMOOTHER_CHEBYSHEV = 1 } tobk_smoother;

typedef struct {
  int iterations;        /* CG iterations (max over RHS) or eigensolver outer iterations */
  int converged;         /* 1 if every RHS / eigenpair met its tolerance */
  int num_rhs;           /* right-hand sides solved in the call */
  double rel_residual;   /* max over RHS of the true relative residual recomputed at exit, or the
                            max eigen-residual */
  double time_ms;        /* device time of the call */
  int status_detail;     /* implementation detail code (0 = none) */
} tobk_solve_info;

typedef struct tobk_handle tobk_handle;

/* Fills *desc with defaults: nu 0.3, E0 1, Emin 1e-6, p 3, 3 levels, eig_level 1, 6 modes, FP64,
 * rtol 1e-8, max_iter 500, omega 0.6, nu_pre = nu_post = 2, eig_tol 1e-8, eig_max_iter 200,
 * max_rhs = num_modes + 4, no Kaczmarz sweeps, no per-level Ritz projection, one fine solve, plain
 * Q4 / H8 elements, FP64 CUDA-core Gram products in the eigensolver, no consistent sensitivities, the early
 * fine solve on.
 * Returns TOBK_OK. */
int tobk_default_desc(tobk_desc* desc);

/* Creates a handle on the current CUDA device and the given stream (cudaStream_t; NULL = legacy
 * default stream).  Allocates all device memory the problem needs.  Errors: TOBK_E_ARG for
 * inconsistent sizes, TOBK_E_NOMEM, TOBK_E_CUDA. */
int tobk_create(const tobk_desc* desc, void* cuda_stream, tobk_handle** out);
void tobk_destroy(tobk_handle* h);
/* Message of the last failed call on h (or of the last failed tobk_create when h is NULL). */
const char* tobk_last_error(const tobk_handle* h);

/* Physical densities x [m], each finite and in [0, 1] (Sec. 2 design field after filtering and
 * projection).  Builds the multigrid hierarchy: SIMP moduli, Galerkin coarse operators
 * K^{j+1} = I^T K^j I (Sec. 2.1 step 1), Jacobi diagonals and the coarsest dense inverse. */
int tobk_set_densities(tobk_handle* h, const double* x, int64_t m, int on_device);
/* Reference load vector f [n] (Algorithm 1, step 1).  Entries at fixed DOFs are ignored. */
int tobk_set_load(tobk_handle* h, const double* f, int64_t n, int on_device);
/* Dirichlet mask [n] (uint8, 1 = fixed).  Coarse levels fix a DOF when the fine DOF at the
 * coinciding node is fixed. */
int tobk_set_fixed(tobk_handle* h, const uint8_t* fixed, int64_t n, int on_device);
/* Optional initial guess u0 for the next solve_equilibrium (length n; NULL clears it).  The solve
 * starts from alpha u0 with alpha = u0^T f / u0^T K u0, the multiple of u0 closest to the solution in
 * the energy norm (so never farther from it than the zero guess). */
int tobk_set_initial_guess(tobk_handle* h, const double* u0, int64_t n, int on_device);

/* LA (Algorithm 1 step 2): u = K^{-1} f by mgPCG to desc.rtol; *compliance = f^T u (may be NULL).
 * Also builds the element stress stiffness G_e = E_sigma G_e0[u_e] (Algorithm 1 step 3). */
int tobk_solve_equilibrium(tobk_handle* h, double* compliance, tobk_solve_info* info);

/* EA: the q lowest positive buckling load factors of (K + lambda G) phi = 0 (eq.
 * eigenvalueProblem0), ascending, written to lambda [q] (host).  eig_level = 1: exact fine-grid
 * eigenpairs.  eig_level = l > 1: Sec. 2.1 steps 1-4 (coarse eigenpairs of the Galerkin pencil
 * (K^l, G^l), prolongation to Omega_1, fine solve K Phi = G Psi, per-column Rayleigh quotients,
 * re-sorted ascending).  Modes are scaled to phi^T K phi = 1 and signed so that their entry of
 * largest magnitude is positive. */
int tobk_compute_buckling(tobk_handle* h, double* lambda, tobk_solve_info* info);

/* Sensitivities (Sec. 2): dlambda_dx [q][m] and dJ_dx [m] (either may be NULL), with
 *   d lambda_i / d x_e = -[phi^T K' phi + lambda phi^T G' phi - lambda z^T K' u] / (phi^T G phi),
 *   K z_i = phi_i^T (grad_u G) phi_i   (eq. AdjointSystem; all q systems in one multi-RHS solve),
 *   dJ/dx_e = -dE_kappa/dx_e u_e^T K_e0 u_e.
 * (eq. SensitivityLambda is the bracket; the factor -1/(phi^T G phi) equals lambda under the K
 * normalisation.)  out_on_device selects device or host output pointers.
 *
 * With desc.consistent_sens on the multilevel path, dlambda_dx is instead the exact derivative of the
 * multilevel load factors lambda_i = R(phi_i), phi_i = K^{-1} G P psi_i (Sec. 2.1; eq. eigResidual and
 * eq. consistentSensitivity): with y_i = (K + lambda_i G) phi_i, mu_i the coarse load factor of psi_i and
 * Psi_i = P psi_i,
 *   K w_i = y_i                                        (fine adjoint, mgPCG)
 *   (K^l + mu_i G^l) c_i = P^T G w_i, psi_i^T G^l c_i = 0   (coarse adjoint, deflated PCG on Omega_l)
 *   K z_i = g_i = grad_u [lambda_i phi_i^T G phi_i + (2 w_i - 2 mu_i P c_i)^T G Psi_i]
 *   d lambda_i / d x_e = -{ dE_kappa [(phi - 2w)^T K_e0 phi - 2 (Pc)^T K_e0 Psi - z^T K_e0 u]
 *                          + dE_sigma [lambda phi^T G_e0 phi + (2w - 2 mu Pc)^T G_e0 Psi] } / (phi^T G phi).
 * info reports the largest iteration count of the three solves and, in status_detail, the coarse
 * adjoint's CG iterations; TOBK_E_NOT_CONVERGED if one of them stopped at max_iter. */
int tobk_compute_sensitivities(tobk_handle* h, double* dlambda_dx, double* dJ_dx, int out_on_device,
                               tobk_solve_info* info);

/* Copies a field (tobk_field) to out (len doubles). */
int tobk_get_field(tobk_handle* h, int which, double* out, int64_t len, int out_on_device);

/* Number of CUDA kernels the library has launched in this process (all handles). */
long long tobk_launch_count(void);

/* Kernel classes timed by the profiler (CUDA events around each launch of the class, on the
 * handle's stream, while profiling is enabled). */
typedef enum {
  TOBK_KC_FINE_SMOOTH = 0,     /* damped-Jacobi sweep on the fine grid (matrix-free K v fused) */
  TOBK_KC_FINE_RESIDUAL = 1,   /* residual b - K z on the fine grid */
  TOBK_KC_FINE_CG_MATVEC = 2,  /* CG direction update fused with q = K p on the fine grid */
  TOBK_KC_COARSE = 3,          /* smoother / residual / CG matvec on Galerkin levels */
  TOBK_KC_TRANSFER = 4,        /* restriction and prolongation */
  TOBK_KC_COARSEST = 5,        /* dense coarsest-level solve */
  TOBK_KC_VECTOR = 6,          /* CG dot products and vector updates, first Jacobi sweep */
  TOBK_KC_EIGEN_DENSE = 7,     /* eigensolver: dense Rayleigh-Ritz and block Cholesky kernels */
  TOBK_KC_EIGEN_BLOCK = 8,     /* eigensolver: block orthogonalisation and Ritz-vector kernels */
  TOBK_KC_COUNT = 9
} tobk_kernel_class;

/* Enables (1) or disables (0) kernel-class timing on h; enabling resets the counters. */
int tobk_profile_enable(tobk_handle* h, int enable);
/* Launch count, total device milliseconds and total work (DOF x RHS processed) of a kernel class
 * since profiling was enabled (any output pointer may be NULL). */
int tobk_profile_read(tobk_handle* h, int kernel_class, long long* launches, double* total_ms,
                      double* dof_rhs);

/* Phases of the last tobk_compute_buckling, in device milliseconds (CUDA events on the handle's
 * stream, recorded while phase timing is on): the eigensolve (eq. eigenvalueProblemCoarseScale on
 * Omega_l, or eq. eigenvalueProblem0 on the fine grid), and within it the multigrid preconditioner
 * applications and the dense Rayleigh-Ritz steps; the prolongation Psi^j = I^j_{j+1} Psi^{j+1} with
 * the right-hand sides G Psi (Sec. 2.1 step 2); the fine block solve K Phi = G Psi (eq. FineScaleBVP);
 * the Rayleigh quotients and the normalisation of the modes (eq. FineScaleRQ); and the eigensolver's
 * outer iterations (a count, not a time). */
typedef enum {
  TOBK_PHASE_EIGEN = 0,
  TOBK_PHASE_EIGEN_PRECOND = 1,
  TOBK_PHASE_EIGEN_RR = 2,
  TOBK_PHASE_PROLONG = 3,
  TOBK_PHASE_FINE_SOLVE = 4,
  TOBK_PHASE_RQ = 5,
  TOBK_PHASE_EIGEN_ITERS = 6,
  TOBK_PHASE_COUNT = 7
} tobk_phase;
/* Turns phase timing on (1) or off (0); it adds a few CUDA events per eigensolver iteration. */
int tobk_phase_enable(tobk_handle* h, int enable);
/* Copies min(len, TOBK_PHASE_COUNT) phase values of the last compute_buckling to out (host). */
int tobk_phase_read(tobk_handle* h, double* out, int len);

/* ---- unit-level entry points (device pointers) ------------------------------------------------ */
/* Element and DOF counts of a 1-based level: out[0..2] = nel, out[3] = n (DOFs), out[4] = m. */
int tobk_level_info(tobk_handle* h, int level, int64_t* out5);
/* y = K^level v for nrhs vectors of length n_level (level 1: matrix-free SIMP operator, Sec. 2;
 * level > 1: Galerkin operator).  Requires densities. */
int tobk_apply_K(tobk_handle* h, int level, const double* v, double* y, int nrhs);
/* y = G^level v (requires solve_equilibrium; levels 1..eig_level). */
int tobk_apply_G(tobk_handle* h, int level, const double* v, double* y, int nrhs);
/* Multi-RHS mgPCG solve K^level X = B at the given level (nrhs <= desc.max_rhs), X overwritten. */
int tobk_solve(tobk_handle* h, int level, const double* B, double* X, int nrhs, tobk_solve_info* info);
/* Copies the stored Galerkin element matrices of a coarse level (which: 0 = K, 1 = G) to out
 * [m_level][nd*nd] (device pointer), nd = dim * 2^dim. */
int tobk_get_element_matrices(tobk_handle* h, int level, int which, double* out, int64_t len);

/* C [na][nb] = A B^T for na, nb <= 64 FP64 vectors of length n (rows of A and B stride doubles
 * apart; device pointers): the Gram product of the eigensolver (eq. eigenvalueProblemCoarseScale,
 * solved to a residual of 1e-8, Appendix A) on the tensor cores.  Every vector is scaled by a power of
 * two and cut into eight 7-bit digit planes held exactly in bfloat16; the plane products are summed
 * exactly (FP32 tensor-core accumulators over chunks of 64 entries, then int64) and combined in FP64,
 * so the result is within about n 2^-53 max|A_i| max|B_j| of the exact product (error-free
 * splitting, Ozaki et al. 2012).  For unit tests; synchronised on cuda_stream before return.
 * TOBK_E_ARG for bad sizes, TOBK_E_NONFINITE for a NaN / infinity in the input, TOBK_E_TIMEOUT if a
 * bounded device wait gave up. */
int tobk_gram_tc(const double* A, int na, const double* B, int nb, int64_t n, int64_t stride, double* C,
                 void* cuda_stream);

/* ---- many designs solved together ------------------------------------------------------------
 * A batch holds nd independent 2D designs (each its own grid, densities, Dirichlet set and multigrid
 * hierarchy) that share one CUDA stream and are solved together: K_d X_d = B_d with nrhs right-hand
 * sides per design (e.g. the load and the q adjoint systems of eq. AdjointSystem), by flexible CG in
 * FP64 preconditioned with an FP32 V-cycle (the TOBK_FP32_VCYCLE form of the mgPCG of Appendix A).
 * Every phase of the iteration is one launch over all designs (grouped work lists, persistent-style
 * grid stride), two CG iterations are replayed from a captured CUDA graph, and the smoother tile
 * shapes are chosen by tobk_batch_autotune.
 *
 * Packed layouts: design d owns elements [elem_off[d], elem_off[d+1]) of the packed densities and
 * DOFs [dof_off[d], dof_off[d+1]) of the packed Dirichlet mask; the packed right-hand sides and
 * solutions put design d's block [nrhs][n_d] at offset nrhs * dof_off[d].
 * Limits: dim = 2; 2 <= mg_levels <= 8; all designs share nu, nu_pre, nu_post and the smoother;
 * rtol and max_iter of descs[0] apply to every design; 1 <= nrhs <= 64.  Errors as for the
 * single-design calls; tobk_batch_last_error() gives the message. */
typedef struct tobk_batch tobk_batch;
int tobk_batch_create(const tobk_desc* descs, int ndesigns, int nrhs, void* cuda_stream, tobk_batch** out);
void tobk_batch_destroy(tobk_batch* b);
const char* tobk_batch_last_error(const tobk_batch* b);
/* dof_offsets, elem_offsets: [ndesigns + 1] (either may be NULL). */
int tobk_batch_layout(const tobk_batch* b, int64_t* dof_offsets, int64_t* elem_offsets);
/* Packed densities x and Dirichlet masks (host or device); builds every design's hierarchy. */
int tobk_batch_set_designs(tobk_batch* b, const double* x, const uint8_t* fixed, int on_device);
/* Solves every design's K_d X_d = B_d to rtol (B, X packed, host or device).  infos: [ndesigns]
 * (may be NULL), per design: CG iterations (max over its RHS), converged, the worst true relative
 * residual at exit, the device time of the whole batch call. */
int tobk_batch_solve(tobk_batch* b, const double* B, double* X, int on_device, tobk_solve_info* infos);
/* Times the candidate variants of the grouped smoother kernels on the current designs and keeps
 * the fastest: fine FP32 smoother node tiles 0: 32x8, 1: 32x4, 2: 64x4, 3: 16x16; coarse stencil
 * kernel 0/1/2: 1/2/4 right-hand sides per thread.  Outputs the choices (either may be NULL). */
int tobk_batch_autotune(tobk_batch* b, int* fine_variant, int* coarse_variant);
/* Sets the variants explicitly (same numbering). */
int tobk_batch_set_variants(tobk_batch* b, int fine_variant, int coarse_variant);

/* ---- learned warm start (not part of the paper's method) -------------------------------------
 * A small 3D U-Net maps a design (densities x [m] and load f [n] of an H8 grid) to an initial guess
 * u0 [n] for tobk_set_initial_guess; mgPCG then runs to the same tolerance as without it, so the
 * network can change the iteration count but never the accepted accuracy.  Architecture: `levels`
 * encoder levels of two 3x3x3 convolutions + ReLU (2x2x2 average pooling between levels), a
 * decoder with nearest 2x upsampling and skip concatenation, a 1x1x1 output head on the finest
 * decoder level plus a coarse-correction head on the bottleneck (upsampled and added), node
 * averaging of the per-element output times a fixed output scale c (t), and a per-design scale
 * s = mean(E_kappa) / (largest element load sum): u0 = t / s.  Input features: 2x - 1 and the
 * element load sums normalised by their largest magnitude.  Loss of a sample with solution u,
 * t* = s u, K the sample's stiffness: the relative energy-norm error (t - t*)^T K (t - t*) /
 * t*^T K t* over the free DOFs (default; what CG convergence depends on), or the relative squared
 * error sum_free (t - t*)^2 / sum_free t*^2.
 * Parameters: one FP32 vector (Adam's master copy) in the order enc_l a, enc_l b (l = 0..L-1),
 * dec_l a, dec_l b (l = L-2..0), head, coarse head; each layer W [Cout][Cin][taps] then b [Cout];
 * the convolutions use a bfloat16 copy with FP32 accumulation.  Hand-written CUDA kernels for the
 * forward and backward passes and the Adam update; all pointers below are DEVICE pointers. */
typedef enum { TOBK_UNET_LOSS_MSE = 0, TOBK_UNET_LOSS_ENERGY = 1 } tobk_unet_loss_kind;
typedef struct {
  int nel[3];           /* H8 element grid (x, y, z); each divisible by 2^(levels-1) */
  int levels;           /* 1..4 */
  int channels[4];      /* per level, multiples of 16, at most 256 */
  int in_channels;      /* 4 */
  int out_channels;     /* 3 */
  double penal, E0, Emin;  /* SIMP parameters of the designs (scale s, energy loss) */
  double nu;            /* Poisson ratio (energy loss) */
  int loss;             /* tobk_unet_loss_kind: relative energy-norm error of the guess (default) or
                           relative squared error of the scaled displacements */
  unsigned long long seed; /* weight initialisation (He normal, zero biases) */
} tobk_unet_desc;
typedef struct tobk_unet tobk_unet;
/* defaults: 128 x 64 x 64, 4 levels, channels 16/32/64/64, p 3, E0 1, Emin 1e-6 */
int tobk_unet_default_desc(tobk_unet_desc* desc);
int tobk_unet_create(const tobk_unet_desc* desc, void* cuda_stream, tobk_unet** out);
void tobk_unet_destroy(tobk_unet* net);
const char* tobk_unet_last_error(const tobk_unet* net);
int64_t tobk_unet_num_params(const tobk_unet* net);
/* The output scale c of the guess t = c * (node average of the output) (default 1; chosen from the
 * training data so that the network's outputs are of order one). */
int tobk_unet_set_output_scale(tobk_unet* net, double scale);
double tobk_unet_output_scale(const tobk_unet* net);
/* The design scale s = mean(E_kappa) / (largest element load sum) of x [m] (FP32), f [n] -> *s (host). */
int tobk_unet_design_scale(tobk_unet* net, const float* x, const double* f, double* s);
/* Parameters, Adam moments and step count (checkpoint / resume); any array pointer may be NULL on
 * get; on set, NULL moments restart Adam from zero.  on_device selects device or host arrays. */
int tobk_unet_get_state(tobk_unet* net, float* params, float* adam_m, float* adam_v, long long* step, int on_device);
int tobk_unet_set_state(tobk_unet* net, const float* params, const float* adam_m, const float* adam_v, long long step,
                        int on_device);
/* u0 [n] (FP64, zero at fixed DOFs) from x [m] (FP64), f [n] (FP64), fixed [n].  3x3x3 convolutions
 * that run on the tensor cores (see tobk_unet_set_tensor_cores) are tcgen05 implicit GEMMs with the
 * activations rounded to bfloat16 (FP32 accumulation); TOBK_E_TIMEOUT if one of their bounded
 * device waits gave up (no output is valid then). */
int tobk_unet_predict(tobk_unet* net, const double* x, const double* f, const uint8_t* fixed, double* u0);
/* Selects the inference convolutions: mode 0 the FP32 direct convolution that training uses; 1 (the
 * default) the tensor cores on levels of at least 128 * 2 * 152 voxels (two 128-voxel tiles per
 * SM; smaller levels stay direct, which is faster there); 2 the tensor cores on every level.
 * Layers whose output channels are not 16, 32, 64 or 128 always use the direct convolution. */
int tobk_unet_set_tensor_cores(tobk_unet* net, int mode);
/* One 3x3x3 convolution on the tensor cores (the kernel of tobk_unet_predict), for unit tests:
 * out[co][z][y][x] = bias[co] + sum_ci sum_tap w[co][ci][tap] bf16(in[ci][(z,y,x) + tap]) with zero
 * padding, taps ordered (dz, dy, dx) in {-1,0,1}^3 with dx fastest, then max(0, .) if relu.
 * in [Cin][D][H][W], out [Cout][D][H][W] (FP32, device), weight [Cout][Cin][27] and bias [Cout]
 * (FP32, device; rounded to bfloat16; bias may be NULL).  Cout in {16, 32, 64, 128}; stream-ordered
 * on cuda_stream and synchronised before return.  TOBK_E_ARG for unsupported shapes, TOBK_E_TIMEOUT
 * if a bounded device wait gave up. */
int tobk_conv3_bf16(const float* in, int Cin, int D, int H, int W, const float* weight, const float* bias, int Cout,
                    int relu, float* out, void* cuda_stream);
/* Loss of one sample (x [m] FP32, target solution [n] FP32) and its gradient grad [num_params]
 * (may be NULL). */
int tobk_unet_loss_grad(tobk_unet* net, const float* x, const double* f, const float* target, const uint8_t* fixed,
                        float* loss, float* grad);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, learning rate lr) on the mean gradient of nbatch samples
 * x [nbatch][m], target [nbatch][n] (FP32) sharing f and fixed; *loss = mean sample loss. */
int tobk_unet_train_step(tobk_unet* net, const float* x, const double* f, const float* target, const uint8_t* fixed,
                         int nbatch, float lr, float* loss);

/* ---- allocation-free residual check ------------------------------------------------------------
 * Not part of the paper's method (it has no counterpart there): a utility for callers that must not
 * allocate device memory when they verify a solution, e.g. code running while a stream is being
 * captured into a CUDA graph (cudaMalloc is not allowed there), programs whose device memory is
 * owned by another framework's pool allocator, or latency-critical loops that cannot afford
 * cudaMalloc's implicit synchronisation.  It needs no handle and allocates nothing.
 *
 * For r = 0..nrhs-1 writes relres[r] = ||B_r - K(x) X_r||_2 / ||B_r||_2 over the free DOFs of the
 * fine grid described by desc (dim, nel, nu, E0, Emin, penal, element; other fields ignored), K(x)
 * being the SIMP stiffness of tobk_apply_K at level 1.  Entries of X at fixed DOFs are read as zero (the
 * residual of the free-DOF system), and when B_r is zero on the free DOFs relres[r] is the absolute
 * residual norm ||K(x) X_r||_2.  x [m], fixed [n] (uint8, 1 = fixed), B and X
 * [nrhs][n] and relres [nrhs] are DEVICE pointers on the current device; the caller owns them.
 * The work is enqueued on cuda_stream (NULL = legacy default stream); relres is valid once that
 * stream has reached this point.
 * Limits: nrhs <= 16 (otherwise TOBK_E_ARG): the reduction scratch is a fixed array of 256 KiB in
 * the library's own device memory, which every GPU that loads the library keeps until the process
 * exits.  Every call on a device shares that array: calls whose kernels may overlap on the GPU
 * (different streams without ordering) race and must not be issued.  The first call on each
 * device does the set-up: it looks up the array's device address (cudaGetSymbolAddress, with that
 * device current), so that first call should come before any stream capture begins.  Later calls
 * look the address up again unless their stream is in capture mode, so that it stays valid after a
 * device reset.
 * Errors: TOBK_E_ARG (null pointer, bad dim or sizes, nrhs out of range, the material checks of
 * tobk_create: -1 < nu < 0.5, E0 > 0, Emin > 0, penal >= 1), TOBK_E_CUDA; tobk_last_error(NULL), on the
 * calling thread, then names the check that failed. */
int tobk_residual_noalloc(const tobk_desc* desc, const double* x, const uint8_t* fixed, const double* B,
                          const double* X, int nrhs, double* relres, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TOBK_H_ */
