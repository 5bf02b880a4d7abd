// Host-side launch wrappers for the CUDA kernels of the library (all kernels live in kernels.cu).
// Every wrapper enqueues work on the given stream and returns immediately; pointers are device
// pointers; multi-RHS blocks are RHS-major with the given stride (elements between RHS columns).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tobk_internal.cuh"

namespace tobk {

// Per-RHS scalar state ([nr][kScStride]) of the CG driver running on this host thread, or null.
// While set, the V-cycle kernels skip right-hand sides that have converged.
const double* active_rhs();
void set_active_rhs(const double* sc);

// Which element operator a level uses.
struct LevelOpDesc {
  Grid g;
  const uint8_t* fixed;
  // fine (level 1): matrix-free scale_e * T0 with T0 = Ke0 (double) / Ke0f (float)
  const double* scale64;
  const float* scale32;
  const double* T0;     // host pointer to the nd*nd table (copied into kernel parameters)
  const double* T0dev;  // device copy of the same table
  // coarse: stored element matrices
  const double* Ke64;
  const float* Ke32;
  bool stored;
  // coarse: the same operator assembled per node as a 3^d-point stencil of d x d blocks
  // ([node][neighbour][d][d]); when set, smoother and residual launches use it
  const double* S64 = nullptr;
  const float* S32 = nullptr;
  double nu = 0.3;  // Poisson ratio (the factored fine H8 operator builds its constants from it)
  int element = 0;  // tobk_element of the fine level (the factored H8 operator's correction)
};

// Assembles the per-node stencil of a stored-element-matrix level (rows/columns of fixed DOFs
// zeroed); also writes the float copy when S32 != nullptr.
void launch_stencil_assemble(const Grid& g, const double* Ke, const uint8_t* fixed, double* S, float* S32,
                             cudaStream_t s);

enum ApplyMode { APPLY_KV = 0, APPLY_RES = 1, APPLY_JAC = 2 };

// One smoothing step (APPLY_JAC): r = dinv (b - K v); dn = coef[0] d_in + coef[1] r; y = v + dn;
// d_out = dn.  d_in == nullptr means a zero previous increment; coef is a device pointer (so that
// captured graphs stay valid when the coefficients change).  Damped Jacobi: coef = (0, omega);
// Chebyshev: the per-step recurrence coefficients.
template <typename T>
struct SmoothArgs {
  const T* coef = nullptr;
  const T* d_in = nullptr;
  T* d_out = nullptr;
};

// y = K v | y = b - K v | y = v + omega dinv (b - K v), for nr RHS (double or float vectors).
void launch_apply(const LevelOpDesc& op, int mode, const double* v, const double* b, const double* dinv,
                  double* y, SmoothArgs<double> sm, int nr, int64_t stride, cudaStream_t s);
void launch_apply32(const LevelOpDesc& op, int mode, const float* v, const float* b, const float* dinv,
                    float* y, SmoothArgs<float> sm, int nr, int64_t stride, cudaStream_t s);

// CG direction p = z + beta p_old, q = K p, p.q and alpha on a stencil level (stencil.cu); the
// contract of launch_cg_direction.
void launch_stencil_cg_direction(const Grid& g, const double* S, const uint8_t* fixed, const double* z,
                                 const double* p_old, double* p_new, double* q, int nr, int64_t stride, double* sc,
                                 double* partial, unsigned* counters, int64_t pstride, cudaStream_t s);
// 2D stencil levels, transfers fused into the sweeps (stencil.cu):
// y = v + d with v = z + P zc (the prolongated coarse correction added on the fly, not at fixed
// DOFs) and d = coef[0] d_in + coef[1] dinv (b - K v) -- the prolongation and the first
// post-smoothing step of a V-cycle level in one launch (zc [nr][cstride] on the coarse grid gc).
template <typename T>
void launch_stencil_jac_prolong_2d(const Grid& g, const Grid& gc, const T* S, const uint8_t* fixed, const T* z,
                                   const T* zc, const T* b, const T* dinv, T* y, SmoothArgs<T> sm, int nr,
                                   int64_t stride, int64_t cstride, cudaStream_t s);
// bc = P^T (b - K z) on the coarse grid gc (0 at its fixed DOFs), and when zc != nullptr the coarse
// level's first damped step zc = coef_c[1] dinv_c bc (also into dc when dc != nullptr) -- the
// residual, the restriction and the coarse pre-smoothing start in one launch.
template <typename T>
void launch_stencil_res_restrict_2d(const Grid& g, const Grid& gc, const T* S, const uint8_t* fixed, const T* z,
                                    const T* b, int64_t stride, const uint8_t* fixed_c, T* bc, int64_t cstride,
                                    const T* dinv_c, const T* coef_c, T* zc, T* dc, int nr, cudaStream_t s);
// y = G v with G_e = Gs_e (x) I (Gs includes E_sigma), fine level.
void launch_apply_kron(const Grid& g, const uint8_t* fixed, const double* Gs, const double* v, double* y,
                       int nr, int64_t stride, cudaStream_t s);
// dinv = 1/diag(K) (0 at fixed DOFs); also a float copy when dinv32 != nullptr.
void launch_diag(const LevelOpDesc& op, double* dinv, float* dinv32, cudaStream_t s);
// z = omega dinv b (first damped-Jacobi sweep from a zero guess)
void launch_jacobi0(const double* b, const double* dinv, double* z, SmoothArgs<double> sm, int64_t n, int nr,
                    int64_t stride, cudaStream_t s);
void launch_jacobi0_32(const float* b, const float* dinv, float* z, SmoothArgs<float> sm, int64_t n, int nr,
                       int64_t stride, cudaStream_t s);
// coarse b = P^T r_fine (masked); fine z += P z_coarse (masked).  With zc != null the restriction
// also takes the coarse level's first smoothing step from z = 0: zc = coef_c[1] dinv_c b (and dc = zc
// when dc != null), the work of launch_jacobi0 on the coarse level.
void launch_restrict(const Grid& gf, const Grid& gc, const uint8_t* fixed_c, const double* rf, double* bc,
                     int nr, int64_t sf, int64_t sc, cudaStream_t s, const double* dinv_c = nullptr,
                     const double* coef_c = nullptr, double* zc = nullptr, double* dc = nullptr);
void launch_restrict32(const Grid& gf, const Grid& gc, const uint8_t* fixed_c, const float* rf, float* bc,
                       int nr, int64_t sf, int64_t sc, cudaStream_t s, const float* dinv_c = nullptr,
                       const float* coef_c = nullptr, float* zc = nullptr, float* dc = nullptr);
void launch_prolong_add(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* zc, double* zf,
                        int nr, int64_t sf, int64_t sc, cudaStream_t s);
void launch_prolong_add32(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const float* zc, float* zf,
                          int nr, int64_t sf, int64_t sc, cudaStream_t s);
// z = Ainv b (dense, n x n, FP64 matrix), nr RHS
void launch_dense_gemv(const double* Ainv, const double* b, double* z, int64_t n, int nr, int64_t stride,
                       cudaStream_t s);
void launch_dense_gemv32(const double* Ainv, const float* b, float* z, int64_t n, int nr, int64_t stride,
                         cudaStream_t s);
// Dense assembly of a level operator (identity rows/cols at fixed DOFs), then in-place-free
// Gauss-Jordan inversion (SPD, no pivoting) ping-ponging between A and work.
void launch_dense_assemble(const LevelOpDesc& op, double* A, cudaStream_t s);
// returns the buffer holding the inverse (A or work)
double* launch_dense_invert(double* A, double* work, int64_t n, double* rcp2, cudaStream_t s);

// Galerkin coarse element matrices.  child source: fine K (scale * table), fine G (Es * Gs0 (x) I),
// or stored matrices of the previous level.  Rows/cols of fixed fine DOFs are masked.
void launch_galerkin_fine_K(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* scale,
                            const double* Ke0, const double* W, double* Kc, cudaStream_t s);
void launch_galerkin_fine_G(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* Gs,
                            const double* W, double* Gc, cudaStream_t s);
void launch_galerkin_stored(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* Kf,
                            const double* W, double* Kc, cudaStream_t s);

// Element stress stiffness: Gs0[e] = sum_gp w|J| dN^T S(D B u_e) dN (unit modulus), Gs = E_sigma Gs0.
// dN [ngp][dim][nn] and D [nv][nv] are device tables.
void launch_stress_gs_dev(const Grid& g, const double* u, const double* Es, const double* dN, const double* D,
                          double wdet, double* Gs0, double* Gs, cudaStream_t s);
int64_t cg_partial_stride(const Grid& g);
// Thread blocks of the factored fine Q4 kernels for one RHS (tiles of 32 x 8 nodes).
int64_t fine_q4_tiles(const Grid& g);
// Largest number of thread blocks per RHS of the factored fine H8 kernels.
int64_t fine_h8_blocks(const Grid& g);
// Factored fine H8 operator: y = K v | b - K v | smoothing step (same contract as launch_apply).
template <typename T>
void launch_fine_h8(const Grid& g, const T* Ek, const uint8_t* fixed, double nu, int element, int mode, const T* v, const T* b,
                    const T* dinv, T* y, SmoothArgs<T> sm, int nr, int64_t stride, cudaStream_t s);
// CG direction on the fine H8 level in factored form (same contract as launch_cg_direction).
void launch_fine_h8_cg_direction(const Grid& g, const double* Ek, const uint8_t* fixed, double nu, int element, const double* z,
                                 const double* p_old, double* p_new, double* q, int nr, int64_t stride, double* sc,
                                 double* partial, unsigned* counters, int64_t pstride, cudaStream_t s);
// CG direction on the fine Q4 level in factored form: p_new = z + beta p_old, q = K p_new,
// sc[SC_PQ] = p_new . q, sc[SC_ALPHA] (same contract as launch_cg_direction).
void launch_fine_q4_cg_direction(const Grid& g, const double* Ek, const uint8_t* fixed, const double* Ke0,
                                 const double* z, const double* p_old, double* p_new, double* q, int nr,
                                 int64_t stride, double* sc, double* partial, unsigned* counters, int64_t pstride,
                                 cudaStream_t s);

// SIMP moduli (paper Sec. 2): Ek = Emin + x^p (E0 - Emin), Es = x^p E0, derivatives.
void launch_simp(const double* x, int64_t m, double penal, double E0, double Emin, double* Ek, double* Es,
                 double* dEk, double* dEs, float* Ek32, cudaStream_t s);

// elementwise helpers
void launch_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
void launch_f32_to_f64(const float* a, double* b, int64_t n, cudaStream_t s);
void launch_mask_copy(const double* src, const uint8_t* fixed, double* dst, int64_t n, int nr, int64_t stride,
                      cudaStream_t s);

// ---- multi-RHS PCG kernels (FP64).  sc: [nr][kScStride] scalars; partial/counters: scratch.
// The first smoothing step of the next V-cycle from a zero guess, z = coef[1] dinv r (also into d),
// taken by the kernel that writes the residual r (cg_init, cg_update) instead of a launch of its own;
// z == nullptr: off.
struct CGZ0 {
  const double* dinv = nullptr;
  const double* coef = nullptr;
  double* z = nullptr;
  double* d = nullptr;
};
void launch_cg_init(const LevelOpDesc& op, const double* b, double* x, double* r, bool use_x0, double rtol,
                    int nr, int64_t stride, double* sc, double* partial, unsigned* counters, cudaStream_t s,
                    CGZ0 z0 = CGZ0{});
void launch_cg_dots(int64_t n, const double* z, const double* r, const double* q, const double* p, bool flexible,
                    int nr, int64_t stride, double* sc, double* partial, unsigned* counters, cudaStream_t s);
void launch_cg_direction(const LevelOpDesc& op, const double* z, const double* p_old, double* p_new, double* q,
                         int nr, int64_t stride, double* sc, double* partial, unsigned* counters, cudaStream_t s);
void launch_cg_update(int64_t n, double* x, double* r, const double* p, const double* q, int nr, int64_t stride,
                      double* sc, double* partial, unsigned* counters, cudaStream_t s, CGZ0 z0 = CGZ0{});
// true residual: r = b - K x; sc[SC_RELRES] = ||r|| / ||b||
void launch_true_residual(const LevelOpDesc& op, const double* b, const double* x, double* r, int nr,
                          int64_t stride, double* sc, double* partial, unsigned* counters, cudaStream_t s);

// ---- dense small-block kernels for block methods: C[i][j] = sum_k A[i][k] B[j][k] over rows
//      of A [na][n] and B [nb][n] (RHS-major vectors).  Deterministic two-stage reduction.
void launch_gram(const double* A, int na, const double* B, int nb, int64_t n, int64_t stride, double* C,
                 double* partial, cudaStream_t s);
// Y[j][:] (+)= sum_i X[i][:] * C[i][j]  (X [nx][n], C [nx][ny] row-major, Y [ny][n]); beta: 0 or 1
// for overwrite / accumulate; alpha scales the product.
void launch_combine(const double* X, int nx, const double* C, int ldc, int ny, double alpha, double beta,
                    double* Y, int64_t n, int64_t stride, cudaStream_t s);
// Y_s = X_s C (s = 0, 1, 2; X_s [nx][stride], Y_s [ny][stride]) in one launch
void launch_combine3(const double* X0, const double* X1, const double* X2, int nx, const double* C, int ldc, int ny,
                     double* Y0, double* Y1, double* Y2, int64_t n, int64_t stride, cudaStream_t s);
int gram_partial_blocks(int64_t n);
// C[o] = sum over chunks of partial[c][o] in a fixed order (the second stage of launch_gram)
void launch_gram_final(const double* partial, int nchunks, int nout, double* C, cudaStream_t s);
// The same Gram product on the tensor cores with FP64 accuracy (gram_tc.cu); partial
// [gram_tc_chunks(n)][na][nb] is FP64 scratch (at most the launch_gram partials), err [2] is set on a
// timed-out wait / a non-finite input.  na, nb <= 64.
void launch_gram_tc(const double* A, int na, const double* B, int nb, int64_t n, int64_t stride, double* C,
                    double* partial, unsigned* err, cudaStream_t s);
int gram_tc_chunks(int64_t n);

// ---- incompatible-mode elements (incompatible.cu) ---------------------------------------------------
// Gfull [m][nf*nf] and the condensed unit-modulus stress stiffness Gc0 [m][nd*nd] from u.
void launch_inc_stress(const Grid& g, const double* u, const double* A, const double* dN, const double* D,
                       double wdet, double* Gfull, double* Gc0, cudaStream_t s);
// y = sum_e Es[e] Gc0[e] v_e for nr vectors (rows of fixed DOFs zero)
void launch_inc_apply_g(const Grid& g, const uint8_t* fixed, const double* Gc0, const double* Es, const double* v,
                        double* y, int nr, int64_t stride, cudaStream_t s);
// adjoint right-hand side b = phi^T (grad_u G) phi via element vectors ev [m][nd] (masked)
void launch_inc_adjoint(const Grid& g, const uint8_t* fixed, const double* phi, const double* Es, const double* A,
                        const double* dN, const double* D, double wdet, double* ev, double* b, cudaStream_t s);
// Galerkin coarse element matrices from stored fine element matrices times a per-element scale
void launch_galerkin_scaled_stored(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* Kf,
                                   const double* scale, const double* W, double* Kc, cudaStream_t s);

// ---- Kaczmarz smoothing of prolongated modes (kaczmarz.cu) -----------------------------------------
// Nodal stencil S of A = K + sigma G at a level and its squared row norms rn2 [n].  K from E_kappa
// [m] and the unit matrix Ke0 (fine level, Ek != nullptr) or stored element matrices Ke; G from the
// fine scalar matrices Gs [m][nn*nn] (Gs != nullptr) or stored element matrices Ge, times Gscale[e]
// when Gscale != nullptr.
void launch_pencil_stencil(const Grid& g, const uint8_t* fixed, const double* Ek, const double* Ke0,
                           const double* Ke, const double* Gs, const double* Ge, const double* Gscale, double sigma,
                           double* S, double* rn2, cudaStream_t s);
// `sweeps` multicolour Kaczmarz sweeps on A psi = 0 for q modes Psi [q][stride].
void launch_kaczmarz_sweeps(const Grid& g, const uint8_t* fixed, const double* S, const double* rn2, double* Psi,
                            int q, int64_t stride, int sweeps, cudaStream_t s);

}  // namespace tobk
