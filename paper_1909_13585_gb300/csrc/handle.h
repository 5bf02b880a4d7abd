// The solver handle behind the opaque tobk_handle* of the C-ABI, and the host-side entry points that
// the C-ABI functions call.  One handle = one structured-grid problem on one CUDA stream.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/tobk.h"
#include "kernels.h"
#include "tobk_internal.cuh"

struct tobk_handle {
  tobk_desc desc{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int dim = 2;
  int L = 1;                 // multigrid levels
  int eig = 0;               // 0-based level of the coarse eigenproblem
  int q = 1;                 // modes
  int rmax = 1;              // RHS capacity of the multi-RHS solver
  tobk::ElementTables tab;
  tobk::Arena arena;
  tobk::Level lv[tobk::kMaxLevels];

  // device tables
  double* d_Ke0 = nullptr;   // [nd*nd]
  double* d_W = nullptr;     // [2^d][nn][nn]
  double* d_dN = nullptr;    // [ngp][d][nn]
  double* d_D = nullptr;     // [nv][nv]
  // fine-level design fields
  double *x = nullptr, *Ek = nullptr, *Es = nullptr, *dEk = nullptr, *dEs = nullptr;
  float* Ek32 = nullptr;
  double *f = nullptr, *u = nullptr, *u0 = nullptr;
  double *Gs0 = nullptr, *Gs = nullptr;  // [m][nn*nn] stress stiffness (unit modulus / with E_sigma)
  // incompatible-mode elements: condensation map [d*d][nd], per-element G over the 2^d + d functions
  // [m][nf*nf] and the condensed unit-modulus stress stiffness [m][nd*nd] (times E_sigma in use)
  double *d_A = nullptr, *Gfull = nullptr, *Gc0 = nullptr;
  // coarsest dense inverse
  double *Adense = nullptr, *Awork = nullptr, *Ainv = nullptr;
  // multi-RHS CG work (sized for the fine level)
  tobk::CGWork cg{};
  double* bwork = nullptr;   // [rmax][n] right-hand-side staging
  double* xwork = nullptr;   // [rmax][n]
  // buckling / sensitivity outputs
  double* modes = nullptr;   // [q][n] fine-grid modes (K-normalised)
  double* lam = nullptr;     // [q] device
  double* adj_blockB = nullptr;  // [q+1][n]: f, then the adjoint right-hand sides
  double* adj_blockX = nullptr;  // [q+1][n]: u of the fused solve, then the adjoint solutions
  double* adj = nullptr;     // [q][n] adjoint solutions
  double* adj_rhs = nullptr; // [q][n]
  double* dlam = nullptr;    // [q][m]
  double* dJ = nullptr;      // [m]
  double* esens = nullptr;   // [m][...] element scratch for adjoint RHS (Gauss-point vectors)
  // eigen workspace at the eigen level
  int eig_nb = 0, eig_mmax = 0;
  double *V = nullptr, *KV = nullptr, *GV = nullptr, *EW = nullptr, *EKW = nullptr;
  double *Hs = nullptr, *Bs = nullptr, *Ys = nullptr, *Cs = nullptr, *gram_partial = nullptr;
  double* small_host = nullptr;  // pinned
  double* tri = nullptr;         // scratch of the split small eigensolver (reflectors, T, vectors)
  // Algorithm 2 smoothing: nodal stencil of K^j + sigma G^j and its squared row norms (sized for the
  // finest level, allocated only when kaczmarz_sweeps > 0)
  double* kz_S = nullptr;
  double* kz_rn2 = nullptr;
  // tensor-core Gram products of the eigensolver (partials in gram_partial): error flags [2]
  // (timed-out wait, non-finite input); used for vectors up to gtc_nmax long
  unsigned* gtc_err = nullptr;
  int64_t gtc_nmax = 0;
  // consistent sensitivities of the multilevel load factors (allocated when desc.consistent_sens is set on
  // the multilevel path): the coarse modes as the eigensolver returned them (K^l-orthonormal) and their
  // load factors, the pairing of the normalised fine modes with them (fine mode r = cs_scale[r] times the
  // solution from coarse mode cs_perm[r]), fine [q][n] fields Psi, w, P c, coarse [q][n_l] CG vectors
  double *cs_psi = nullptr, *cs_Kpsi = nullptr, *cs_b = nullptr, *cs_c = nullptr, *cs_r = nullptr, *cs_r0 = nullptr,
         *cs_z = nullptr, *cs_p = nullptr, *cs_ap = nullptr, *cs_t = nullptr;
  double *cs_Psi = nullptr, *cs_W = nullptr, *cs_C = nullptr;
  double* cs_scal = nullptr;     // device scalars [tobk::kCsSize]
  double cs_mu[64] = {0};
  double cs_scale[64] = {0};
  int cs_perm[64] = {0};
  bool cs_ready = false;  // the pairing of the last compute_buckling is recorded
  bool have_cs = false;   // the last compute_sensitivities took the consistent path
  // small scalars
  double* dscal = nullptr;       // device scratch scalars [256]
  double* hscal = nullptr;       // pinned host scratch [256]

  // CUDA graphs of CG iteration pairs, keyed by (level, RHS count, precision)
  struct CGGraph {
    cudaGraphExec_t exec;
    long long kernels;
  };
  std::map<uint64_t, CGGraph> cg_graphs;
  bool use_graphs = true;
  // Split multi-RHS solves: the second half of the right-hand sides runs on stream2 (forked from
  // and joined to the handle's stream by events), so that one half's latency-bound coarse levels
  // overlap the other half's FP64-bound fine level.  rhs_off = first RHS column of the half being
  // enqueued (0 otherwise); every RHS-sized work buffer is used from that column on.
  cudaStream_t stream2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int rhs_off = 0;
  // Early fine solve of the multilevel path (compute_buckling): the fine systems K phi = G P psi of
  // the coarse modes that have converged while the eigensolver still works on the others run on
  // streams of their own, on RHS columns q .. q + early_gmax - 1 of every work buffer (the eigensolver's
  // preconditioner uses columns 0 .. q - 1): coarse snapshot [early_gmax][n_l], prolongated modes,
  // right-hand sides and solutions [early_gmax][n]
  int early_gmax = 0;
  static constexpr int kEarlyStreams = 4;  // groups of early modes take these in turn (lowest priority)
  cudaStream_t stream3[kEarlyStreams] = {};
  cudaEvent_t ev_early[kEarlyStreams] = {};
  cudaStream_t stream_hi = nullptr, stream_hi2 = nullptr;  // the eigensolve meanwhile (highest priority)
  cudaEvent_t ev_snap = nullptr, ev_hi = nullptr;
  double *ea_psi = nullptr, *ea_Psi = nullptr, *ea_rhs = nullptr, *ea_Phi = nullptr, *ea_scale = nullptr;
  int la_iters = 0;  // CG iterations of the last linear analysis (sizes the early solve's queue)
  bool solve_only = false;

  // kernel-class timing
  struct ProfPending {
    int kc;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<ProfPending> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[TOBK_KC_COUNT] = {0};
  long long prof_cnt[TOBK_KC_COUNT] = {0};
  double prof_units[TOBK_KC_COUNT] = {0};  // DOF x RHS processed by the timed launches
  // phase timing of compute_buckling (CUDA events on the stream; see tobk_phase_read)
  bool phase_on = false;
  double phase_ms[TOBK_PHASE_COUNT] = {0};

  double compliance = 0.0;
  double lam_host[64];
  bool have_x = false, have_f = false, have_fixed = false, setup_done = false, have_u = false,
       have_G = false, have_modes = false, have_sens = false, have_u0 = false;
  std::string err;
};

namespace tobk {

// solve_only: allocate the multigrid hierarchy and CG work space only (no buckling / sensitivity
// storage); such a handle serves tobk_solve-style solves, e.g. as one design of a batch.
int create_handle(const tobk_desc* desc, void* stream, tobk_handle** out, bool solve_only = false);
void destroy_handle(tobk_handle* h);
int set_densities(tobk_handle* h, const double* x, bool on_device);
int set_load(tobk_handle* h, const double* f, bool on_device);
int set_fixed(tobk_handle* h, const uint8_t* fixed, bool on_device);
int setup_hierarchy(tobk_handle* h);
// lambda_max(D^{-1} K) per level and the smoother coefficients (called by setup_hierarchy)
void setup_smoothers(tobk_handle* h);
LevelOpDesc level_op(tobk_handle* h, int j);
// Multi-RHS MGCG solve at level s (0-based): K_s X = B, nr RHS (device, [nr][n_s]).
// fixed_iters: exactly max_iter iterations (rounded up to pairs) as an approximate inverse, without
// host synchronisation or exit check (a preconditioner)
int pcg_solve(tobk_handle* h, int s, const double* B, double* X, int nr, double rtol, int max_iter, bool use_x0,
              int precision, tobk_solve_info* info, bool fixed_iters = false);
// Enqueue-only multi-RHS CG at level s on RHS columns [off, off + nr) of every work buffer, on stream st,
// without host synchronisation: begin (from X0), iteration pairs, end (iterate copied to X).  The
// kernels deactivate a right-hand side once its recursive residual meets rtol ||b||.
void cg_async_begin(tobk_handle* h, cudaStream_t st, int off, int s, const double* B, const double* X0, int nr,
                    double rtol, int precision);
int cg_async_pairs(tobk_handle* h, cudaStream_t st, int off, int s, int nr, int pairs, int precision);
void cg_async_end(tobk_handle* h, cudaStream_t st, int off, int s, double* X, int nr);
int solve_equilibrium(tobk_handle* h, double* compliance, tobk_solve_info* info);
int setup_stress(tobk_handle* h);  // Gs from u, Galerkin G down to the eigen level
int compute_buckling(tobk_handle* h, double* lambda, tobk_solve_info* info);
int compute_sensitivities(tobk_handle* h, double* dlam, double* dJ, bool out_on_device, tobk_solve_info* info);
// consistent sensitivities (consistent.cu): the fine and coarse adjoints and the u-adjoint right-hand
// side g [q][n]; then, after K z = g, the derivative of the multilevel load factors into h->dlam
constexpr int kCsSize = 2240;
int consistent_adjoint_rhs(tobk_handle* h, double* g_out, tobk_solve_info* info);
void launch_sens_consistent(tobk_handle* h, const double* pGp);
// Called by eigen_solve after the convergence test of every outer iteration that did not finish:
// X [>= q][n] the current Ritz vectors (device, on the handle's stream; overwritten by the next
// iteration), theta [>= q] their Ritz values (host, descending; lambda = 1 / theta), conv[i] whether
// pair i < q meets eig_tol.
struct EigenHook {
  virtual ~EigenHook() = default;
  virtual void iteration(const double* X, int64_t n, const double* theta, const bool* conv, int q) = 0;
};
// eigensolver at level j: q lowest positive load factors, modes K_j-normalised -> out [q][n_j]
int eigen_solve(tobk_handle* h, int j, int q, double* out_modes, double* out_lam_host, tobk_solve_info* info,
                EigenHook* hook = nullptr);
// Rayleigh-Ritz projection of (K^j, G^j) on span Psi (q columns, stride n_j; Algorithm 2 'R[Psi]'):
// Psi is replaced by the K-normalised Ritz vectors, lam_host [q] by their load factors, ascending.
int ritz_level(tobk_handle* h, int j, int q, double* Psi, double* lam_host);
// G_j v at level j (fine: matrix-free from Gs; coarse: Galerkin Ge)
void apply_G_level(tobk_handle* h, int j, const double* v, double* y, int nr, int64_t stride);
void apply_K_level(tobk_handle* h, int j, const double* v, double* y, int nr, int64_t stride);
// out = M r: one multigrid V-cycle for K on level j and below (nr RHS, stride n_j); r must not be
// one of level j's own work vectors
void apply_vcycle(tobk_handle* h, int j, int nr, const double* r, double* out);
void prof_begin(tobk_handle* h, int kc, double units);
void prof_end(tobk_handle* h);
void prof_flush(tobk_handle* h);
int fail(tobk_handle* h, int code, const std::string& msg);
int check_cuda(tobk_handle* h, const char* where);

// CUDA events recorded on the handle's stream while phase timing is on (no-ops otherwise); read
// them only after the stream has passed the last mark.
struct PhaseMarks {
  tobk_handle* h;
  std::vector<cudaEvent_t> ev;
  explicit PhaseMarks(tobk_handle* hh) : h(hh) {}
  int mark() {
    if (!h->phase_on) return -1;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, h->stream);
    ev.push_back(e);
    return (int)ev.size() - 1;
  }
  double ms(int a, int b) const {
    if (a < 0 || b < 0 || a >= (int)ev.size() || b >= (int)ev.size()) return 0.0;
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[a], ev[b]);
    return t;
  }
  ~PhaseMarks() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

}  // namespace tobk
