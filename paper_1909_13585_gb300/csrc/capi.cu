// extern "C" entry points of libtobk.so (declared and documented in include/tobk.h).  The calls
// follow the paper's problem statement: densities, loads and supports, the linear analysis
// (Algorithm 1 step 3), the buckling analysis (Algorithm 1 steps 4-5 exact; Sec. 2.1 / Algorithm 2
// multilevel) and the sensitivities (eq. SensitivityLambda, eq. AdjointSystem).
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "handle.h"

using namespace tobk;

static thread_local std::string g_create_error;

namespace tobk {
// message of a failed call that has no handle (tobk_create, tobk_residual_noalloc), read through
// tobk_last_error(NULL) on the same thread
void set_handleless_error(const char* msg) { g_create_error = msg; }
}  // namespace tobk

#define TOBK_GUARD(h)                                  \
  do {                                                 \
    if (!(h)) return TOBK_E_ARG;                       \
  } while (0)

extern "C" {

int tobk_default_desc(tobk_desc* d) {
  if (!d) return TOBK_E_ARG;
  std::memset(d, 0, sizeof(*d));
  d->dim = 2;
  d->nel[0] = d->nel[1] = 4;
  d->nel[2] = 1;
  d->nu = 0.3;
  d->E0 = 1.0;
  d->Emin = 1e-6;
  d->penal = 3.0;
  d->mg_levels = 3;
  d->eig_level = 1;
  d->num_modes = 6;
  d->precision = TOBK_FP64;
  d->rtol = 1e-8;
  d->max_iter = 500;
  d->omega = 0.6;
  d->nu_pre = 2;
  d->nu_post = 2;
  d->eig_tol = 1e-8;
  d->eig_max_iter = 200;
  d->max_rhs = 10;
  d->eig_inner_iters = 2;
  d->fuse_load_adjoint = 0;
  d->smoother = TOBK_SMOOTHER_CHEBYSHEV;
  d->cheb_ratio = 10.0;
  d->kaczmarz_sweeps = 0;
  d->ritz_levels = 0;
  d->fine_steps = 1;
  d->element = TOBK_ELEMENT_PLAIN;
  d->eig_gram_tc = 0;
  d->consistent_sens = 0;
  d->early_fine = 1;
  return TOBK_OK;
}

int tobk_create(const tobk_desc* desc, void* cuda_stream, tobk_handle** out) {
  int rc = create_handle(desc, cuda_stream, out);
  if (rc != TOBK_OK) {
    g_create_error = rc == TOBK_E_ARG ? "invalid descriptor (sizes, levels, modes or parameters)"
                     : rc == TOBK_E_NOMEM ? "device allocation failed"
                                          : "CUDA error during creation";
  }
  return rc;
}

void tobk_destroy(tobk_handle* h) { destroy_handle(h); }

const char* tobk_last_error(const tobk_handle* h) {
  if (!h) return g_create_error.c_str();
  return h->err.c_str();
}

int tobk_set_densities(tobk_handle* h, const double* x, int64_t m, int on_device) {
  TOBK_GUARD(h);
  if (m != h->lv[0].g.m) return fail(h, TOBK_E_ARG, "density length != number of elements");
  return set_densities(h, x, on_device != 0);
}

int tobk_set_load(tobk_handle* h, const double* f, int64_t n, int on_device) {
  TOBK_GUARD(h);
  if (n != h->lv[0].g.n) return fail(h, TOBK_E_ARG, "load length != number of DOFs");
  return set_load(h, f, on_device != 0);
}

int tobk_set_fixed(tobk_handle* h, const uint8_t* fixed, int64_t n, int on_device) {
  TOBK_GUARD(h);
  if (n != h->lv[0].g.n) return fail(h, TOBK_E_ARG, "fixed-mask length != number of DOFs");
  return set_fixed(h, fixed, on_device != 0);
}

int tobk_set_initial_guess(tobk_handle* h, const double* u0, int64_t n, int on_device) {
  TOBK_GUARD(h);
  if (!u0) {
    h->have_u0 = false;
    return TOBK_OK;
  }
  if (n != h->lv[0].g.n) return fail(h, TOBK_E_ARG, "initial-guess length != number of DOFs");
  cudaMemcpyAsync(h->u0, u0, sizeof(double) * n, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                  h->stream);
  h->have_u0 = true;
  return check_cuda(h, "set_initial_guess");
}

int tobk_solve_equilibrium(tobk_handle* h, double* compliance, tobk_solve_info* info) {
  TOBK_GUARD(h);
  return solve_equilibrium(h, compliance, info);
}

int tobk_compute_buckling(tobk_handle* h, double* lambda, tobk_solve_info* info) {
  TOBK_GUARD(h);
  return compute_buckling(h, lambda, info);
}

int tobk_compute_sensitivities(tobk_handle* h, double* dlambda_dx, double* dJ_dx, int out_on_device,
                               tobk_solve_info* info) {
  TOBK_GUARD(h);
  return compute_sensitivities(h, dlambda_dx, dJ_dx, out_on_device != 0, info);
}

int tobk_get_field(tobk_handle* h, int which, double* out, int64_t len, int out_on_device) {
  TOBK_GUARD(h);
  if (!out) return fail(h, TOBK_E_ARG, "null output");
  const int64_t n = h->lv[0].g.n;
  const double* src = nullptr;
  int64_t need = 0;
  switch (which) {
    case TOBK_FIELD_U:
      if (!h->have_u) return fail(h, TOBK_E_STATE, "no displacement yet");
      src = h->u;
      need = n;
      break;
    case TOBK_FIELD_MODES:
      if (!h->have_modes) return fail(h, TOBK_E_STATE, "no modes yet");
      src = h->modes;
      need = (int64_t)h->q * n;
      break;
    case TOBK_FIELD_ADJOINT:
      if (!h->have_sens) return fail(h, TOBK_E_STATE, "no adjoints yet");
      src = h->adj;
      need = (int64_t)h->q * n;
      break;
    case TOBK_FIELD_ADJOINT_RHS:
      if (!h->have_sens) return fail(h, TOBK_E_STATE, "no adjoints yet");
      src = h->adj_rhs;
      need = (int64_t)h->q * n;
      break;
    case TOBK_FIELD_FINE_ADJOINT:
    case TOBK_FIELD_COARSE_ADJOINT:
    case TOBK_FIELD_PROLONGATED:
      if (!h->have_sens || !h->have_cs) return fail(h, TOBK_E_STATE, "no consistent sensitivities yet");
      src = which == TOBK_FIELD_FINE_ADJOINT ? h->cs_W : which == TOBK_FIELD_COARSE_ADJOINT ? h->cs_C : h->cs_Psi;
      need = (int64_t)h->q * n;
      break;
    default:
      return fail(h, TOBK_E_ARG, "unknown field");
  }
  if (len != need) return fail(h, TOBK_E_ARG, "field length mismatch");
  cudaMemcpyAsync(out, src, sizeof(double) * need, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                  h->stream);
  cudaStreamSynchronize(h->stream);
  return check_cuda(h, "get_field");
}

long long tobk_launch_count(void) { return g_launch_count.load(); }

int tobk_profile_enable(tobk_handle* h, int enable) {
  TOBK_GUARD(h);
  prof_flush(h);
  h->prof_on = enable != 0;
  if (h->prof_on)
    for (int k = 0; k < TOBK_KC_COUNT; ++k) {
      h->prof_ms[k] = 0.0;
      h->prof_cnt[k] = 0;
      h->prof_units[k] = 0.0;
    }
  return TOBK_OK;
}

int tobk_profile_read(tobk_handle* h, int kc, long long* launches, double* total_ms, double* dof_rhs) {
  TOBK_GUARD(h);
  if (kc < 0 || kc >= TOBK_KC_COUNT) return fail(h, TOBK_E_ARG, "bad kernel class");
  prof_flush(h);
  if (launches) *launches = h->prof_cnt[kc];
  if (total_ms) *total_ms = h->prof_ms[kc];
  if (dof_rhs) *dof_rhs = h->prof_units[kc];
  return check_cuda(h, "profile_read");
}

int tobk_phase_enable(tobk_handle* h, int enable) {
  TOBK_GUARD(h);
  h->phase_on = enable != 0;
  return TOBK_OK;
}

int tobk_phase_read(tobk_handle* h, double* out, int len) {
  TOBK_GUARD(h);
  if (!out || len < 0) return fail(h, TOBK_E_ARG, "bad phase output");
  for (int k = 0; k < len && k < TOBK_PHASE_COUNT; ++k) out[k] = h->phase_ms[k];
  return TOBK_OK;
}

int tobk_level_info(tobk_handle* h, int level, int64_t* out5) {
  TOBK_GUARD(h);
  if (!out5 || level < 1 || level > h->L) return fail(h, TOBK_E_ARG, "bad level");
  const Grid& g = h->lv[level - 1].g;
  out5[0] = g.nel[0];
  out5[1] = g.nel[1];
  out5[2] = g.nel[2];
  out5[3] = g.n;
  out5[4] = g.m;
  return TOBK_OK;
}

int tobk_apply_K(tobk_handle* h, int level, const double* v, double* y, int nrhs) {
  TOBK_GUARD(h);
  if (level < 1 || level > h->L || !v || !y || nrhs < 1 || nrhs > 65535) return fail(h, TOBK_E_ARG, "bad arguments");
  if (!h->setup_done) {
    int rc = setup_hierarchy(h);
    if (rc) return rc;
  }
  const int64_t n = h->lv[level - 1].g.n;
  apply_K_level(h, level - 1, v, y, nrhs, n);
  cudaStreamSynchronize(h->stream);
  return check_cuda(h, "apply_K");
}

int tobk_apply_G(tobk_handle* h, int level, const double* v, double* y, int nrhs) {
  TOBK_GUARD(h);
  if (level < 1 || level > h->eig + 1 || !v || !y || nrhs < 1 || nrhs > 65535)
    return fail(h, TOBK_E_ARG, "bad arguments (G is built on levels 1..eig_level)");
  if (!h->have_G) return fail(h, TOBK_E_STATE, "stress stiffness needs solve_equilibrium");
  const int64_t n = h->lv[level - 1].g.n;
  apply_G_level(h, level - 1, v, y, nrhs, n);
  cudaStreamSynchronize(h->stream);
  return check_cuda(h, "apply_G");
}

int tobk_solve(tobk_handle* h, int level, const double* B, double* X, int nrhs, tobk_solve_info* info) {
  TOBK_GUARD(h);
  if (level < 1 || level > h->L || !B || !X) return fail(h, TOBK_E_ARG, "bad arguments");
  if (nrhs < 1 || nrhs > h->rmax) return fail(h, TOBK_E_ARG, "nrhs exceeds the handle's RHS capacity");
  if (!h->setup_done) {
    int rc = setup_hierarchy(h);
    if (rc) return rc;
  }
  return pcg_solve(h, level - 1, B, X, nrhs, h->desc.rtol, h->desc.max_iter, false, h->desc.precision, info);
}

int tobk_get_element_matrices(tobk_handle* h, int level, int which, double* out, int64_t len) {
  TOBK_GUARD(h);
  if (level < 2 || level > h->L || !out) return fail(h, TOBK_E_ARG, "coarse level expected");
  const Level& L = h->lv[level - 1];
  const int64_t need = L.g.m * h->tab.nd * h->tab.nd;
  if (len != need) return fail(h, TOBK_E_ARG, "length mismatch");
  const double* src = which == 0 ? L.Ke : L.Ge;
  if (which == 1 && (!L.Ge || !h->have_G)) return fail(h, TOBK_E_STATE, "G not built on this level");
  if (which == 0 && !h->setup_done) {
    int rc = setup_hierarchy(h);
    if (rc) return rc;
  }
  cudaMemcpyAsync(out, src, sizeof(double) * need, cudaMemcpyDeviceToDevice, h->stream);
  cudaStreamSynchronize(h->stream);
  return check_cuda(h, "get_element_matrices");
}

}  // extern "C"

extern "C" int tobk_gram_tc(const double* A, int na, const double* B, int nb, int64_t n, int64_t stride, double* C,
                            void* cuda_stream) {
  using namespace tobk;
  if (!A || !B || !C || na < 1 || na > 64 || nb < 1 || nb > 64 || n < 1 || stride < n) return TOBK_E_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const size_t doubles = (size_t)gram_tc_chunks(n) * na * nb + 1;  // partials, then the two flags
  double* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, sizeof(double) * doubles, s) != cudaSuccess) {
    cudaGetLastError();
    return TOBK_E_NOMEM;
  }
  unsigned* err = reinterpret_cast<unsigned*>(buf + doubles - 1);
  cudaMemsetAsync(err, 0, 2 * sizeof(unsigned), s);
  launch_gram_tc(A, na, B, nb, n, stride, C, buf, err, s);
  unsigned herr[2] = {0, 0};
  cudaMemcpyAsync(herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(buf, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return TOBK_E_CUDA;
  if (herr[0]) return TOBK_E_TIMEOUT;
  if (herr[1]) return TOBK_E_NONFINITE;
  return TOBK_OK;
}
