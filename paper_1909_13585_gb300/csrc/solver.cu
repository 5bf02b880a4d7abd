// Host orchestration: element tables, handle memory, multigrid hierarchy set-up, V-cycle and the
// multi-RHS preconditioned CG driver (paper Appendix A: mgPCG / mgBPCG), linear analysis
// (Algorithm 1 step 2) and the stress-stiffness set-up (Algorithm 1 step 3, Algorithm 2 line 5).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>

#include "handle.h"
#include "unit_element.h"

namespace tobk {

std::atomic<long long> g_launch_count{0};

static thread_local const double* t_active_rhs = nullptr;
const double* active_rhs() { return t_active_rhs; }
void set_active_rhs(const double* sc) { t_active_rhs = sc; }

namespace {
struct ActiveRhsScope {
  explicit ActiveRhsScope(const double* sc) { set_active_rhs(sc); }
  ~ActiveRhsScope() { set_active_rhs(nullptr); }
};
}  // namespace

// ================================================================================================
// element tables (Gauss-Legendre 2-point rule per axis; exact for Q4/H8 on unit elements)
// ================================================================================================
ElementTables make_element_tables(int dim, double nu, int element) {
  namespace ue = unit_element;
  ElementTables t;
  t.dim = dim;
  t.element = element;
  t.nn = ue::nodes(dim);
  t.nd = ue::dofs(dim);
  t.ngp = t.nn;
  t.nv = ue::voigt(dim);
  const int nn = t.nn, nd = t.nd, nv = t.nv;
  auto xi_node = ue::xi_node;
  t.wdet = ue::weight_det(dim);
  t.dN.assign((size_t)t.ngp * dim * nn, 0.0);
  for (int q = 0; q < t.ngp; ++q) ue::shape_gradients(dim, q, &t.dN[(size_t)q * dim * nn]);
  t.D.assign((size_t)nv * nv, 0.0);
  ue::constitutive(dim, nu, t.D.data());
  t.Ke0.assign((size_t)nd * nd, 0.0);
  if (element == TOBK_ELEMENT_INCOMPATIBLE) {
    t.A.assign((size_t)ue::internal_dofs(dim) * nd, 0.0);
    ue::incompatible_tables(dim, nu, t.Ke0.data(), t.A.data());
  } else {
    ue::stiffness(dim, nu, t.Ke0.data());
  }
  // interpolation weights child node -> coarse element node, per child position
  t.W.assign((size_t)nn * nn * nn, 0.0);
  for (int kc = 0; kc < nn; ++kc)
    for (int l = 0; l < nn; ++l)
      for (int b = 0; b < nn; ++b) {
        double w = 1.0;
        for (int a = 0; a < dim; ++a) {
          const int ka = xi_node(kc, a) > 0 ? 1 : 0;
          const int la = xi_node(l, a) > 0 ? 1 : 0;
          const int ba = xi_node(b, a) > 0 ? 1 : 0;
          const double p = 0.5 * (ka + la);
          w *= ba ? p : 1.0 - p;
        }
        t.W[((size_t)kc * nn + l) * nn + b] = w;
      }
  return t;
}

// ================================================================================================
// errors
// ================================================================================================
int fail(tobk_handle* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int check_cuda(tobk_handle* h, const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, TOBK_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return TOBK_OK;
}

// ================================================================================================
// handle memory
// ================================================================================================
static void layout(tobk_handle* h, Arena& a) {
  const int nn = h->tab.nn, nd = h->tab.nd;
  const bool mixed = h->desc.precision == TOBK_FP32_VCYCLE;
  const int rm = h->rmax;
  for (int j = 0; j < h->L; ++j) {
    Level& L = h->lv[j];
    const int64_t n = L.g.n, m = L.g.m;
    L.fixed = a.take<uint8_t>(n);
    if (j > 0) {
      const int ne = (h->dim == 2 ? 9 : 27) * h->dim * h->dim;
      L.Ke = a.take<double>(m * nd * nd);
      if (mixed) L.Ke32 = a.take<float>(m * nd * nd);
      L.S = a.take<double>((size_t)ne * L.g.nnode);
      if (mixed) L.S32 = a.take<float>((size_t)ne * L.g.nnode);
    }
    if (j > 0 && j <= h->eig) L.Ge = a.take<double>(m * nd * nd);
    L.dinv = a.take<double>(n);
    if (mixed) L.dinv32 = a.take<float>(n);
    L.coef = a.take<double>(2 * kMaxSmoothSteps + 1);
    if (mixed) L.coef32 = a.take<float>(2 * kMaxSmoothSteps);
    if (h->desc.smoother == TOBK_SMOOTHER_CHEBYSHEV && j + 1 < h->L) {
      if (mixed) {
        L.dA32 = a.take<float>(rm * n);
        L.dB32 = a.take<float>(rm * n);
      } else {
        L.dA = a.take<double>(rm * n);
        L.dB = a.take<double>(rm * n);
      }
    }
    L.b = a.take<double>(rm * n);
    L.z = a.take<double>(rm * n);
    L.t = a.take<double>(rm * n);
    L.r = a.take<double>(rm * n);
    if (mixed) {
      L.b32 = a.take<float>(rm * n);
      L.z32 = a.take<float>(rm * n);
      L.t32 = a.take<float>(rm * n);
      L.r32 = a.take<float>(rm * n);
    }
  }
  const Grid& g = h->lv[0].g;
  h->d_Ke0 = a.take<double>(nd * nd);
  h->d_W = a.take<double>(nn * nn * nn);
  h->d_dN = a.take<double>(h->tab.dN.size());
  h->d_D = a.take<double>(h->tab.D.size());
  h->x = a.take<double>(g.m);
  h->Ek = a.take<double>(g.m);
  h->Es = a.take<double>(g.m);
  h->dEk = a.take<double>(g.m);
  h->dEs = a.take<double>(g.m);
  h->Ek32 = a.take<float>(g.m);
  h->f = a.take<double>(g.n);
  h->u = a.take<double>(g.n);
  h->u0 = a.take<double>(g.n);
  if (!h->solve_only) {
    h->Gs0 = a.take<double>(g.m * nn * nn);
    h->Gs = a.take<double>(g.m * nn * nn);
    if (h->tab.element == TOBK_ELEMENT_INCOMPATIBLE) {
      const int nf = nn + h->dim;
      h->d_A = a.take<double>(h->tab.A.size());
      h->Gfull = a.take<double>(g.m * nf * nf);
      h->Gc0 = a.take<double>(g.m * nd * nd);
    }
  }
  const int64_t nc = h->lv[h->L - 1].g.n;
  h->Adense = a.take<double>(nc * nc);
  h->Awork = a.take<double>(nc * nc);
  const int64_t nf = g.n;
  h->cg.x = a.take<double>(rm * nf);
  h->cg.r = a.take<double>(rm * nf);
  h->cg.z = a.take<double>(rm * nf);
  h->cg.zt = a.take<double>(rm * nf);
  h->cg.p0 = a.take<double>(rm * nf);
  h->cg.p1 = a.take<double>(rm * nf);
  h->cg.q = a.take<double>(rm * nf);
  h->cg.sc = a.take<double>((size_t)kMaxRhs * kScStride);
  h->cg.partial = a.take<double>((size_t)kMaxRhs * cg_partial_stride(g));
  h->cg.counters = a.take<unsigned>((size_t)kNumCounterSets * kMaxRhs);
  h->bwork = a.take<double>(rm * nf);
  h->xwork = a.take<double>(rm * nf);
  if (h->solve_only) {  // linear solves only (a member of a batch): no buckling or sensitivity storage
    h->dscal = a.take<double>(1024);
    return;
  }
  const int q = h->q;
  h->modes = a.take<double>((size_t)q * nf);
  h->lam = a.take<double>(q);
  // [load | q adjoint right-hand sides] and [u | q adjoint solutions], so that the fused solve
  // K [u, Z] = [f, B] is one contiguous (q+1)-RHS block
  h->adj_blockB = a.take<double>((size_t)(q + 1) * nf);
  h->adj_blockX = a.take<double>((size_t)(q + 1) * nf);
  h->adj_rhs = h->adj_blockB + nf;
  h->adj = h->adj_blockX + nf;
  h->dlam = a.take<double>((size_t)q * g.m);
  h->dJ = a.take<double>(g.m);
  h->esens = a.take<double>((size_t)g.m * h->tab.ngp * h->tab.nv);
  // eigen workspace at the eigen level
  const int64_t ne = h->lv[h->eig].g.n;
  const int mm = h->eig_mmax, nb = h->eig_nb;
  h->V = a.take<double>((size_t)mm * ne);
  h->KV = a.take<double>((size_t)mm * ne);
  h->GV = a.take<double>((size_t)mm * ne);
  h->EW = a.take<double>((size_t)(4 * nb + mm) * ne);   // X, KX, GX, W blocks + restart scratch
  h->EKW = a.take<double>((size_t)2 * nb * ne);
  h->Hs = a.take<double>((size_t)mm * mm);
  h->Bs = a.take<double>((size_t)mm * mm);
  h->Ys = a.take<double>((size_t)mm * mm);
  h->Cs = a.take<double>((size_t)mm * mm);
  // Rayleigh-Ritz scratch: five [mm][mm] matrices (FP32-stage and refined eigenvectors, S, R, wanted
  // columns), the refined eigenvalues and the refinement bound
  h->tri = a.take<double>(5 * (size_t)mm * mm + (size_t)mm + 8);
  const int64_t gp_rows = std::max<int64_t>(gram_partial_blocks(ne), gram_partial_blocks(nf));
  h->gram_partial = a.take<double>((size_t)gp_rows * mm * std::max(mm, nb));
  h->dscal = a.take<double>(1024);
  if (h->desc.eig_gram_tc) {  // partials of at most n / 128 chunks fit in gram_partial
    h->gtc_nmax = std::max(ne, nf);
    h->gtc_err = a.take<unsigned>(2);
  }
  if (h->early_gmax > 0) {
    const int64_t nl = h->lv[h->eig].g.n;
    const int ge = h->early_gmax;
    h->ea_psi = a.take<double>((size_t)ge * nl);
    h->ea_Psi = a.take<double>((size_t)ge * nf);
    h->ea_rhs = a.take<double>((size_t)ge * nf);
    h->ea_Phi = a.take<double>((size_t)ge * nf);
    h->ea_scale = a.take<double>(64);
  }
  if (h->desc.consistent_sens && h->eig > 0) {
    const int64_t nl = h->lv[h->eig].g.n;
    for (double** v : {&h->cs_psi, &h->cs_Kpsi, &h->cs_b, &h->cs_c, &h->cs_r, &h->cs_r0, &h->cs_z, &h->cs_p,
                       &h->cs_ap, &h->cs_t})
      *v = a.take<double>((size_t)q * nl);
    h->cs_Psi = a.take<double>((size_t)q * nf);
    h->cs_W = a.take<double>((size_t)q * nf);
    h->cs_C = a.take<double>((size_t)q * nf);
    h->cs_scal = a.take<double>(kCsSize);
  }
  if (h->desc.kaczmarz_sweeps > 0 && h->eig > 0) {
    const int d = h->dim;
    h->kz_S = a.take<double>((size_t)(d == 2 ? 9 : 27) * d * d * g.nnode);
    h->kz_rn2 = a.take<double>((size_t)nf);
  }
}

int create_handle(const tobk_desc* d, void* stream, tobk_handle** out, bool solve_only) {
  if (!d || !out) return TOBK_E_ARG;
  *out = nullptr;
  if (d->dim != 2 && d->dim != 3) return TOBK_E_ARG;
  if (d->mg_levels < 1 || d->mg_levels > kMaxLevels) return TOBK_E_ARG;
  if (d->eig_level < 1 || d->eig_level > d->mg_levels) return TOBK_E_ARG;
  if (d->num_modes < 1 || d->num_modes > 24) return TOBK_E_ARG;
  if (d->nu_pre < 1 || d->nu_post < 0 || !(d->omega > 0.0) || !(d->rtol > 0.0) || d->max_iter < 1) return TOBK_E_ARG;
  if (d->nu_pre > kMaxSmoothSteps || d->nu_post > kMaxSmoothSteps) return TOBK_E_ARG;
  if (d->smoother != TOBK_SMOOTHER_JACOBI && d->smoother != TOBK_SMOOTHER_CHEBYSHEV) return TOBK_E_ARG;
  if (d->smoother == TOBK_SMOOTHER_CHEBYSHEV && !(d->cheb_ratio > 1.0)) return TOBK_E_ARG;
  if (!(d->nu > -1.0 && d->nu < 0.5) || !(d->E0 > 0.0) || !(d->Emin > 0.0) || !(d->penal >= 1.0)) return TOBK_E_ARG;
  if (d->precision != TOBK_FP64 && d->precision != TOBK_FP32_VCYCLE) return TOBK_E_ARG;
  if (d->kaczmarz_sweeps < 0 || d->kaczmarz_sweeps > 64 || (d->ritz_levels != 0 && d->ritz_levels != 1) ||
      d->fine_steps < 0 || d->fine_steps > 64)
    return TOBK_E_ARG;
  if (d->element != TOBK_ELEMENT_PLAIN && d->element != TOBK_ELEMENT_INCOMPATIBLE) return TOBK_E_ARG;
  if (d->element != TOBK_ELEMENT_PLAIN && solve_only) return TOBK_E_ARG;  // batches: plain elements only
  if (d->eig_gram_tc != 0 && d->eig_gram_tc != 1) return TOBK_E_ARG;
  if (d->consistent_sens != 0 && d->consistent_sens != 1) return TOBK_E_ARG;
  if (d->consistent_sens && d->eig_level > 1 &&
      (d->kaczmarz_sweeps > 0 || d->ritz_levels || d->fine_steps > 1 || d->element != TOBK_ELEMENT_PLAIN))
    return TOBK_E_ARG;  // the derivative follows Sec. 2.1 steps 1-4 with plain elements only
  for (int a = 0; a < d->dim; ++a) {
    if (d->nel[a] < 1) return TOBK_E_ARG;
    if (d->nel[a] % (1 << (d->mg_levels - 1)) != 0) return TOBK_E_ARG;
  }
  tobk_handle* h = new tobk_handle();
  h->desc = *d;
  h->solve_only = solve_only;
  h->stream = (cudaStream_t)stream;
  cudaGetDevice(&h->device);
  h->dim = d->dim;
  h->L = d->mg_levels;
  h->eig = d->eig_level - 1;
  h->q = d->num_modes;
  h->eig_nb = h->q;  // block = wanted pairs: as few iterations as q + 2 or q + 4 (measured), less work each
  h->eig_mmax = 64;
  h->rmax = std::max({d->max_rhs, h->eig_nb, h->q + 1, 1});
  // Sec. 2.1 steps 1-4 as they stand: columns beside the eigensolver's for the early fine solve
  if (d->early_fine != 0 && d->early_fine != 1) return TOBK_E_ARG;
  if (!solve_only && d->early_fine && d->eig_level > 1 && d->kaczmarz_sweeps == 0 && !d->ritz_levels &&
      d->fine_steps <= 1 && stream != nullptr) {
    const int want = std::max(2, h->q - 1);
    h->rmax = std::max(h->rmax, std::min(kMaxRhs, h->q + want));
    h->early_gmax = std::min(want, h->rmax - h->q);
  }
  if (h->rmax > kMaxRhs || h->eig_mmax < 2 * h->eig_nb) {
    delete h;
    return TOBK_E_ARG;
  }
  h->tab = make_element_tables(d->dim, d->nu, d->element);
  int nel[3] = {d->nel[0], d->nel[1], d->dim == 3 ? d->nel[2] : 1};
  for (int j = 0; j < h->L; ++j) {
    h->lv[j].g = make_grid(d->dim, nel);
    for (int a = 0; a < d->dim; ++a) nel[a] /= 2;
  }
  if (h->lv[h->L - 1].g.n > 6000) {
    delete h;
    return TOBK_E_ARG;
  }
  Arena sizing;
  sizing.base = nullptr;
  sizing.cap = ~size_t(0) >> 1;
  layout(h, sizing);
  const size_t bytes = sizing.used + 4096;
  void* base = nullptr;
  if (cudaMalloc(&base, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return TOBK_E_NOMEM;
  }
  h->arena.base = (char*)base;
  h->arena.cap = bytes;
  h->arena.used = 0;
  layout(h, h->arena);
  if (cudaMallocHost(&h->cg.host_sc, sizeof(double) * kMaxRhs * kScStride) != cudaSuccess ||
      cudaMallocHost(&h->hscal, sizeof(double) * 1024) != cudaSuccess ||
      cudaMallocHost(&h->small_host, sizeof(double) * 4 * 96 * 96) != cudaSuccess) {
    cudaGetLastError();
    destroy_handle(h);
    return TOBK_E_NOMEM;
  }
  if (h->stream != nullptr &&
      (cudaStreamCreateWithFlags(&h->stream2, cudaStreamNonBlocking) != cudaSuccess ||
       cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
       cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    destroy_handle(h);
    return TOBK_E_CUDA;
  }
  int prio_low = 0, prio_high = 0;
  cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  bool early_ok = true;
  if (h->early_gmax > 0) {
    for (int k = 0; k < tobk_handle::kEarlyStreams; ++k)
      early_ok = early_ok &&
                 cudaStreamCreateWithPriority(&h->stream3[k], cudaStreamNonBlocking, prio_low) == cudaSuccess &&
                 cudaEventCreateWithFlags(&h->ev_early[k], cudaEventDisableTiming) == cudaSuccess;
    early_ok = early_ok &&
               cudaStreamCreateWithPriority(&h->stream_hi, cudaStreamNonBlocking, prio_high) == cudaSuccess &&
               cudaStreamCreateWithPriority(&h->stream_hi2, cudaStreamNonBlocking, prio_high) == cudaSuccess &&
               cudaEventCreateWithFlags(&h->ev_snap, cudaEventDisableTiming) == cudaSuccess &&
               cudaEventCreateWithFlags(&h->ev_hi, cudaEventDisableTiming) == cudaSuccess;
  }
  if (!early_ok) {
    cudaGetLastError();
    destroy_handle(h);
    return TOBK_E_CUDA;
  }
  cudaStream_t s = h->stream;
  cudaMemsetAsync(h->arena.base, 0, bytes, s);
  cudaMemcpyAsync(h->d_Ke0, h->tab.Ke0.data(), sizeof(double) * h->tab.Ke0.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->d_W, h->tab.W.data(), sizeof(double) * h->tab.W.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->d_dN, h->tab.dN.data(), sizeof(double) * h->tab.dN.size(), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(h->d_D, h->tab.D.data(), sizeof(double) * h->tab.D.size(), cudaMemcpyHostToDevice, s);
  if (h->d_A) cudaMemcpyAsync(h->d_A, h->tab.A.data(), sizeof(double) * h->tab.A.size(), cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
  if (check_cuda(h, "tobk_create") != TOBK_OK) {
    destroy_handle(h);
    return TOBK_E_CUDA;
  }
  *out = h;
  return TOBK_OK;
}

void destroy_handle(tobk_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  if (h->stream2) {
    cudaStreamSynchronize(h->stream2);
    cudaStreamDestroy(h->stream2);
  }
  for (int k = 0; k < tobk_handle::kEarlyStreams; ++k) {
    if (h->stream3[k]) {
      cudaStreamSynchronize(h->stream3[k]);
      cudaStreamDestroy(h->stream3[k]);
    }
    if (h->ev_early[k]) cudaEventDestroy(h->ev_early[k]);
  }
  for (cudaStream_t* sp : {&h->stream_hi, &h->stream_hi2})
    if (*sp) {
      cudaStreamSynchronize(*sp);
      cudaStreamDestroy(*sp);
    }
  if (h->ev_hi) cudaEventDestroy(h->ev_hi);
  if (h->ev_snap) cudaEventDestroy(h->ev_snap);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  for (auto& p : h->prof_pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : h->prof_pool) cudaEventDestroy(e);
  for (auto& kv : h->cg_graphs) cudaGraphExecDestroy(kv.second.exec);
  if (h->arena.base) cudaFree(h->arena.base);
  if (h->cg.host_sc) cudaFreeHost(h->cg.host_sc);
  if (h->hscal) cudaFreeHost(h->hscal);
  if (h->small_host) cudaFreeHost(h->small_host);
  delete h;
}

// ================================================================================================
// inputs
// ================================================================================================
static int copy_in(tobk_handle* h, void* dst, const void* src, size_t bytes, bool on_device) {
  cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
  return check_cuda(h, "copy");
}

int set_densities(tobk_handle* h, const double* x, bool on_device) {
  const int64_t m = h->lv[0].g.m;
  if (!x) return fail(h, TOBK_E_ARG, "null densities");
  if (!on_device) {
    for (int64_t e = 0; e < m; ++e)
      if (!(x[e] >= 0.0 && x[e] <= 1.0)) return fail(h, TOBK_E_ARG, "density not finite or outside [0,1]");
  }
  int rc = copy_in(h, h->x, x, sizeof(double) * m, on_device);
  if (rc) return rc;
  h->have_x = true;
  h->setup_done = h->have_u = h->have_G = h->have_modes = h->have_sens = false;
  return TOBK_OK;
}

int set_load(tobk_handle* h, const double* f, bool on_device) {
  if (!f) return fail(h, TOBK_E_ARG, "null load");
  int rc = copy_in(h, h->f, f, sizeof(double) * h->lv[0].g.n, on_device);
  if (rc) return rc;
  h->have_f = true;
  h->have_u = h->have_G = h->have_modes = h->have_sens = false;
  return TOBK_OK;
}

__global__ void k_coarsen_fixed(Grid gf, Grid gc, const uint8_t* ff, uint8_t* fc) {
  const int64_t cn = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (cn >= gc.nnode) return;
  const int I = (int)(cn % gc.nn[0]);
  const int64_t t = cn / gc.nn[0];
  const int J = (int)(t % gc.nn[1]);
  const int K = (int)(t / gc.nn[1]);
  const int64_t fn = 2 * I + (int64_t)gf.nn[0] * (2 * J + (int64_t)gf.nn[1] * 2 * K);
  for (int c = 0; c < gc.dim; ++c) fc[gc.dim * cn + c] = ff[gf.dim * fn + c] ? 1 : 0;
}

__global__ void k_normalize_fixed(uint8_t* f, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = f[i] ? 1 : 0;
}

int set_fixed(tobk_handle* h, const uint8_t* fixed, bool on_device) {
  if (!fixed) return fail(h, TOBK_E_ARG, "null fixed mask");
  const int64_t n = h->lv[0].g.n;
  int rc = copy_in(h, h->lv[0].fixed, fixed, n, on_device);
  if (rc) return rc;
  ::tobk::note_launch(), k_normalize_fixed<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(h->lv[0].fixed, n);
  for (int j = 1; j < h->L; ++j) {
    const Grid& gc = h->lv[j].g;
    ::tobk::note_launch(), k_coarsen_fixed<<<(unsigned)((gc.nnode + 255) / 256), 256, 0, h->stream>>>(h->lv[j - 1].g, gc, h->lv[j - 1].fixed,
                                                                                h->lv[j].fixed);
  }
  h->have_fixed = true;
  h->setup_done = h->have_u = h->have_G = h->have_modes = h->have_sens = false;
  return check_cuda(h, "set_fixed");
}

// ================================================================================================
// hierarchy
// ================================================================================================
LevelOpDesc level_op(tobk_handle* h, int j) {
  LevelOpDesc d{};
  d.g = h->lv[j].g;
  d.fixed = h->lv[j].fixed;
  d.nu = h->desc.nu;
  d.element = h->tab.element;
  if (j == 0) {
    d.stored = false;
    d.scale64 = h->Ek;
    d.scale32 = h->Ek32;
    d.T0 = h->tab.Ke0.data();
    d.T0dev = h->d_Ke0;
  } else {
    d.stored = true;
    d.Ke64 = h->lv[j].Ke;
    d.Ke32 = h->lv[j].Ke32;
    d.S64 = h->lv[j].S;
    d.S32 = h->lv[j].S32;
  }
  return d;
}

int setup_hierarchy(tobk_handle* h) {
  if (!h->have_x) return fail(h, TOBK_E_STATE, "densities not set");
  if (!h->have_fixed) return fail(h, TOBK_E_STATE, "fixed DOFs not set");
  cudaStream_t s = h->stream;
  const tobk_desc& d = h->desc;
  const bool mixed = d.precision == TOBK_FP32_VCYCLE;
  const Grid& g0 = h->lv[0].g;
  launch_simp(h->x, g0.m, d.penal, d.E0, d.Emin, h->Ek, h->Es, h->dEk, h->dEs, h->Ek32, s);
  launch_diag(level_op(h, 0), h->lv[0].dinv, mixed ? h->lv[0].dinv32 : nullptr, s);
  const int nd2 = h->tab.nd * h->tab.nd;
  for (int j = 1; j < h->L; ++j) {
    Level& Lc = h->lv[j];
    const Level& Lf = h->lv[j - 1];
    if (j == 1)
      launch_galerkin_fine_K(Lf.g, Lc.g, Lf.fixed, h->Ek, h->d_Ke0, h->d_W, Lc.Ke, s);
    else
      launch_galerkin_stored(Lf.g, Lc.g, Lf.fixed, Lf.Ke, h->d_W, Lc.Ke, s);
    if (mixed) launch_f64_to_f32(Lc.Ke, Lc.Ke32, Lc.g.m * nd2, s);
    launch_diag(level_op(h, j), Lc.dinv, mixed ? Lc.dinv32 : nullptr, s);
    launch_stencil_assemble(Lc.g, Lc.Ke, Lc.fixed, Lc.S, mixed ? Lc.S32 : nullptr, s);
  }
  // The coarsest inverse (a chain of pivot blocks, each on one SM) and the smoothers' eigenvalue
  // bounds (power iterations on every smoothing level) depend on the Galerkin operators only and not
  // on each other: with a second stream they run concurrently.
  const int jc = h->L - 1;
  cudaStream_t sc = s;
  if (h->stream2 != nullptr) {
    cudaEventRecord(h->ev_fork, s);
    cudaStreamWaitEvent(h->stream2, h->ev_fork, 0);
    sc = h->stream2;
  }
  launch_dense_assemble(level_op(h, jc), h->Adense, sc);
  h->Ainv = launch_dense_invert(h->Adense, h->Awork, h->lv[jc].g.n, h->dscal + 1000, sc);
  setup_smoothers(h);
  if (sc != s) {
    cudaEventRecord(h->ev_join, sc);
    cudaStreamWaitEvent(s, h->ev_join, 0);
  }
  int rc = check_cuda(h, "setup_hierarchy");
  if (rc) return rc;
  h->setup_done = true;
  return TOBK_OK;
}

// ================================================================================================
// V-cycle (multigrid preconditioner)
// ================================================================================================
// ================================================================================================
// kernel-class timing (CUDA events around selected launches while profiling is enabled)
// ================================================================================================
void prof_begin(tobk_handle* h, int kc, double units) {
  if (!h->prof_on) return;
  h->prof_units[kc] += units;
  cudaEvent_t a, b;
  if (h->prof_pool.size() >= 2) {
    a = h->prof_pool.back();
    h->prof_pool.pop_back();
    b = h->prof_pool.back();
    h->prof_pool.pop_back();
  } else {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  cudaEventRecord(a, h->stream);
  h->prof_pending.push_back({kc, a, b});
}

void prof_end(tobk_handle* h) {
  if (!h->prof_on || h->prof_pending.empty()) return;
  cudaEventRecord(h->prof_pending.back().b, h->stream);
  if (h->prof_pending.size() > 4096) prof_flush(h);
}

void prof_flush(tobk_handle* h) {
  if (h->prof_pending.empty()) return;
  cudaStreamSynchronize(h->stream);
  for (auto& p : h->prof_pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.a, p.b);
    h->prof_ms[p.kc] += ms;
    h->prof_cnt[p.kc] += 1;
    h->prof_pool.push_back(p.a);
    h->prof_pool.push_back(p.b);
  }
  h->prof_pending.clear();
}

// The level's work buffers from RHS column h->rhs_off on (vectors are [rhs][n] blocks); per-DOF data
// (mask, operator, diagonal, smoother coefficients) is shared by all right-hand sides.
static Level lvl(tobk_handle* h, int j) {
  Level L = h->lv[j];
  const int64_t o = (int64_t)h->rhs_off * L.g.n;
  if (o) {
    for (double** p : {&L.dA, &L.dB, &L.b, &L.z, &L.t, &L.r})
      if (*p) *p += o;
    for (float** p : {&L.dA32, &L.dB32, &L.b32, &L.z32, &L.t32, &L.r32})
      if (*p) *p += o;
  }
  return L;
}

// The CG work space from RHS column h->rhs_off on: vectors of length n, per-RHS scalars and
// counters, and reduction partials (each kernel writes partial + rhs * its stride, every stride at
// most the fine level's cg_partial_stride, which the buffer is sized for per RHS).
static CGWork cgw(tobk_handle* h, int64_t n) {
  CGWork w = h->cg;
  const int r = h->rhs_off;
  if (r) {
    const int64_t o = (int64_t)r * n;
    for (double** p : {&w.x, &w.r, &w.z, &w.zt, &w.p0, &w.p1, &w.q}) *p += o;
    w.sc += (size_t)r * kScStride;
    w.host_sc += (size_t)r * kScStride;
    w.partial += (size_t)r * cg_partial_stride(h->lv[0].g);
    w.counters += r;
  }
  return w;
}

// Node x RHS count below which a 2D stencil level fuses its residual into the restriction.
constexpr int64_t kFusedResidualWork = 131072;

// z0_ready: the restriction into this level already took the first smoothing step (z, dA written)
static double* vcycle64(tobk_handle* h, int j, int nr, const double* b, double* z, double* t, bool z0_ready = false) {
  cudaStream_t s = h->stream;
  const Level L = lvl(h, j);
  const int64_t n = L.g.n;
  const int ks = j == 0 ? TOBK_KC_FINE_SMOOTH : TOBK_KC_COARSE;
  const int kr = j == 0 ? TOBK_KC_FINE_RESIDUAL : TOBK_KC_COARSE;
  if (j == h->L - 1) {
    prof_begin(h, TOBK_KC_COARSEST, (double)nr * n);
    launch_dense_gemv(h->Ainv, b, z, n, nr, n, s);
    prof_end(h);
    return z;
  }
  const LevelOpDesc op = level_op(h, j);
  // smoothing steps: Chebyshev keeps its increment in dA/dB; damped Jacobi needs none
  double* dA = L.dA;
  double* dB = L.dB;
  if (!z0_ready) {
    prof_begin(h, TOBK_KC_VECTOR, (double)nr * n);
    launch_jacobi0(b, L.dinv, z, SmoothArgs<double>{L.coef, nullptr, dA}, n, nr, n, s);
    prof_end(h);
  }
  for (int it = 1; it < h->desc.nu_pre; ++it) {
    prof_begin(h, ks, (double)nr * n);
    launch_apply(op, APPLY_JAC, z, b, L.dinv, t, SmoothArgs<double>{L.coef + 2 * it, dA, dB}, nr, n, s);
    prof_end(h);
    std::swap(z, t);
    std::swap(dA, dB);
  }
  const Level C = lvl(h, j + 1);
  const bool fuse = j + 1 < h->L - 1;  // the coarse level smooths (it is not the dense coarsest)
  // 2D stencil levels fuse residual + restriction and prolongation + first post-smoothing step.  The
  // fused residual recomputes the tile halos (about an eighth more FP64 work), which pays only while
  // the level is latency-bound: large levels with many right-hand sides keep the two launches.
  const bool fused_transfers = op.S64 != nullptr && op.g.dim == 2;
  const bool fused_res = fused_transfers && op.g.nnode * nr < kFusedResidualWork;
  if (fused_res) {
    prof_begin(h, kr, (double)nr * n);
    launch_stencil_res_restrict_2d<double>(op.g, C.g, op.S64, op.fixed, z, b, n, C.fixed, C.b, C.g.n,
                                           fuse ? C.dinv : nullptr, fuse ? C.coef : nullptr, fuse ? C.z : nullptr,
                                           fuse ? C.dA : nullptr, nr, s);
    prof_end(h);
  } else {
    prof_begin(h, kr, (double)nr * n);
    launch_apply(op, APPLY_RES, z, b, nullptr, L.r, SmoothArgs<double>{}, nr, n, s);
    prof_end(h);
    prof_begin(h, TOBK_KC_TRANSFER, (double)nr * n);
    if (fuse)
      launch_restrict(L.g, C.g, C.fixed, L.r, C.b, nr, n, C.g.n, s, C.dinv, C.coef, C.z, C.dA);
    else
      launch_restrict(L.g, C.g, C.fixed, L.r, C.b, nr, n, C.g.n, s);
    prof_end(h);
  }
  double* zc = vcycle64(h, j + 1, nr, C.b, C.z, C.t, fuse);
  int it0 = 0;
  if (fused_transfers && h->desc.nu_post > 0) {
    prof_begin(h, ks, (double)nr * n);
    launch_stencil_jac_prolong_2d<double>(op.g, C.g, op.S64, op.fixed, z, zc, b, L.dinv, t,
                                          SmoothArgs<double>{L.coef, nullptr, dB}, nr, n, C.g.n, s);
    prof_end(h);
    std::swap(z, t);
    std::swap(dA, dB);
    it0 = 1;
  } else {
    prof_begin(h, TOBK_KC_TRANSFER, (double)nr * n);
    launch_prolong_add(L.g, C.g, L.fixed, zc, z, nr, n, C.g.n, s);
    prof_end(h);
  }
  for (int it = it0; it < h->desc.nu_post; ++it) {
    prof_begin(h, ks, (double)nr * n);
    launch_apply(op, APPLY_JAC, z, b, L.dinv, t, SmoothArgs<double>{L.coef + 2 * it, it == 0 ? nullptr : dA, dB},
                 nr, n, s);
    prof_end(h);
    std::swap(z, t);
    std::swap(dA, dB);
  }
  return z;
}

static float* vcycle32(tobk_handle* h, int j, int nr, const float* b, float* z, float* t, bool z0_ready = false) {
  cudaStream_t s = h->stream;
  const Level L = lvl(h, j);
  const int64_t n = L.g.n;
  const int ks = j == 0 ? TOBK_KC_FINE_SMOOTH : TOBK_KC_COARSE;
  const int kr = j == 0 ? TOBK_KC_FINE_RESIDUAL : TOBK_KC_COARSE;
  if (j == h->L - 1) {
    prof_begin(h, TOBK_KC_COARSEST, (double)nr * n);
    launch_dense_gemv32(h->Ainv, b, z, n, nr, n, s);
    prof_end(h);
    return z;
  }
  const LevelOpDesc op = level_op(h, j);
  float* dA = L.dA32;
  float* dB = L.dB32;
  if (!z0_ready) {
    prof_begin(h, TOBK_KC_VECTOR, (double)nr * n);
    launch_jacobi0_32(b, L.dinv32, z, SmoothArgs<float>{L.coef32, nullptr, dA}, n, nr, n, s);
    prof_end(h);
  }
  for (int it = 1; it < h->desc.nu_pre; ++it) {
    prof_begin(h, ks, (double)nr * n);
    launch_apply32(op, APPLY_JAC, z, b, L.dinv32, t, SmoothArgs<float>{L.coef32 + 2 * it, dA, dB}, nr, n, s);
    prof_end(h);
    std::swap(z, t);
    std::swap(dA, dB);
  }
  const Level C = lvl(h, j + 1);
  const bool fuse = j + 1 < h->L - 1;
  const bool fused_transfers = op.S32 != nullptr && op.g.dim == 2;
  const bool fused_res = fused_transfers && op.g.nnode * nr < kFusedResidualWork;
  if (fused_res) {
    prof_begin(h, kr, (double)nr * n);
    launch_stencil_res_restrict_2d<float>(op.g, C.g, op.S32, op.fixed, z, b, n, C.fixed, C.b32, C.g.n,
                                          fuse ? C.dinv32 : nullptr, fuse ? C.coef32 : nullptr,
                                          fuse ? C.z32 : nullptr, fuse ? C.dA32 : nullptr, nr, s);
    prof_end(h);
  } else {
    prof_begin(h, kr, (double)nr * n);
    launch_apply32(op, APPLY_RES, z, b, nullptr, L.r32, SmoothArgs<float>{}, nr, n, s);
    prof_end(h);
    prof_begin(h, TOBK_KC_TRANSFER, (double)nr * n);
    if (fuse)
      launch_restrict32(L.g, C.g, C.fixed, L.r32, C.b32, nr, n, C.g.n, s, C.dinv32, C.coef32, C.z32, C.dA32);
    else
      launch_restrict32(L.g, C.g, C.fixed, L.r32, C.b32, nr, n, C.g.n, s);
    prof_end(h);
  }
  float* zc = vcycle32(h, j + 1, nr, C.b32, C.z32, C.t32, fuse);
  int it0 = 0;
  if (fused_transfers && h->desc.nu_post > 0) {
    prof_begin(h, ks, (double)nr * n);
    launch_stencil_jac_prolong_2d<float>(op.g, C.g, op.S32, op.fixed, z, zc, b, L.dinv32, t,
                                         SmoothArgs<float>{L.coef32, nullptr, dB}, nr, n, C.g.n, s);
    prof_end(h);
    std::swap(z, t);
    std::swap(dA, dB);
    it0 = 1;
  } else {
    prof_begin(h, TOBK_KC_TRANSFER, (double)nr * n);
    launch_prolong_add32(L.g, C.g, L.fixed, zc, z, nr, n, C.g.n, s);
    prof_end(h);
  }
  for (int it = it0; it < h->desc.nu_post; ++it) {
    prof_begin(h, ks, (double)nr * n);
    launch_apply32(op, APPLY_JAC, z, b, L.dinv32, t,
                   SmoothArgs<float>{L.coef32 + 2 * it, it == 0 ? nullptr : dA, dB}, nr, n, s);
    prof_end(h);
    std::swap(z, t);
    std::swap(dA, dB);
  }
  return z;
}

// z = M r at level s (FP64 result in one of z / zt)
static double* precondition(tobk_handle* h, int s, int nr, const double* r, double* z, double* zt, int precision,
                           bool z0_ready = false) {
  if (precision == TOBK_FP64) return vcycle64(h, s, nr, r, z, zt, z0_ready);
  const Level L = lvl(h, s);
  const int64_t n = L.g.n;
  launch_f64_to_f32(r, L.b32, (int64_t)nr * n, h->stream);
  float* z32 = vcycle32(h, s, nr, L.b32, L.z32, L.t32);
  launch_f32_to_f64(z32, z, (int64_t)nr * n, h->stream);
  return z;
}

void apply_vcycle(tobk_handle* h, int j, int nr, const double* r, double* out) {
  Level& L = h->lv[j];
  double* z = precondition(h, j, nr, r, L.z, L.t, h->desc.precision);
  cudaMemcpyAsync(out, z, sizeof(double) * nr * L.g.n, cudaMemcpyDeviceToDevice, h->stream);
}

// ================================================================================================
// multi-RHS preconditioned CG
// ================================================================================================
// Two CG iterations (the two direction buffers swap roles twice, so the launch sequence and every
// pointer in it are the same each time): V-cycle, dot products + beta, direction + q = K p + alpha,
// x/r update + convergence test.  The iterate lives in the handle's buffer w.x.
// The FP64 V-cycle's first smoothing step at the CG's level (z = coef dinv r into the V-cycle's z and
// increment buffers), taken by cg_init and cg_update as they write r; none for the FP32 V-cycle or a
// level solved directly.
static CGZ0 cg_z0(tobk_handle* h, int s, int precision) {
  CGZ0 z0;
  if (precision != TOBK_FP64 || s >= h->L - 1) return z0;
  const Level L = lvl(h, s);
  z0.dinv = L.dinv;
  z0.coef = L.coef;
  z0.z = cgw(h, L.g.n).z;
  z0.d = L.dA;
  return z0;
}

static void enqueue_cg_pair(tobk_handle* h, int s, int nr, int precision) {
  cudaStream_t st = h->stream;
  const LevelOpDesc op = level_op(h, s);
  const int64_t n = op.g.n;
  const CGWork w = cgw(h, n);
  const bool flexible = precision != TOBK_FP64;
  const CGZ0 z0 = cg_z0(h, s, precision);
  for (int k = 0; k < 2; ++k) {
    double* p_old = k == 0 ? w.p0 : w.p1;
    double* p_new = k == 0 ? w.p1 : w.p0;
    double* z = precondition(h, s, nr, w.r, w.z, w.zt, precision, z0.z != nullptr);
    prof_begin(h, TOBK_KC_VECTOR, (double)nr * n);
    launch_cg_dots(n, z, w.r, w.q, p_old, flexible, nr, n, w.sc, w.partial, w.counters, st);
    prof_end(h);
    prof_begin(h, s == 0 ? TOBK_KC_FINE_CG_MATVEC : TOBK_KC_COARSE, (double)nr * n);
    launch_cg_direction(op, z, p_old, p_new, w.q, nr, n, w.sc, w.partial, w.counters, st);
    prof_end(h);
    prof_begin(h, TOBK_KC_VECTOR, (double)nr * n);
    launch_cg_update(n, w.x, w.r, p_new, w.q, nr, n, w.sc, w.partial, w.counters, st, z0);
    prof_end(h);
  }
}

// Runs one iteration pair: replayed from a CUDA graph captured on first use for this (level, RHS
// count, precision), or launched directly while profiling or on the legacy default stream.
static int run_cg_pair(tobk_handle* h, int s, int nr, int precision) {
  if (h->prof_on || h->stream == nullptr || !h->use_graphs) {
    enqueue_cg_pair(h, s, nr, precision);
    return TOBK_OK;
  }
  const uint64_t key = (uint64_t)s | ((uint64_t)nr << 8) | ((uint64_t)precision << 16) | ((uint64_t)h->rhs_off << 24);
  auto it = h->cg_graphs.find(key);
  if (it == h->cg_graphs.end()) {
    cudaGraph_t g = nullptr;
    const long long c0 = g_launch_count.load();
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return check_cuda(h, "graph capture");
    enqueue_cg_pair(h, s, nr, precision);
    if (cudaStreamEndCapture(h->stream, &g) != cudaSuccess) return check_cuda(h, "graph capture");
    const long long kernels = g_launch_count.load() - c0;
    g_launch_count.fetch_sub(kernels);
    cudaGraphExec_t ex = nullptr;
    if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      return check_cuda(h, "graph instantiate");
    }
    cudaGraphDestroy(g);
    it = h->cg_graphs.emplace(key, tobk_handle::CGGraph{ex, kernels}).first;
  }
  cudaGraphLaunch(it->second.exec, h->stream);
  g_launch_count.fetch_add(it->second.kernels);
  return TOBK_OK;
}

// Enqueues the work of one half of a split solve: the handle's stream, RHS offset and active-RHS
// pointer are switched to the half's for the lifetime of the scope.
struct HalfScope {
  tobk_handle* h;
  cudaStream_t s0;
  int off0;
  const double* act0;
  HalfScope(tobk_handle* hh, cudaStream_t s, int off) : h(hh), s0(hh->stream), off0(hh->rhs_off), act0(active_rhs()) {
    h->stream = s;
    h->rhs_off = off;
    set_active_rhs(h->cg.sc + (size_t)off * kScStride);
  }
  ~HalfScope() {
    h->stream = s0;
    h->rhs_off = off0;
    set_active_rhs(act0);
  }
};

// One CG iteration pair for every still-active half of the solve: the first n0 right-hand sides on
// the handle's stream, the rest (when split) on stream2, forked after the work already enqueued.
static int run_cg_pair_halves(tobk_handle* h, int s, int nr, int n0, int precision, const bool (&active)[2]) {
  if (n0 >= nr) return run_cg_pair(h, s, nr, precision);
  cudaEventRecord(h->ev_fork, h->stream);
  cudaStreamWaitEvent(h->stream2, h->ev_fork, 0);
  int rc = TOBK_OK;
  if (active[0]) rc = run_cg_pair(h, s, n0, precision);
  if (rc == TOBK_OK && active[1]) {
    HalfScope hs(h, h->stream2, n0);
    rc = run_cg_pair(h, s, nr - n0, precision);
  }
  cudaEventRecord(h->ev_join, h->stream2);
  cudaStreamWaitEvent(h->stream, h->ev_join, 0);
  return rc;
}

void cg_async_begin(tobk_handle* h, cudaStream_t st, int off, int s, const double* B, const double* X0, int nr,
                    double rtol, int precision) {
  HalfScope hs(h, st, off);
  const LevelOpDesc op = level_op(h, s);
  const int64_t n = op.g.n;
  const CGWork w = cgw(h, n);
  cudaMemcpyAsync(w.x, X0, sizeof(double) * nr * n, cudaMemcpyDeviceToDevice, st);
  launch_cg_init(op, B, w.x, w.r, true, rtol, nr, n, w.sc, w.partial, w.counters, st, cg_z0(h, s, precision));
  cudaMemsetAsync(w.p0, 0, sizeof(double) * nr * n, st);
  cudaMemsetAsync(w.q, 0, sizeof(double) * nr * n, st);
}

int cg_async_pairs(tobk_handle* h, cudaStream_t st, int off, int s, int nr, int pairs, int precision) {
  HalfScope hs(h, st, off);
  for (int k = 0; k < pairs; ++k) {
    const int rc = run_cg_pair(h, s, nr, precision);
    if (rc) return rc;
  }
  return TOBK_OK;
}

void cg_async_end(tobk_handle* h, cudaStream_t st, int off, int s, double* X, int nr) {
  HalfScope hs(h, st, off);
  const int64_t n = h->lv[s].g.n;
  const CGWork w = cgw(h, n);
  cudaMemcpyAsync(X, w.x, sizeof(double) * nr * n, cudaMemcpyDeviceToDevice, st);
}

int pcg_solve(tobk_handle* h, int s, const double* B, double* X, int nr, double rtol, int max_iter, bool use_x0,
              int precision, tobk_solve_info* info, bool fixed_iters) {
  if (nr < 1 || nr > h->rmax) return fail(h, TOBK_E_ARG, "bad RHS count");
  if (!h->setup_done) {
    int rc = setup_hierarchy(h);
    if (rc) return rc;
  }
  cudaStream_t st = h->stream;
  const LevelOpDesc op = level_op(h, s);
  const int64_t n = op.g.n;
  CGWork& w = h->cg;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  ActiveRhsScope active_scope(w.sc);
  if (use_x0) cudaMemcpyAsync(w.x, X, sizeof(double) * nr * n, cudaMemcpyDeviceToDevice, st);
  int pairs = 0;
  int rc = TOBK_OK;
  double worst = 0.0;
  int iters = 0;
  bool all_conv = true;
  // independent CG recurrences: with two or more right-hand sides on a stream of the caller's, the
  // second half of them runs concurrently on stream2 (graph-replayed pairs only)
  const bool split = nr >= 2 && h->stream != nullptr && h->stream2 != nullptr && h->use_graphs && !h->prof_on;
  const int n0 = split ? (nr + 1) / 2 : nr;
  bool half_active[2] = {true, true};
  if (fixed_iters) {
    // a fixed number of iterations as an approximate inverse (a preconditioner): no host
    // synchronisation, no exit check; breakdown shows in the caller's own residuals
    launch_cg_init(op, B, w.x, w.r, use_x0, rtol, nr, n, w.sc, w.partial, w.counters, st, cg_z0(h, s, precision));
    cudaMemsetAsync(w.p0, 0, sizeof(double) * nr * n, st);
    cudaMemsetAsync(w.q, 0, sizeof(double) * nr * n, st);
    while (2 * pairs < max_iter) {
      rc = run_cg_pair_halves(h, s, nr, n0, precision, half_active);
      if (rc) break;
      ++pairs;
    }
    cudaMemcpyAsync(X, w.x, sizeof(double) * nr * n, cudaMemcpyDeviceToDevice, st);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (info) {
      *info = tobk_solve_info{};
      info->iterations = 2 * pairs;
      info->num_rhs = nr;
      info->status_detail = 2 * pairs;
    }
    return rc ? rc : check_cuda(h, "pcg_solve");
  }
  for (int attempt = 0; attempt < 4; ++attempt) {
    launch_cg_init(op, B, w.x, w.r, use_x0 || attempt > 0, rtol, nr, n, w.sc, w.partial, w.counters, st,
                   cg_z0(h, s, precision));
    cudaMemsetAsync(w.p0, 0, sizeof(double) * nr * n, st);
    cudaMemsetAsync(w.q, 0, sizeof(double) * nr * n, st);
    half_active[0] = half_active[1] = true;
    while (2 * pairs < max_iter) {
      rc = run_cg_pair_halves(h, s, nr, n0, precision, half_active);
      if (rc) break;
      ++pairs;
      cudaMemcpyAsync(w.host_sc, w.sc, sizeof(double) * nr * kScStride, cudaMemcpyDeviceToHost, st);
      cudaStreamSynchronize(st);
      half_active[0] = half_active[1] = false;
      for (int r = 0; r < nr; ++r) half_active[r < n0 ? 0 : 1] |= w.host_sc[r * kScStride + SC_ACTIVE] != 0.0;
      if (!half_active[0] && !half_active[1]) break;
    }
    if (rc) break;
    int status = 0;
    for (int r = 0; r < nr; ++r) {
      status = std::max(status, (int)w.host_sc[r * kScStride + SC_STATUS]);
      iters = std::max(iters, (int)w.host_sc[r * kScStride + SC_ITERS]);
    }
    // true residual recomputed at exit
    launch_true_residual(op, B, w.x, w.zt, nr, n, w.sc, w.partial, w.counters, st);
    cudaMemcpyAsync(w.host_sc, w.sc, sizeof(double) * nr * kScStride, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    rc = check_cuda(h, "pcg_solve");
    if (rc) break;
    worst = 0.0;
    all_conv = true;
    for (int r = 0; r < nr; ++r) {
      const double rel = w.host_sc[r * kScStride + SC_RELRES];
      worst = std::max(worst, std::isfinite(rel) ? rel : INFINITY);
      if (!(rel <= rtol)) all_conv = false;
    }
    if (status == 1) {
      rc = fail(h, TOBK_E_BREAKDOWN, "CG breakdown: p^T K p <= 0");
      break;
    }
    if (status == 2 || !std::isfinite(worst)) {
      rc = fail(h, TOBK_E_NONFINITE, "non-finite value in CG");
      break;
    }
    if (all_conv || 2 * pairs >= max_iter) break;
    // the recursive residual met the target but the true one did not: restart from the iterate
  }
  cudaMemcpyAsync(X, w.x, sizeof(double) * nr * n, cudaMemcpyDeviceToDevice, st);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->iterations = iters;
    info->converged = all_conv ? 1 : 0;
    info->num_rhs = nr;
    info->rel_residual = worst;
    info->time_ms = ms;
    info->status_detail = 2 * pairs;
  }
  if (rc == TOBK_OK && !all_conv) rc = fail(h, TOBK_E_NOT_CONVERGED, "CG iteration limit reached");
  return rc;
}

void apply_K_level(tobk_handle* h, int j, const double* v, double* y, int nr, int64_t stride) {
  launch_apply(level_op(h, j), APPLY_KV, v, nullptr, nullptr, y, SmoothArgs<double>{}, nr, stride, h->stream);
}

void apply_G_level(tobk_handle* h, int j, const double* v, double* y, int nr, int64_t stride) {
  if (j == 0 && h->Gc0) {
    launch_inc_apply_g(h->lv[0].g, h->lv[0].fixed, h->Gc0, h->Es, v, y, nr, stride, h->stream);
  } else if (j == 0) {
    launch_apply_kron(h->lv[0].g, h->lv[0].fixed, h->Gs, v, y, nr, stride, h->stream);
  } else {
    LevelOpDesc d{};
    d.g = h->lv[j].g;
    d.fixed = h->lv[j].fixed;
    d.stored = true;
    d.Ke64 = h->lv[j].Ge;
    launch_apply(d, APPLY_KV, v, nullptr, nullptr, y, SmoothArgs<double>{}, nr, stride, h->stream);
  }
}

// ================================================================================================
// linear analysis and stress stiffness
// ================================================================================================
int setup_stress(tobk_handle* h) {
  cudaStream_t s = h->stream;
  const Grid& g = h->lv[0].g;
  if (h->Gc0)
    launch_inc_stress(g, h->u, h->d_A, h->d_dN, h->d_D, h->tab.wdet, h->Gfull, h->Gc0, s);
  else
    launch_stress_gs_dev(g, h->u, h->Es, h->d_dN, h->d_D, h->tab.wdet, h->Gs0, h->Gs, s);
  for (int j = 1; j <= h->eig; ++j) {
    Level& Lc = h->lv[j];
    const Level& Lf = h->lv[j - 1];
    if (j == 1 && h->Gc0)
      launch_galerkin_scaled_stored(Lf.g, Lc.g, Lf.fixed, h->Gc0, h->Es, h->d_W, Lc.Ge, s);
    else if (j == 1)
      launch_galerkin_fine_G(Lf.g, Lc.g, Lf.fixed, h->Gs, h->d_W, Lc.Ge, s);
    else
      launch_galerkin_stored(Lf.g, Lc.g, Lf.fixed, Lf.Ge, h->d_W, Lc.Ge, s);
  }
  int rc = check_cuda(h, "setup_stress");
  if (rc) return rc;
  h->have_G = true;
  return TOBK_OK;
}

// u <- (d[0] / d[1]) u with d = (u^T f, u^T K u): the multiple of an initial guess closest to the
// solution in the energy norm (never farther than the zero guess); zero if u^T K u is not positive
__global__ void k_energy_scale(double* u, int64_t n, const double* d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double den = d[1];
  u[i] *= (den > 0.0 && isfinite(d[0] / den)) ? d[0] / den : 0.0;
}

int solve_equilibrium(tobk_handle* h, double* compliance, tobk_solve_info* info) {
  if (!h->have_x || !h->have_f || !h->have_fixed) return fail(h, TOBK_E_STATE, "densities, load and fixed DOFs must be set");
  if (!h->setup_done) {
    int rc = setup_hierarchy(h);
    if (rc) return rc;
  }
  cudaStream_t s = h->stream;
  const int64_t n = h->lv[0].g.n;
  launch_mask_copy(h->f, h->lv[0].fixed, h->bwork, n, 1, n, s);
  if (h->have_u0) {
    // the caller's guess (e.g. the learned warm start), scaled to minimise its energy-norm error
    cudaMemcpyAsync(h->u, h->u0, sizeof(double) * n, cudaMemcpyDeviceToDevice, s);
    apply_K_level(h, 0, h->u, h->xwork, 1, n);
    launch_gram(h->bwork, 1, h->u, 1, n, n, h->dscal + 960, h->gram_partial, s);
    launch_gram(h->u, 1, h->xwork, 1, n, n, h->dscal + 961, h->gram_partial, s);
    ::tobk::note_launch(), k_energy_scale<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(h->u, n, h->dscal + 960);
  }
  tobk_solve_info li{};
  int rc = pcg_solve(h, 0, h->bwork, h->u, 1, h->desc.rtol, h->desc.max_iter, h->have_u0, h->desc.precision,
                     info ? info : &li);
  if (rc && rc != TOBK_E_NOT_CONVERGED) return rc;
  h->la_iters = (info ? info : &li)->iterations;
  launch_gram(h->bwork, 1, h->u, 1, n, n, h->dscal, h->gram_partial, s);
  cudaMemcpyAsync(h->hscal, h->dscal, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  h->compliance = h->hscal[0];
  if (compliance) *compliance = h->compliance;
  int rc2 = setup_stress(h);
  if (rc2) return rc2;
  h->have_u = true;
  h->have_modes = h->have_sens = false;
  return rc;
}

}  // namespace tobk
