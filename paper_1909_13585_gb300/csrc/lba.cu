// Linearized buckling analysis and sensitivities on the GPU.
//
//   exact LBA (eig_level 1) ........ Algorithm 1: eigenpairs of (K + lambda G) phi = 0 on Omega_1
//   multilevel LBA (eig_level l) .... Sec. 2.1 steps 1-4 / Algorithm 2 lines 5-18 without the
//                                     optional per-level smoothing: coarse Galerkin eigenpairs,
//                                     Psi^j = I^j_{j+1} Psi^{j+1}, fine solve K Phi = G Psi,
//                                     Rayleigh quotients (eq. FineScaleRQ)
//   adjoint right-hand sides ........ phi^T (grad_u G) phi (eq. AdjointSystem)
//   sensitivities ................... eq. SensitivityLambda with the factor -1/(phi^T G phi)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "device_common.cuh"
#include "handle.h"

namespace tobk {

void launch_coldots(const double* A, const double* B, int ncols, int64_t n, int64_t stride, double* out,
                    double* partial, cudaStream_t s);

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// ------------------------------------------------------------------------------------------------
// mode post-processing: scale to phi^T K phi = 1, sign (largest-magnitude entry positive), order
// ------------------------------------------------------------------------------------------------
// per column: index of the entry of largest magnitude (smallest index on ties), two stages
__global__ void k_argmax_partial(const double* A, int64_t n, int64_t stride, double* pv, long long* pi) {
  __shared__ double sv[256];
  __shared__ long long si[256];
  const int col = blockIdx.y;
  double best = -1.0;
  long long bi = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double v = fabs(A[(int64_t)col * stride + k]);
    if (v > best) {
      best = v;
      bi = k;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double a = sv[threadIdx.x], b = sv[threadIdx.x + o];
      const long long ia = si[threadIdx.x], ib = si[threadIdx.x + o];
      if (b > a || (b == a && ib < ia)) {
        sv[threadIdx.x] = b;
        si[threadIdx.x] = ib;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[(size_t)col * gridDim.x + blockIdx.x] = sv[0];
    pi[(size_t)col * gridDim.x + blockIdx.x] = si[0];
  }
}

// One thread: per column the sign entry, the scale 1/sqrt(num) and the ascending order of lambda.
// lam_in[i] = lambda of column i; num[i] = phi_i^T K phi_i.  Outputs: perm[r] = source column of
// rank r, scale[r], lam_out[r].
__global__ void k_order_modes(const double* A, int64_t stride, const double* pv, const long long* pi, int chunks,
                              const double* lam_in, const double* num, int q, int* perm, double* scale,
                              double* lam_out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int order[64];
  for (int i = 0; i < q; ++i) order[i] = i;
  for (int i = 1; i < q; ++i) {  // insertion sort, stable
    const int c = order[i];
    int k = i - 1;
    while (k >= 0 && lam_in[order[k]] > lam_in[c]) {
      order[k + 1] = order[k];
      --k;
    }
    order[k + 1] = c;
  }
  for (int r = 0; r < q; ++r) {
    const int c = order[r];
    double best = -1.0;
    long long bi = 0;
    for (int b = 0; b < chunks; ++b) {
      const double v = pv[(size_t)c * chunks + b];
      const long long ii = pi[(size_t)c * chunks + b];
      if (v > best || (v == best && ii < bi)) {
        best = v;
        bi = ii;
      }
    }
    const double sg = A[(int64_t)c * stride + bi] < 0.0 ? -1.0 : 1.0;
    perm[r] = c;
    scale[r] = sg / sqrt(num[c]);
    lam_out[r] = lam_in[c];
  }
}

__global__ void k_permute_scale(const double* A, const int* perm, const double* scale, double* B, int64_t n,
                                int64_t stride) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int r = blockIdx.y;
  B[(int64_t)r * stride + k] = scale[r] * A[(int64_t)perm[r] * stride + k];
}

// X[r] = s[r] A[r] for the q columns of length n.
__global__ void k_scale_cols(const double* A, const double* s, double* X, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int r = blockIdx.y;
  X[(int64_t)r * n + k] = s[r] * A[(int64_t)r * n + k];
}

__global__ void k_rq(const double* num, const double* den, int q, double* lam) {
  const int i = threadIdx.x;
  if (i < q) lam[i] = -num[i] / den[i];
}

// Normalises the q columns of A (length n) into `out` (may alias neither): K scaling, sign, order.
static void finalize_modes(tobk_handle* h, const double* A, const double* lam_dev, const double* num_dev, double* out,
                           double* lam_out_dev) {
  cudaStream_t st = h->stream;
  const int64_t n = h->lv[0].g.n;
  const int q = h->q;
  const int chunks = 64;
  double* pv = h->gram_partial;
  long long* pi = (long long*)(h->gram_partial + (size_t)q * chunks);
  ::tobk::note_launch(), k_argmax_partial<<<dim3(chunks, q), 256, 0, st>>>(A, n, n, pv, pi);
  int* perm = (int*)(h->dscal + 640);
  double* scale = h->dscal + 704;
  ::tobk::note_launch(), k_order_modes<<<1, 32, 0, st>>>(A, n, pv, pi, chunks, lam_dev, num_dev, q, perm, scale, lam_out_dev);
  ::tobk::note_launch(), k_permute_scale<<<dim3(nblk(n), q), 256, 0, st>>>(A, perm, scale, out, n, n);
}

// Early fine solve (Sec. 2.1 step 3 for part of the modes).  The coarse pairs converge one after the
// other; whenever a few more of them meet eig_tol, their fine systems K phi = G P psi are started as a
// group on a stream of its own (and its own RHS columns q + c0 .. of the work buffers) while the
// eigensolver iterates on the rest, so that the FP64-bound fine solves fill the SMs the latency-bound
// eigensolver leaves idle.  The snapshot of a converged pair is as good an eigenpair as its final
// iterate (both meet eig_tol).  Iteration pairs are enqueued without host synchronisation, one per
// group and further outer iteration; compute_buckling finishes the solves to rtol.
struct EarlyFine : EigenHook {
  struct Group {
    int c0 = 0, pairs = 0;
    cudaStream_t st = nullptr;
    bool failed = false;
    std::vector<int> S;        // coarse indices
    std::vector<double> lam;   // their load factors at the snapshot
  };
  tobk_handle* h;
  int l, gnew, used = 0;
  std::vector<Group> groups;
  std::vector<char> taken;
  double scale_h[64];
  EarlyFine(tobk_handle* hh, int level, int q) : h(hh), l(level), gnew(std::max(2, q / 4)), taken(q, 0) {}
  void iteration(const double* X, int64_t nl, const double* theta, const bool* conv, int q) override {
    for (Group& G : groups) {
      if (G.failed) continue;
      if (cg_async_pairs(h, G.st, q + G.c0, 0, (int)G.S.size(), 1, h->desc.precision)) G.failed = true;
      ++G.pairs;
    }
    std::vector<int> idx;
    for (int i = 0; i < q; ++i)
      if (conv[i] && !taken[i]) idx.push_back(i);
    const int room = h->early_gmax - used;
    if ((int)idx.size() < gnew || room < gnew) return;
    if ((int)idx.size() > room) idx.resize(room);
    Group G;
    G.c0 = used;
    G.S = idx;
    G.st = h->stream3[groups.size() % tobk_handle::kEarlyStreams];
    cudaStream_t s3 = G.st;
    const int g = (int)idx.size();
    const int64_t n = h->lv[0].g.n;
    for (int k = 0; k < g; ++k) {
      taken[idx[k]] = 1;
      cudaMemcpyAsync(h->ea_psi + (size_t)(G.c0 + k) * nl, X + (size_t)idx[k] * nl, sizeof(double) * nl,
                      cudaMemcpyDeviceToDevice, h->stream);
      G.lam.push_back(1.0 / theta[idx[k]]);
      scale_h[k] = -theta[idx[k]];  // Phi_0 = -Psi / lambda
    }
    used += g;
    cudaEventRecord(h->ev_snap, h->stream);
    cudaStreamWaitEvent(s3, h->ev_snap, 0);
    // Psi = P psi through the group's columns of the finer levels' b buffers
    const double* src = h->ea_psi + (size_t)G.c0 * nl;
    double* Psi = h->ea_Psi + (size_t)G.c0 * n;
    double* rhs = h->ea_rhs + (size_t)G.c0 * n;
    double* Phi = h->ea_Phi + (size_t)G.c0 * n;
    for (int j = l; j >= 1; --j) {
      Level& C = h->lv[j];
      Level& F = h->lv[j - 1];
      double* dst = j == 1 ? Psi : F.b + (size_t)(q + G.c0) * F.g.n;
      cudaMemsetAsync(dst, 0, sizeof(double) * g * F.g.n, s3);
      launch_prolong_add(F.g, C.g, F.fixed, src, dst, g, F.g.n, C.g.n, s3);
      src = dst;
    }
    {
      cudaStream_t s0 = h->stream;
      h->stream = s3;
      apply_G_level(h, 0, Psi, rhs, g, n);
      h->stream = s0;
    }
    cudaMemcpyAsync(h->ea_scale + G.c0, scale_h, sizeof(double) * g, cudaMemcpyHostToDevice, s3);
    ::tobk::note_launch(), k_scale_cols<<<dim3(nblk(n), g), 256, 0, s3>>>(Psi, h->ea_scale + G.c0, Phi, n);
    cg_async_begin(h, s3, q + G.c0, 0, rhs, Phi, g, h->desc.rtol, h->desc.precision);
    if (cg_async_pairs(h, s3, q + G.c0, 0, g, 2, h->desc.precision)) G.failed = true;
    G.pairs = 2;
    groups.push_back(G);
  }
};

int compute_buckling(tobk_handle* h, double* lambda, tobk_solve_info* info) {
  if (!h->have_u || !h->have_G) return fail(h, TOBK_E_STATE, "solve_equilibrium must come first");
  cudaStream_t st = h->stream;
  const int q = h->q;
  const int64_t n = h->lv[0].g.n;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  tobk_solve_info ei{};
  double lam_h[64];
  int rc = TOBK_OK;
  PhaseMarks pm(h);
  const int m_begin = pm.mark();
  int m_eig = -1, m_prolong = -1, m_solve = -1;
  double* num = h->dscal + 768;   // [q]
  double* den = h->dscal + 832;   // [q]
  double* lraw = h->dscal + 896;  // [q]
  if (h->eig == 0) {
    // Algorithm 1 EA on the fine grid
    double* Phi = h->lv[0].b;     // [q][n] scratch
    rc = eigen_solve(h, 0, q, Phi, lam_h, &ei);
    if (rc && rc != TOBK_E_NOT_CONVERGED) return rc;
    m_eig = m_prolong = m_solve = pm.mark();
    double* KP = h->xwork;
    apply_K_level(h, 0, Phi, KP, q, n);
    launch_coldots(Phi, KP, q, n, n, num, h->gram_partial, st);
    cudaMemcpyAsync(lraw, lam_h, sizeof(double) * q, cudaMemcpyHostToDevice, st);
    finalize_modes(h, Phi, lraw, num, h->modes, h->lam);
  } else {
    // Sec. 2.1 step 1: coarse eigenpairs on Omega_l of the Galerkin pencil
    const int l = h->eig;
    double* Psi = h->lv[l].b;
    const bool plain_steps =
        h->desc.kaczmarz_sweeps == 0 && !h->desc.ritz_levels && std::max(1, h->desc.fine_steps) == 1;
    const bool use_early = h->early_gmax > 0 && h->stream3[0] != nullptr && st != nullptr && h->use_graphs &&
                           !h->prof_on && plain_steps;
    EarlyFine early(h, l, q);
    if (use_early) {
      // the eigensolve on the handle's highest-priority stream pair, forked from and joined back to the
      // caller's stream, so that its short kernels are scheduled ahead of the early fine solve's
      cudaEventRecord(h->ev_hi, st);
      cudaStreamWaitEvent(h->stream_hi, h->ev_hi, 0);
      h->stream = h->stream_hi;
      std::swap(h->stream2, h->stream_hi2);
      rc = eigen_solve(h, l, q, Psi, lam_h, &ei, &early);
      std::swap(h->stream2, h->stream_hi2);
      h->stream = st;
      cudaEventRecord(h->ev_hi, h->stream_hi);
      cudaStreamWaitEvent(st, h->ev_hi, 0);
    } else {
      rc = eigen_solve(h, l, q, Psi, lam_h, &ei, nullptr);
    }
    std::vector<int> S;  // coarse modes whose fine solve ran early (kept if they are still the same pairs),
                         // their iterates compacted to columns 0 .. |S| - 1 of ea_rhs / ea_Phi
    std::vector<int> Scol;  // the early column of each kept mode before compaction
    if (!early.groups.empty()) {
      const int64_t n0 = h->lv[0].g.n, nl = h->lv[l].g.n;
      // pairs up to the linear analysis' iteration count of this design (the fine systems share its
      // operator); the finishing solve below takes any that remain
      const int want = h->la_iters > 0 ? (h->la_iters + 1) / 2 : 16;
      for (auto& G : early.groups) {
        const int g = (int)G.S.size();
        if (!G.failed && want > G.pairs &&
            cg_async_pairs(h, G.st, q + G.c0, 0, g, want - G.pairs, h->desc.precision))
          G.failed = true;
        cg_async_end(h, G.st, q + G.c0, 0, h->ea_Phi + (size_t)G.c0 * n0, g);
      }
      for (int k = 0; k < tobk_handle::kEarlyStreams; ++k) cudaEventRecord(h->ev_early[k], h->stream3[k]);
      for (auto& G : early.groups) {
        bool same = rc == TOBK_OK && !G.failed;
        for (size_t k = 0; k < G.S.size() && same; ++k) {
          const double a = lam_h[G.S[k]], b = G.lam[k];
          same = std::fabs(a - b) <= 1e-9 * std::fabs(b);
        }
        if (!same) continue;
        for (size_t k = 0; k < G.S.size(); ++k) {  // the pairs the early solve started from
          const int i = G.S[k];
          cudaMemcpyAsync(Psi + (size_t)i * nl, h->ea_psi + (size_t)(G.c0 + k) * nl, sizeof(double) * nl,
                          cudaMemcpyDeviceToDevice, st);
          lam_h[i] = G.lam[k];
          S.push_back(i);
          Scol.push_back(G.c0 + (int)k);
        }
      }
      if (S.empty())  // the early solves' buffers are free again after this point
        for (int k = 0; k < tobk_handle::kEarlyStreams; ++k) cudaStreamWaitEvent(st, h->ev_early[k], 0);
    }
    if (rc && rc != TOBK_E_NOT_CONVERGED) return rc;
    m_eig = pm.mark();
    if (h->cs_psi) {  // the coarse pairs, for the consistent sensitivities
      cudaMemcpyAsync(h->cs_psi, Psi, sizeof(double) * q * h->lv[l].g.n, cudaMemcpyDeviceToDevice, st);
      for (int i = 0; i < q; ++i) h->cs_mu[i] = lam_h[i];
    }
    // step 2: Psi^j = I^j_{j+1} Psi^{j+1}, and on each finer level the optional steps of
    // Algorithm 2: Kaczmarz smoothing on K^j + sigma G^j (sigma the smallest load factor known from
    // the level above) and the Rayleigh-Ritz projection of (K^j, G^j) on span Psi^j
    const int sweeps = h->desc.kaczmarz_sweeps;
    const bool ritz = h->desc.ritz_levels != 0;
    double shift = lam_h[0];
    for (int i = 1; i < q; ++i) shift = std::min(shift, lam_h[i]);
    for (int j = l; j >= 1; --j) {
      Level& C = h->lv[j];
      Level& F = h->lv[j - 1];
      cudaMemsetAsync(F.b, 0, sizeof(double) * q * F.g.n, st);
      launch_prolong_add(F.g, C.g, F.fixed, C.b, F.b, q, F.g.n, C.g.n, st);
      if (sweeps > 0) {
        if (j - 1 == 0 && h->Gc0)
          launch_pencil_stencil(F.g, F.fixed, h->Ek, h->d_Ke0, nullptr, nullptr, h->Gc0, h->Es, shift, h->kz_S,
                                h->kz_rn2, st);
        else if (j - 1 == 0)
          launch_pencil_stencil(F.g, F.fixed, h->Ek, h->d_Ke0, nullptr, h->Gs, nullptr, nullptr, shift, h->kz_S,
                                h->kz_rn2, st);
        else
          launch_pencil_stencil(F.g, F.fixed, nullptr, nullptr, F.Ke, nullptr, F.Ge, nullptr, shift, h->kz_S,
                                h->kz_rn2, st);
        launch_kaczmarz_sweeps(F.g, F.fixed, h->kz_S, h->kz_rn2, F.b, q, F.g.n, sweeps, st);
      }
      if (ritz) {
        const int rrc = ritz_level(h, j - 1, q, F.b, lam_h);
        if (rrc) return rrc;
        shift = lam_h[0];
      }
    }
    // steps 3-4, repeated fine_steps times (inverse iteration on Omega_1): K Phi = G Psi by one
    // multi-RHS mgPCG solve, then the Rayleigh quotients lambda_i = -phi^T K phi / phi^T G phi.
    // Initial guess Phi_0 = -Psi / lambda: for the first step (K + lambda_c G) Psi is the fine
    // residual of the prolongated coarse pair, and with Galerkin coarse operators its restriction
    // to Omega_l is the coarse eigen residual (1e-8), so the starting error has no component the
    // coarse space represents.
    const int steps = std::max(1, h->desc.fine_steps);
    const double* src = h->lv[0].b;
    double* rhs = h->bwork;
    double* Phi = h->xwork;
    if (!S.empty()) {
      // the modes not solved early (compact in xwork / bwork), beside the early solve's last pairs
      std::vector<int> B;
      for (int i = 0; i < q; ++i)
        if (std::find(S.begin(), S.end(), i) == S.end()) B.push_back(i);
      const int nbq = (int)B.size(), g = (int)S.size();
      double s_h[64];
      for (int k = 0; k < nbq; ++k) {
        cudaMemcpyAsync(h->xwork + (size_t)k * n, src + (size_t)B[k] * n, sizeof(double) * n,
                        cudaMemcpyDeviceToDevice, st);
        const double lb = lam_h[B[k]];
        s_h[k] = (lb > 0.0 && std::isfinite(lb)) ? -1.0 / lb : 0.0;
      }
      apply_G_level(h, 0, h->xwork, h->bwork, nbq, n);
      cudaMemcpyAsync(den, s_h, sizeof(double) * nbq, cudaMemcpyHostToDevice, st);
      ::tobk::note_launch(), k_scale_cols<<<dim3(nblk(n), nbq), 256, 0, st>>>(h->xwork, den, h->xwork, n);
      m_prolong = pm.mark();
      tobk_solve_info sb{}, sa{};
      int brc = pcg_solve(h, 0, h->bwork, h->xwork, nbq, h->desc.rtol, h->desc.max_iter, true, h->desc.precision, &sb);
      if (brc && brc != TOBK_E_NOT_CONVERGED) return brc;
      // the early modes: their iterates (compacted, in the order of S), finished to rtol on the handle's stream
      for (int k = 0; k < tobk_handle::kEarlyStreams; ++k) cudaStreamWaitEvent(st, h->ev_early[k], 0);
      int early_pairs = 0;
      for (auto& G : early.groups) early_pairs = std::max(early_pairs, G.pairs);
      for (int k = 0; k < g; ++k)
        if (Scol[k] != k) {  // Scol is increasing, so a column is moved only down onto a free one
          cudaMemcpyAsync(h->ea_rhs + (size_t)k * n, h->ea_rhs + (size_t)Scol[k] * n, sizeof(double) * n,
                          cudaMemcpyDeviceToDevice, st);
          cudaMemcpyAsync(h->ea_Phi + (size_t)k * n, h->ea_Phi + (size_t)Scol[k] * n, sizeof(double) * n,
                          cudaMemcpyDeviceToDevice, st);
        }
      int arc = pcg_solve(h, 0, h->ea_rhs, h->ea_Phi, g, h->desc.rtol, h->desc.max_iter, true, h->desc.precision, &sa);
      if (arc && arc != TOBK_E_NOT_CONVERGED) return arc;
      ei.iterations += std::max(sb.iterations, 2 * early_pairs + sa.iterations);
      m_solve = pm.mark();
      // Phi in the coarse modes' order
      Phi = h->bwork;
      for (int k = 0; k < g; ++k)
        cudaMemcpyAsync(Phi + (size_t)S[k] * n, h->ea_Phi + (size_t)k * n, sizeof(double) * n,
                        cudaMemcpyDeviceToDevice, st);
      for (int k = 0; k < nbq; ++k)
        cudaMemcpyAsync(Phi + (size_t)B[k] * n, h->xwork + (size_t)k * n, sizeof(double) * n,
                        cudaMemcpyDeviceToDevice, st);
      double* KP = h->lv[0].z;
      double* GP = h->lv[0].t;
      apply_K_level(h, 0, Phi, KP, q, n);
      apply_G_level(h, 0, Phi, GP, q, n);
      launch_coldots(Phi, KP, q, n, n, num, h->gram_partial, st);
      launch_coldots(Phi, GP, q, n, n, den, h->gram_partial, st);
      ::tobk::note_launch(), k_rq<<<1, 64, 0, st>>>(num, den, q, lraw);
      finalize_modes(h, Phi, lraw, num, h->modes, h->lam);
    }
    for (int stp = 0; stp < (S.empty() ? steps : 0); ++stp) {
      if (stp > 0) {  // the previous step's normalised modes and load factors
        src = h->modes;
        cudaMemcpyAsync(h->hscal, h->lam, sizeof(double) * q, cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        for (int i = 0; i < q; ++i) lam_h[i] = h->hscal[i];
      }
      apply_G_level(h, 0, src, rhs, q, n);
      double s_h[64];
      for (int i = 0; i < q; ++i) s_h[i] = (lam_h[i] > 0.0 && std::isfinite(lam_h[i])) ? -1.0 / lam_h[i] : 0.0;
      cudaMemcpyAsync(den, s_h, sizeof(double) * q, cudaMemcpyHostToDevice, st);
      ::tobk::note_launch(), k_scale_cols<<<dim3(nblk(n), q), 256, 0, st>>>(src, den, Phi, n);
      if (stp == 0) m_prolong = pm.mark();
      tobk_solve_info si{};
      int src_rc = pcg_solve(h, 0, rhs, Phi, q, h->desc.rtol, h->desc.max_iter, true, h->desc.precision, &si);
      if (src_rc && src_rc != TOBK_E_NOT_CONVERGED) return src_rc;
      ei.iterations += si.iterations;
      if (stp == steps - 1) m_solve = pm.mark();
      double* KP = h->lv[0].z;
      double* GP = h->lv[0].t;
      apply_K_level(h, 0, Phi, KP, q, n);
      apply_G_level(h, 0, Phi, GP, q, n);
      launch_coldots(Phi, KP, q, n, n, num, h->gram_partial, st);
      launch_coldots(Phi, GP, q, n, n, den, h->gram_partial, st);
      ::tobk::note_launch(), k_rq<<<1, 64, 0, st>>>(num, den, q, lraw);
      finalize_modes(h, Phi, lraw, num, h->modes, h->lam);
    }
  }
  cudaMemcpyAsync(h->hscal, h->lam, sizeof(double) * q, cudaMemcpyDeviceToHost, st);
  const bool record_cs = h->cs_psi && h->eig > 0;
  if (record_cs) {  // fine mode r = scale[r] x the solution from coarse mode perm[r] (finalize_modes)
    cudaMemcpyAsync(h->hscal + 64, h->dscal + 640, sizeof(int) * q, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(h->hscal + 128, h->dscal + 704, sizeof(double) * q, cudaMemcpyDeviceToHost, st);
  }
  const int m_end = pm.mark();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  int crc = check_cuda(h, "compute_buckling");
  if (crc) return crc;
  if (h->phase_on) {
    h->phase_ms[TOBK_PHASE_EIGEN] = pm.ms(m_begin, m_eig);
    h->phase_ms[TOBK_PHASE_PROLONG] = pm.ms(m_eig, m_prolong);
    h->phase_ms[TOBK_PHASE_FINE_SOLVE] = pm.ms(m_prolong, m_solve);
    h->phase_ms[TOBK_PHASE_RQ] = pm.ms(m_solve, m_end);
  }
  for (int i = 0; i < q; ++i) h->lam_host[i] = h->hscal[i];
  h->cs_ready = record_cs;
  if (record_cs) {
    const int* perm = (const int*)(h->hscal + 64);
    for (int i = 0; i < q; ++i) {
      h->cs_perm[i] = perm[i];
      h->cs_scale[i] = h->hscal[128 + i];
    }
  }
  if (lambda)
    for (int i = 0; i < q; ++i) lambda[i] = h->lam_host[i];
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    *info = ei;
    info->time_ms = ms;
  }
  h->have_modes = true;
  h->have_sens = false;
  h->have_cs = false;
  return rc;
}

// ------------------------------------------------------------------------------------------------
// adjoint right-hand side  b = phi^T (grad_u G) phi
//   element part: sum_gp w|J| B^T D h(phi_e),  h = Voigt(sum_c d_a phi_c d_b phi_c), shear doubled
// ------------------------------------------------------------------------------------------------
template <int DIM>
__global__ void k_adjoint_gp(Grid g, const double* __restrict__ phi, const double* __restrict__ Es,
                             const double* __restrict__ dN, const double* __restrict__ D, double wdet,
                             double* __restrict__ sgp) {
  constexpr int NN = Dims<DIM>::NN, NV = Dims<DIM>::NV;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.m) return;
  const int ei = (int)(e % g.nel[0]);
  const int64_t rest = e / g.nel[0];
  const int ej = (int)(rest % g.nel[1]);
  const int ek = (int)(rest / g.nel[1]);
  const int64_t n0 = ei + (int64_t)g.nn[0] * (ej + (int64_t)g.nn[1] * ek);
  double pe[NN][DIM];
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    const int64_t nb = n0 + corner_x(l) + (int64_t)g.nn[0] * (corner_y(l) + (int64_t)g.nn[1] * corner_z(l));
#pragma unroll
    for (int c = 0; c < DIM; ++c) pe[l][c] = phi[DIM * nb + c];
  }
  const double es = Es[e] * wdet;
  for (int gp = 0; gp < NN; ++gp) {
    const double* dn = dN + gp * DIM * NN;
    double Gr[DIM][DIM];  // Gr[a][c] = d phi_c / d x_a
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < NN; ++l) s += dn[a * NN + l] * pe[l][c];
        Gr[a][c] = s;
      }
    double Hm[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) s += Gr[a][c] * Gr[b][c];
        Hm[a][b] = s;
      }
    double hv[NV];
    if (DIM == 2) {
      hv[0] = Hm[0][0];
      hv[1] = Hm[1][1];
      hv[2] = 2.0 * Hm[0][1];
    } else {
      hv[0] = Hm[0][0];
      hv[1] = Hm[1][1];
      hv[2] = Hm[DIM - 1][DIM - 1];
      hv[3] = 2.0 * Hm[0][1];
      hv[4] = 2.0 * Hm[1][DIM - 1];
      hv[5] = 2.0 * Hm[DIM - 1][0];
    }
#pragma unroll
    for (int p = 0; p < NV; ++p) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < NV; ++q) s += D[p * NV + q] * hv[q];
      sgp[(e * NN + gp) * NV + p] = es * s;
    }
  }
}

// b[a,c] = sum_{e adj a} sum_gp (B(gp)^T s_{e,gp})[local row of (a,c)]  (masked)
template <int DIM>
__global__ void k_adjoint_gather(Grid g, const uint8_t* __restrict__ fixed, const double* __restrict__ sgp,
                                 const double* __restrict__ dN, double* __restrict__ b) {
  constexpr int NN = Dims<DIM>::NN, NV = Dims<DIM>::NV;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(g, node, i, j, k)) return;
  double acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = 0.0;
#pragma unroll
  for (int cz = 0; cz < (DIM == 3 ? 2 : 1); ++cz)
#pragma unroll
    for (int cy = 0; cy < 2; ++cy)
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const int ei = i - cx, ej = j - cy, ek = k - cz;
        if (ei < 0 || ei >= g.nel[0] || ej < 0 || ej >= g.nel[1]) continue;
        if (DIM == 3 && (ek < 0 || ek >= g.nel[2])) continue;
        const int64_t e = ei + (int64_t)g.nel[0] * (ej + (int64_t)g.nel[1] * ek);
        const int ln = local_node(cx, cy, cz);
        for (int gp = 0; gp < NN; ++gp) {
          const double* s = sgp + (e * NN + gp) * NV;
          const double* dn = dN + gp * DIM * NN;
          const double dx = dn[0 * NN + ln], dy = dn[1 * NN + ln];
          if (DIM == 2) {
            acc[0] += dx * s[0] + dy * s[2];
            acc[1] += dy * s[1] + dx * s[2];
          } else {
            const double dz = dn[(DIM - 1) * NN + ln];
            acc[0] += dx * s[0] + dy * s[3] + dz * s[5];
            acc[1] += dy * s[1] + dx * s[3] + dz * s[4];
            acc[DIM - 1] += dz * s[2] + dy * s[4] + dx * s[5];
          }
        }
      }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t idx = DIM * node + c;
    b[idx] = fixed[idx] ? 0.0 : acc[c];
  }
}

void launch_adjoint_gather(const Grid& g, const uint8_t* fixed, const double* sgp, const double* dN, double* b,
                           cudaStream_t st) {
  if (g.dim == 2)
    ::tobk::note_launch(), k_adjoint_gather<2><<<nblk(g.nnode), 256, 0, st>>>(g, fixed, sgp, dN, b);
  else
    ::tobk::note_launch(), k_adjoint_gather<3><<<nblk(g.nnode), 256, 0, st>>>(g, fixed, sgp, dN, b);
}

// per element: dJ and, for every mode, dlambda (eq. SensitivityLambda with -1/(phi^T G phi))
template <int DIM>
__global__ void k_sensitivities(Grid g, int q, const double* __restrict__ u, const double* __restrict__ modes,
                                const double* __restrict__ adj, const double* __restrict__ Gs0,
                                const double* __restrict__ Gc0, const double* __restrict__ Ke0,
                                const double* __restrict__ dEk,
                                const double* __restrict__ dEs, const double* __restrict__ lam,
                                const double* __restrict__ pGp_glob, double* __restrict__ dlam,
                                double* __restrict__ dJ) {
  constexpr int NN = Dims<DIM>::NN, ND = Dims<DIM>::ND;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.m) return;
  const int ei = (int)(e % g.nel[0]);
  const int64_t rest = e / g.nel[0];
  const int ej = (int)(rest % g.nel[1]);
  const int ek = (int)(rest / g.nel[1]);
  const int64_t n0 = ei + (int64_t)g.nn[0] * (ej + (int64_t)g.nn[1] * ek);
  int64_t dof[ND];
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    const int64_t nb = n0 + corner_x(l) + (int64_t)g.nn[0] * (corner_y(l) + (int64_t)g.nn[1] * corner_z(l));
#pragma unroll
    for (int c = 0; c < DIM; ++c) dof[l * DIM + c] = DIM * nb + c;
  }
  double Ku[ND];
  double uKu = 0.0;
  {
    double ue[ND];
#pragma unroll
    for (int a = 0; a < ND; ++a) ue[a] = u[dof[a]];
    for (int a = 0; a < ND; ++a) {
      double s = 0.0;
#pragma unroll
      for (int b = 0; b < ND; ++b) s += Ke0[a * ND + b] * ue[b];
      Ku[a] = s;
      uKu += ue[a] * s;
    }
  }
  const double dek = dEk[e], des = dEs[e];
  dJ[e] = -dek * uKu;
  const double* G0 = Gs0 + e * NN * NN;
  const int64_t n = g.n;
  for (int i = 0; i < q; ++i) {
    double pe[ND];
#pragma unroll
    for (int a = 0; a < ND; ++a) pe[a] = modes[(int64_t)i * n + dof[a]];
    double pKp = 0.0;
    for (int a = 0; a < ND; ++a) {
      double s = 0.0;
#pragma unroll
      for (int b = 0; b < ND; ++b) s += Ke0[a * ND + b] * pe[b];
      pKp += pe[a] * s;
    }
    double pGp = 0.0;
    if (Gc0) {  // condensed stress stiffness of the incompatible-mode element (dense, unit modulus)
      const double* Gc = Gc0 + e * ND * ND;
      for (int a = 0; a < ND; ++a) {
        double s = 0.0;
        for (int b = 0; b < ND; ++b) s += Gc[a * ND + b] * pe[b];
        pGp += pe[a] * s;
      }
    } else {
      for (int a = 0; a < NN; ++a)
        for (int b = 0; b < NN; ++b) {
          double s = 0.0;
#pragma unroll
          for (int c = 0; c < DIM; ++c) s += pe[a * DIM + c] * pe[b * DIM + c];
          pGp += G0[a * NN + b] * s;
        }
    }
    double zKu = 0.0;
#pragma unroll
    for (int a = 0; a < ND; ++a) zKu += adj[(int64_t)i * n + dof[a]] * Ku[a];
    const double li = lam[i];
    dlam[(int64_t)i * g.m + e] = -(dek * pKp + li * des * pGp - li * dek * zKu) / pGp_glob[i];
  }
}

int compute_sensitivities(tobk_handle* h, double* dlam_out, double* dJ_out, bool out_on_device,
                          tobk_solve_info* info) {
  if (!h->have_modes) return fail(h, TOBK_E_STATE, "compute_buckling must come first");
  cudaStream_t st = h->stream;
  const Grid& g = h->lv[0].g;
  const int64_t n = g.n;
  const int q = h->q;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  // consistent sensitivities of the multilevel pairs: fine and coarse adjoints, combined right-hand sides
  const bool cons = h->cs_ready && h->cs_psi;
  tobk_solve_info ci{};
  int rc_c = TOBK_OK;
  if (cons) {
    rc_c = consistent_adjoint_rhs(h, h->adj_rhs, &ci);
    if (rc_c && rc_c != TOBK_E_NOT_CONVERGED) return rc_c;
  }
  // adjoint right-hand sides, one mode at a time through the element Gauss-point scratch
  for (int i = 0; i < (cons ? 0 : q); ++i) {
    const double* phi = h->modes + (size_t)i * n;
    double* b = h->adj_rhs + (size_t)i * n;
    if (h->Gc0) {
      launch_inc_adjoint(g, h->lv[0].fixed, phi, h->Es, h->d_A, h->d_dN, h->d_D, h->tab.wdet, h->esens, b, st);
    } else if (g.dim == 2) {
      ::tobk::note_launch(), k_adjoint_gp<2><<<nblk(g.m, 128), 128, 0, st>>>(g, phi, h->Es, h->d_dN, h->d_D, h->tab.wdet, h->esens);
      ::tobk::note_launch(), k_adjoint_gather<2><<<nblk(g.nnode), 256, 0, st>>>(g, h->lv[0].fixed, h->esens, h->d_dN, b);
    } else {
      ::tobk::note_launch(), k_adjoint_gp<3><<<nblk(g.m, 128), 128, 0, st>>>(g, phi, h->Es, h->d_dN, h->d_D, h->tab.wdet, h->esens);
      ::tobk::note_launch(), k_adjoint_gather<3><<<nblk(g.nnode), 256, 0, st>>>(g, h->lv[0].fixed, h->esens, h->d_dN, b);
    }
  }
  // adjoint systems K z_i = b_i: one multi-RHS mgPCG solve (optionally with the load as an extra
  // column, K [u, Z] = [f, B], the new u replacing the stored one)
  tobk_solve_info si{};
  int rc;
  if (h->desc.fuse_load_adjoint) {
    launch_mask_copy(h->f, h->lv[0].fixed, h->adj_blockB, n, 1, n, st);
    rc = pcg_solve(h, 0, h->adj_blockB, h->adj_blockX, q + 1, h->desc.rtol, h->desc.max_iter, false,
                   h->desc.precision, &si);
    if (rc && rc != TOBK_E_NOT_CONVERGED) return rc;
    cudaMemcpyAsync(h->u, h->adj_blockX, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  } else {
    rc = pcg_solve(h, 0, h->adj_rhs, h->adj, q, h->desc.rtol, h->desc.max_iter, false, h->desc.precision, &si);
    if (rc && rc != TOBK_E_NOT_CONVERGED) return rc;
  }
  // phi_i^T G phi_i
  double* GP = h->lv[0].z;
  apply_G_level(h, 0, h->modes, GP, q, n);
  double* pGp = h->dscal + 960;
  launch_coldots(h->modes, GP, q, n, n, pGp, h->gram_partial, st);
  const int qs = cons ? 0 : q;  // the consistent path leaves dJ alone to this kernel
  if (g.dim == 2)
    ::tobk::note_launch(), k_sensitivities<2><<<nblk(g.m, 128), 128, 0, st>>>(g, qs, h->u, h->modes, h->adj, h->Gs0, h->Gc0, h->d_Ke0, h->dEk,
                                                       h->dEs, h->lam, pGp, h->dlam, h->dJ);
  else
    ::tobk::note_launch(), k_sensitivities<3><<<nblk(g.m, 64), 64, 0, st>>>(g, qs, h->u, h->modes, h->adj, h->Gs0, h->Gc0, h->d_Ke0, h->dEk, h->dEs,
                                                     h->lam, pGp, h->dlam, h->dJ);
  if (cons) launch_sens_consistent(h, pGp);
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (dlam_out) cudaMemcpyAsync(dlam_out, h->dlam, sizeof(double) * q * g.m, kind, st);
  if (dJ_out) cudaMemcpyAsync(dJ_out, h->dJ, sizeof(double) * g.m, kind, st);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  int crc = check_cuda(h, "compute_sensitivities");
  if (crc) return crc;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    *info = si;
    info->time_ms = ms;
    if (cons) {
      info->iterations = std::max(si.iterations, ci.iterations);
      info->converged = si.converged && ci.converged;
      info->status_detail = ci.status_detail;
    }
  }
  h->have_sens = true;
  h->have_cs = cons;
  return rc ? rc : rc_c;
}

}  // namespace tobk
