// Consistent sensitivities of the multilevel load factors (Sec. 2.1, eq. eigResidual; Appendix A,
// eq. consistentSensitivity): the exact derivative of lambda_i = -phi^T K phi / phi^T G phi with
// phi = K^{-1} G P psi_i, through the coarse pencil (K^l, G^l), the prolongation P and the fine solve.
// With D = -1/(phi^T G phi), Psi = P psi and mu the coarse load factor of psi:
//
//   y = (K + lambda G) phi                               residual of the pair (eq. eigResidual)
//   K w = y                                              fine adjoint: multi-RHS mgPCG (SPD)
//   b = P^T G w                                          restriction to Omega_l (psi^T b = y^T phi = 0)
//   (K^l + mu G^l) c = b,  psi^T G^l c = 0               coarse adjoint: deflated PCG (below)
//   g = grad_v [lambda phi^T G[v] phi + (2 w - 2 mu P c)^T G[v] Psi]   right-hand side of the u-adjoint
//   K z = g                                              (the solve of eq. AdjointSystem)
//   d lambda / d x_e = D { dE_kappa [ (phi - 2 w)^T K_e0 phi - 2 (P c)^T K_e0 Psi - z^T K_e0 u ]
//                        + dE_sigma [ lambda phi^T G_e0 phi + (2 w - 2 mu P c)^T G_e0 Psi ] }
//
// w = 0 and c = 0 leave eq. SensitivityLambda.  lambda does not change when psi is scaled, so the
// pairing of a fine mode with its coarse mode only has to keep one scale: the normalised fine mode
// phi_r = s_r K^{-1} G P psi_{perm r} goes with Psi_r = s_r P psi_{perm r} (perm, s from the mode
// normalisation of compute_buckling).
//
// Coarse adjoint.  In the eigenbasis of the pencil (K^l psi_j = -mu_j G^l psi_j, psi_j^T K^l psi_k =
// delta_jk) the operator K^l + mu G^l scales component j by 1 - mu / mu_j: negative for the modes below
// the wanted one, zero for it, and at least 1 - mu / mu_{q+1} > 0 beyond the q computed modes.  The
// computed modes' components are therefore taken exactly, c_j = psi_j^T b / (1 - mu / mu_j) (none
// along the wanted mode, which is the constraint psi^T G^l c = 0), and the rest by CG on the
// K^l-orthogonal complement of the computed modes, where the operator is positive definite: residuals
// projected by I - K^l Q Q^T, preconditioned residuals (one V-cycle of K^l) by I - Q Q^T K^l, with the
// flexible (Polak-Ribiere) step so that an FP32 V-cycle may serve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"
#include "handle.h"

namespace tobk {

void launch_coldots(const double* A, const double* B, int ncols, int64_t n, int64_t stride, double* out,
                    double* partial, cudaStream_t s);
void launch_adjoint_gather(const Grid& g, const uint8_t* fixed, const double* sgp, const double* dN, double* b,
                           cudaStream_t st);

namespace {

// device scalar layout of h->cs_scal (kCsSize doubles): three [q][q] blocks (q <= 24), per-mode arrays
constexpr int kCsC0 = 0, kCsC1 = 576, kCsCoef = 1152, kCsMu = 1728, kCsRzA = 1792, kCsRzB = 1856, kCsRzM = 1920,
              kCsPq = 1984, kCsRr = 2048, kCsScale = 2112, kCsPerm = 2176;
static_assert(kCsPerm + 32 <= kCsSize, "consistent-sensitivity scalars overflow");

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Y_r = A_r + coef[r] B_r for the nr columns of length n (stride n); Y may alias A.
__global__ void k_cols_axpy(const double* A, const double* B, const double* coef, double* Y, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int64_t o = (int64_t)blockIdx.y * n + k;
  Y[o] = A[o] + coef[blockIdx.y] * B[o];
}

// dst_r = scale[r] src_{perm[r]}
__global__ void k_perm_scale(const double* src, const int* perm, const double* scale, double* dst, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int r = blockIdx.y;
  dst[(int64_t)r * n + k] = scale[r] * src[(int64_t)perm[r] * n + k];
}

// x_r += alpha_r p_r, r_r -= alpha_r ap_r with alpha_r = rz[r] / pq[r] (0 where pq[r] = 0)
__global__ void k_pcg_step(double* x, double* r, const double* p, const double* ap, const double* rz,
                           const double* pq, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int c = blockIdx.y;
  const double d = pq[c];
  const double alpha = d != 0.0 ? rz[c] / d : 0.0;
  const int64_t o = (int64_t)c * n + k;
  x[o] += alpha * p[o];
  r[o] -= alpha * ap[o];
}

// p_r = z_r + beta_r p_r, beta_r = (rz_new[r] - rz_mix[r]) / rz_old[r] (flexible form; 0 where rz_old = 0)
__global__ void k_pcg_dir(double* p, const double* z, const double* rz_new, const double* rz_mix,
                          const double* rz_old, int64_t n) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int c = blockIdx.y;
  const double d = rz_old[c];
  const double beta = d != 0.0 ? (rz_new[c] - rz_mix[c]) / d : 0.0;
  const int64_t o = (int64_t)c * n + k;
  p[o] = z[o] + beta * p[o];
}

// Gauss-point vectors of the u-adjoint right-hand side of one mode:
//   s_gp = E_sigma w|J| D h,  h = lam h(phi, phi) + h(a, Psi),  a = 2 w - 2 mu Chat,
// h(a, c) the Voigt vector of H_ij = sum_k d_i a_k d_j c_k with the shear entries H_ij + H_ji (S : H for
// a symmetric stress S); the element gather B^T s gives grad_v of the bilinear stress forms.
template <int DIM>
__global__ void k_adjoint_gp_pair(Grid g, const double* __restrict__ phi, const double* __restrict__ w,
                                  const double* __restrict__ ch, const double* __restrict__ Psi, double lam,
                                  double mu, const double* __restrict__ Es, const double* __restrict__ dN,
                                  const double* __restrict__ D, double wdet, double* __restrict__ sgp) {
  constexpr int NN = Dims<DIM>::NN, NV = Dims<DIM>::NV;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.m) return;
  const int ei = (int)(e % g.nel[0]);
  const int64_t rest = e / g.nel[0];
  const int ej = (int)(rest % g.nel[1]);
  const int ek = (int)(rest / g.nel[1]);
  const int64_t n0 = ei + (int64_t)g.nn[0] * (ej + (int64_t)g.nn[1] * ek);
  double pe[NN][DIM], ae[NN][DIM], se[NN][DIM];
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    const int64_t nb = n0 + corner_x(l) + (int64_t)g.nn[0] * (corner_y(l) + (int64_t)g.nn[1] * corner_z(l));
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t k = DIM * nb + c;
      pe[l][c] = phi[k];
      ae[l][c] = 2.0 * w[k] - 2.0 * mu * ch[k];
      se[l][c] = Psi[k];
    }
  }
  const double es = Es[e] * wdet;
  for (int gp = 0; gp < NN; ++gp) {
    const double* dn = dN + gp * DIM * NN;
    double Gp[DIM][DIM], Ga[DIM][DIM], Gs[DIM][DIM];  // [i][k] = d v_k / d x_i
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double sp = 0.0, sa = 0.0, ss = 0.0;
#pragma unroll
        for (int l = 0; l < NN; ++l) {
          const double d = dn[i * NN + l];
          sp += d * pe[l][c];
          sa += d * ae[l][c];
          ss += d * se[l][c];
        }
        Gp[i][c] = sp;
        Ga[i][c] = sa;
        Gs[i][c] = ss;
      }
    double H[DIM][DIM];
#pragma unroll
    for (int i = 0; i < DIM; ++i)
#pragma unroll
      for (int j = 0; j < DIM; ++j) {
        double hp = 0.0, hb = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          hp += Gp[i][c] * Gp[j][c];
          hb += Ga[i][c] * Gs[j][c];
        }
        H[i][j] = lam * hp + hb;
      }
    double hv[NV];
    if (DIM == 2) {
      hv[0] = H[0][0];
      hv[1] = H[1][1];
      hv[2] = H[0][1] + H[1][0];
    } else {
      hv[0] = H[0][0];
      hv[1] = H[1][1];
      hv[2] = H[DIM - 1][DIM - 1];
      hv[3] = H[0][1] + H[1][0];
      hv[4] = H[1][DIM - 1] + H[DIM - 1][1];
      hv[5] = H[DIM - 1][0] + H[0][DIM - 1];
    }
#pragma unroll
    for (int p = 0; p < NV; ++p) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < NV; ++k) s += D[p * NV + k] * hv[k];
      sgp[(e * NN + gp) * NV + p] = es * s;
    }
  }
}

template <int DIM>
constexpr int kSensBlock = DIM == 2 ? 128 : 64;

// per element and mode: the consistent derivative (header formula); dJ is left to the plain kernel.
// Every element array is indexed by unrolled loops only (registers, no local memory); Ke0 and the
// element's node-block stress stiffness are read through the cache.
template <int DIM>
__global__ void __launch_bounds__(kSensBlock<DIM>) k_sens_consistent(Grid g, int q, const double* __restrict__ u, const double* __restrict__ phi,
                                  const double* __restrict__ w, const double* __restrict__ ch,
                                  const double* __restrict__ Psi, const double* __restrict__ z,
                                  const double* __restrict__ Gs0, const double* __restrict__ Ke0,
                                  const double* __restrict__ dEk, const double* __restrict__ dEs,
                                  const double* __restrict__ lam, const double* __restrict__ mu,
                                  const double* __restrict__ pGp, double* __restrict__ dlam) {
  constexpr int NN = Dims<DIM>::NN, ND = Dims<DIM>::ND;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.m) return;
  const int ei = (int)(e % g.nel[0]);
  const int64_t rest = e / g.nel[0];
  const int ej = (int)(rest % g.nel[1]);
  const int ek = (int)(rest / g.nel[1]);
  const int64_t n0 = ei + (int64_t)g.nn[0] * (ej + (int64_t)g.nn[1] * ek);
  int64_t nb[NN];  // first DOF of each element node
#pragma unroll
  for (int l = 0; l < NN; ++l)
    nb[l] = DIM * (n0 + corner_x(l) + (int64_t)g.nn[0] * (corner_y(l) + (int64_t)g.nn[1] * corner_z(l)));
  __shared__ double sKu[ND * kSensBlock<DIM>];  // K_e0 u_e, [a][thread]
  double* Ku = sKu + threadIdx.x;
  {
    double ue[ND];
#pragma unroll
    for (int a = 0; a < ND; ++a) ue[a] = u[nb[a / DIM] + a % DIM];
#pragma unroll
    for (int a = 0; a < ND; ++a) {
      double s = 0.0;
#pragma unroll
      for (int b = 0; b < ND; ++b) s += __ldg(Ke0 + a * ND + b) * ue[b];
      Ku[a * kSensBlock<DIM>] = s;
    }
  }
  const double dek = dEk[e], des = dEs[e];
  const double* G0 = Gs0 + e * NN * NN;
  const int64_t n = g.n;
  for (int i = 0; i < q; ++i) {
    const int64_t o = (int64_t)i * n;
    double pe[ND], se[ND];
#pragma unroll
    for (int a = 0; a < ND; ++a) {
      pe[a] = phi[o + nb[a / DIM] + a % DIM];
      se[a] = Psi[o + nb[a / DIM] + a % DIM];
    }
    double kpart = 0.0;
#pragma unroll
    for (int a = 0; a < ND; ++a) {
      double kp = 0.0, ks = 0.0;
#pragma unroll
      for (int b = 0; b < ND; ++b) {
        const double k0 = __ldg(Ke0 + a * ND + b);
        kp += k0 * pe[b];
        ks += k0 * se[b];
      }
      const int64_t k = o + nb[a / DIM] + a % DIM;
      kpart += (pe[a] - 2.0 * w[k]) * kp - 2.0 * ch[k] * ks - z[k] * Ku[a * kSensBlock<DIM>];
    }
    // lambda phi^T G0 phi + (2 w - 2 mu P c)^T G0 Psi, G0 acting on each displacement component
    const double li = lam[i], mi = mu[i];
    double gpart = 0.0;
#pragma unroll
    for (int il = 0; il < NN; ++il)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double tp = 0.0, ts = 0.0;
#pragma unroll
        for (int j = 0; j < NN; ++j) {
          const double g0 = G0[il * NN + j];
          tp += g0 * pe[j * DIM + c];
          ts += g0 * se[j * DIM + c];
        }
        const int64_t k = o + nb[il] + c;
        gpart += li * pe[il * DIM + c] * tp + (2.0 * w[k] - 2.0 * mi * ch[k]) * ts;
      }
    dlam[(int64_t)i * g.m + e] = -(dek * kpart + des * gpart) / pGp[i];
  }
}

void prolong_chain(tobk_handle* h, const double* coarse, double* fine, int q) {
  // Omega_l -> Omega_1 through the level buffers b (free in this phase): Psi^j = I^j_{j+1} Psi^{j+1}
  cudaStream_t st = h->stream;
  const int l = h->eig;
  cudaMemcpyAsync(h->lv[l].b, coarse, sizeof(double) * q * h->lv[l].g.n, cudaMemcpyDeviceToDevice, st);
  for (int j = l; j >= 1; --j) {
    Level& C = h->lv[j];
    Level& F = h->lv[j - 1];
    double* dst = j == 1 ? fine : F.b;
    cudaMemsetAsync(dst, 0, sizeof(double) * q * F.g.n, st);
    launch_prolong_add(F.g, C.g, F.fixed, C.b, dst, q, F.g.n, C.g.n, st);
  }
}

void restrict_chain(tobk_handle* h, const double* fine, double* coarse, int q) {
  // b = P^T r: Omega_1 -> Omega_l through the level buffers b
  cudaStream_t st = h->stream;
  const int l = h->eig;
  const double* src = fine;
  for (int j = 0; j < l; ++j) {
    Level& F = h->lv[j];
    Level& C = h->lv[j + 1];
    double* dst = j + 1 == l ? coarse : C.b;
    launch_restrict(F.g, C.g, C.fixed, src, dst, q, F.g.n, C.g.n, st);
    src = dst;
  }
}

}  // namespace

// The coarse adjoint (K^l + mu_r G^l) c_r = b_r, psi_r^T G^l c_r = 0 for the q modes (header).  b, c
// [q][n_l] in the fine modes' order; the pencil's computed modes are h->cs_psi (eigensolver order).
static int coarse_adjoint(tobk_handle* h, const double* b, double* c, int* iters) {
  cudaStream_t st = h->stream;
  const int l = h->eig, q = h->q;
  const int64_t nl = h->lv[l].g.n;
  const dim3 grid(nblk(nl), q);
  double* Q = h->cs_psi;
  double* KQ = h->cs_Kpsi;
  double* R = h->cs_r;
  double* R0 = h->cs_r0;
  double* Z = h->cs_z;
  double* P = h->cs_p;
  double* AP = h->cs_ap;
  double* GP = h->cs_t;
  double* sc = h->cs_scal;
  double* C0 = sc + kCsC0;  // [q][q] Gram blocks
  double* C1 = sc + kCsC1;
  double* coef = sc + kCsCoef;
  double* mu_dev = sc + kCsMu;
  double* rz_a = sc + kCsRzA;
  double* rz_b = sc + kCsRzB;
  double* rz_m = sc + kCsRzM;
  double* pq = sc + kCsPq;
  double* rr = sc + kCsRr;
  apply_K_level(h, l, Q, KQ, q, nl);
  // components along the computed modes: C0[j][r] = psi_j^T b_r; R = b - K^l Q C0
  launch_gram(Q, q, b, q, nl, nl, C0, h->gram_partial, st);
  cudaMemcpyAsync(R, b, sizeof(double) * q * nl, cudaMemcpyDeviceToDevice, st);
  launch_combine(KQ, q, C0, q, q, -1.0, 1.0, R, nl, nl, st);
  cudaMemsetAsync(c, 0, sizeof(double) * q * nl, st);
  auto project_s = [&](double* X) {  // X -= Q (K^l Q)^T X
    launch_gram(KQ, q, X, q, nl, nl, C1, h->gram_partial, st);
    launch_combine(Q, q, C1, q, q, -1.0, 1.0, X, nl, nl, st);
  };
  auto project_r = [&](double* X) {  // X -= K^l Q Q^T X
    launch_gram(Q, q, X, q, nl, nl, C1, h->gram_partial, st);
    launch_combine(KQ, q, C1, q, q, -1.0, 1.0, X, nl, nl, st);
  };
  apply_vcycle(h, l, q, R, Z);
  project_s(Z);
  cudaMemcpyAsync(P, Z, sizeof(double) * q * nl, cudaMemcpyDeviceToDevice, st);
  launch_coldots(R, Z, q, nl, nl, rz_a, h->gram_partial, st);
  launch_coldots(R, R, q, nl, nl, rr, h->gram_partial, st);
  double* hs = h->hscal;
  cudaMemcpyAsync(hs, rr, sizeof(double) * q, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  double tol2[64];
  for (int r = 0; r < q; ++r) tol2[r] = h->desc.rtol * h->desc.rtol * hs[r];
  bool done = true;  // nothing to do when every projected right-hand side is 0
  for (int r = 0; r < q; ++r)
    if (hs[r] > 0.0) done = false;
  // Two iterations and the exit test (||r_r||^2 into the pinned host scalars) per replay of a CUDA graph
  // captured on first use; launched directly while profiling or on the legacy default stream.
  auto enqueue_pair = [&]() {
    for (int k = 0; k < 2; ++k) {
      double* rz_old = k == 0 ? rz_a : rz_b;
      double* rz_new = k == 0 ? rz_b : rz_a;
      apply_K_level(h, l, P, AP, q, nl);
      apply_G_level(h, l, P, GP, q, nl);
      ::tobk::note_launch(), k_cols_axpy<<<grid, 256, 0, st>>>(AP, GP, mu_dev, AP, nl);
      project_r(AP);
      launch_coldots(P, AP, q, nl, nl, pq, h->gram_partial, st);
      cudaMemcpyAsync(R0, R, sizeof(double) * q * nl, cudaMemcpyDeviceToDevice, st);
      ::tobk::note_launch(), k_pcg_step<<<grid, 256, 0, st>>>(c, R, P, AP, rz_old, pq, nl);
      apply_vcycle(h, l, q, R, Z);
      project_s(Z);
      launch_coldots(R, Z, q, nl, nl, rz_new, h->gram_partial, st);
      launch_coldots(R0, Z, q, nl, nl, rz_m, h->gram_partial, st);
      ::tobk::note_launch(), k_pcg_dir<<<grid, 256, 0, st>>>(P, Z, rz_new, rz_m, rz_old, nl);
    }
    launch_coldots(R, R, q, nl, nl, rr, h->gram_partial, st);
    cudaMemcpyAsync(hs, rr, sizeof(double) * q, cudaMemcpyDeviceToHost, st);
  };
  const bool graphs = !h->prof_on && st != nullptr && h->use_graphs;
  const uint64_t key = (1ull << 40) | (uint64_t)l;  // beside the CG pairs' (level, RHS, precision) keys
  const int maxit = h->desc.max_iter;
  int it = 0;
  while (!done && it < maxit) {
    if (graphs) {
      auto g = h->cg_graphs.find(key);
      if (g == h->cg_graphs.end()) {
        cudaGraph_t gr = nullptr;
        const long long c0 = g_launch_count.load();
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
          return check_cuda(h, "coarse adjoint capture");
        enqueue_pair();
        if (cudaStreamEndCapture(st, &gr) != cudaSuccess) return check_cuda(h, "coarse adjoint capture");
        const long long kernels = g_launch_count.load() - c0;
        g_launch_count.fetch_sub(kernels);
        cudaGraphExec_t ex = nullptr;
        if (cudaGraphInstantiate(&ex, gr, 0) != cudaSuccess) {
          cudaGraphDestroy(gr);
          return check_cuda(h, "coarse adjoint instantiate");
        }
        cudaGraphDestroy(gr);
        g = h->cg_graphs.emplace(key, tobk_handle::CGGraph{ex, kernels}).first;
      }
      cudaGraphLaunch(g->second.exec, st);
      g_launch_count.fetch_add(g->second.kernels);
    } else {
      enqueue_pair();
    }
    it += 2;
    cudaStreamSynchronize(st);
    done = true;
    for (int r = 0; r < q; ++r) {
      if (!std::isfinite(hs[r])) return fail(h, TOBK_E_NONFINITE, "coarse adjoint: non-finite residual");
      if (hs[r] > tol2[r]) done = false;
    }
  }
  // c += sum_{j != perm r} psi_j (psi_j^T b_r) / (1 - mu_r / mu_j)
  std::vector<double> c0((size_t)q * q), cf((size_t)q * q, 0.0);
  cudaMemcpyAsync(c0.data(), C0, sizeof(double) * q * q, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  for (int j = 0; j < q; ++j)
    for (int r = 0; r < q; ++r) {
      if (j == h->cs_perm[r]) continue;
      const double m_r = h->cs_mu[h->cs_perm[r]], m_j = h->cs_mu[j];
      const double d = 1.0 - m_r / m_j;  // 0 only for a repeated coarse load factor (no unique derivative)
      cf[(size_t)j * q + r] = d != 0.0 ? c0[(size_t)j * q + r] / d : 0.0;
    }
  cudaMemcpyAsync(coef, cf.data(), sizeof(double) * q * q, cudaMemcpyHostToDevice, st);
  launch_combine(Q, q, coef, q, q, 1.0, 1.0, c, nl, nl, st);
  cudaStreamSynchronize(st);  // cf is read by the copy above
  *iters = it;
  return done ? TOBK_OK : TOBK_E_NOT_CONVERGED;
}

// Everything of the consistent derivative up to the u-adjoint right-hand side, written to g [q][n]
// (fine adjoint w, coarse adjoint P c and the prolongated modes Psi stay in the handle for the
// sensitivity kernel and tobk_get_field).
int consistent_adjoint_rhs(tobk_handle* h, double* g_out, tobk_solve_info* info) {
  cudaStream_t st = h->stream;
  const Grid& g = h->lv[0].g;
  const int64_t n = g.n;
  const int q = h->q;
  double* sc = h->cs_scal;
  double* mu_dev = sc + kCsMu;
  double* scale_dev = sc + kCsScale;
  int* perm_dev = (int*)(sc + kCsPerm);
  {
    double hm[64], hsc[64];
    for (int r = 0; r < q; ++r) {
      hm[r] = h->cs_mu[h->cs_perm[r]];
      hsc[r] = h->cs_scale[r];
    }
    cudaMemcpyAsync(mu_dev, hm, sizeof(double) * q, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(scale_dev, hsc, sizeof(double) * q, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(perm_dev, h->cs_perm, sizeof(int) * q, cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);  // the host arrays above are on the stack
  }
  // Psi_r = s_r P psi_{perm r}
  prolong_chain(h, h->cs_psi, h->xwork, q);
  ::tobk::note_launch(), k_perm_scale<<<dim3(nblk(n), q), 256, 0, st>>>(h->xwork, perm_dev, scale_dev, h->cs_Psi, n);
  // y = K phi + lambda G phi; K w = y
  double* Y = h->bwork;
  apply_K_level(h, 0, h->modes, Y, q, n);
  apply_G_level(h, 0, h->modes, h->xwork, q, n);
  ::tobk::note_launch(), k_cols_axpy<<<dim3(nblk(n), q), 256, 0, st>>>(Y, h->xwork, h->lam, Y, n);
  tobk_solve_info si{};
  int rc = pcg_solve(h, 0, Y, h->cs_W, q, h->desc.rtol, h->desc.max_iter, false, h->desc.precision, &si);
  if (rc && rc != TOBK_E_NOT_CONVERGED) return rc;
  // b = P^T G w; coarse adjoint c; P c
  apply_G_level(h, 0, h->cs_W, h->xwork, q, n);
  restrict_chain(h, h->xwork, h->cs_b, q);
  int cit = 0;
  int crc = coarse_adjoint(h, h->cs_b, h->cs_c, &cit);
  if (crc && crc != TOBK_E_NOT_CONVERGED) return crc;
  prolong_chain(h, h->cs_c, h->cs_C, q);
  // g = grad_v [lambda phi^T G[v] phi + (2 w - 2 mu P c)^T G[v] Psi], one mode at a time
  for (int r = 0; r < q; ++r) {
    const int64_t o = (int64_t)r * n;
    const double lam = h->lam_host[r], mu = h->cs_mu[h->cs_perm[r]];
    if (g.dim == 2)
      ::tobk::note_launch(), k_adjoint_gp_pair<2><<<nblk(g.m, 128), 128, 0, st>>>(
          g, h->modes + o, h->cs_W + o, h->cs_C + o, h->cs_Psi + o, lam, mu, h->Es, h->d_dN, h->d_D, h->tab.wdet,
          h->esens);
    else
      ::tobk::note_launch(), k_adjoint_gp_pair<3><<<nblk(g.m, 64), 64, 0, st>>>(
          g, h->modes + o, h->cs_W + o, h->cs_C + o, h->cs_Psi + o, lam, mu, h->Es, h->d_dN, h->d_D, h->tab.wdet,
          h->esens);
    launch_adjoint_gather(g, h->lv[0].fixed, h->esens, h->d_dN, g_out + o, st);
  }
  if (info) {
    info->iterations = si.iterations;
    info->status_detail = cit;
    info->converged = (rc == TOBK_OK && crc == TOBK_OK) ? 1 : 0;
  }
  return (rc == TOBK_OK && crc == TOBK_OK) ? TOBK_OK : TOBK_E_NOT_CONVERGED;
}

void launch_sens_consistent(tobk_handle* h, const double* pGp) {
  cudaStream_t st = h->stream;
  const Grid& g = h->lv[0].g;
  const double* mu_sorted_dev = h->cs_scal + kCsMu;
  if (g.dim == 2)
    ::tobk::note_launch(), k_sens_consistent<2><<<nblk(g.m, kSensBlock<2>), kSensBlock<2>, 0, st>>>(
        g, h->q, h->u, h->modes, h->cs_W, h->cs_C, h->cs_Psi, h->adj, h->Gs0, h->d_Ke0, h->dEk, h->dEs, h->lam,
        mu_sorted_dev, pGp, h->dlam);
  else
    ::tobk::note_launch(), k_sens_consistent<3><<<nblk(g.m, kSensBlock<3>), kSensBlock<3>, 0, st>>>(
        g, h->q, h->u, h->modes, h->cs_W, h->cs_C, h->cs_Psi, h->adj, h->Gs0, h->d_Ke0, h->dEk, h->dEs, h->lam,
        mu_sorted_dev, pGp, h->dlam);
}

}  // namespace tobk
