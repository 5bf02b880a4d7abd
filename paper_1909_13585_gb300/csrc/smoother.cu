// Smoother of the geometric multigrid that preconditions mgPCG (Appendix A; the paper leaves the
// smoother open).
//
// Multigrid smoother set-up: the spectral radius of D^{-1} K on every level (power iteration on the
// device) and the per-step coefficients of the smoother (damped Jacobi, or a Chebyshev polynomial
// in D^{-1} K over [lambda_max / ratio, lambda_max]).
//
// On unit H8 elements the largest eigenvalue of D^{-1} K is about 4.5, so damped Jacobi with the
// customary omega = 0.6 amplifies the highest frequencies (omega lambda_max > 2) and the
// preconditioned CG needs hundreds of iterations; the Chebyshev smoother adapts to the measured
// lambda_max on each level and each design.
#include <cuda_runtime.h>

#include <cmath>

#include "device_common.cuh"
#include "handle.h"

namespace tobk {

__global__ void k_fill_hash(double* v, const uint8_t* fixed, int64_t n, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t x = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  v[i] = fixed[i] ? 0.0 : (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// y <- dinv .* y, and its squared norm (written by the last block to nrm2[0])
__global__ void k_dinv_scale_norm(double* y, const double* dinv, int64_t n, double* partial, unsigned* counter,
                                  double* nrm2) {
  __shared__ double smem[32];
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double s = dinv[i] * y[i];
    y[i] = s;
    v[0] += s * s;
  }
  double tot[1];
  if (grid_sum_last<1>(v, partial, counter, tot, smem) && threadIdx.x == 0) nrm2[0] = tot[0];
}

__global__ void k_normalize(const double* y, double* v, int64_t n, const double* nrm2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
  v[i] = y[i] * s;
}

// Per-step coefficients (a_k, c_k) for k = 0..steps-1:
//   Chebyshev on [lmin, lmax]: theta = (lmax + lmin)/2, delta = (lmax - lmin)/2, sigma = theta/delta,
//   rho_0 = 1/sigma, (a_0, c_0) = (0, 1/theta), rho_k = 1/(2 sigma - rho_{k-1}),
//   a_k = rho_k rho_{k-1}, c_k = 2 rho_k / delta;  the step is d_k = a_k d_{k-1} + c_k D^{-1} r_k.
//   Damped Jacobi: (0, omega) for every step.
__global__ void k_smoother_coefs(const double* nrm2, int steps, int chebyshev, double ratio, double omega,
                                 double* coef, float* coef32) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double lmax = 1.1 * sqrt(nrm2[0]);  // ||D^{-1} K v|| with ||v|| = 1, plus a safety margin
  if (!chebyshev || !(lmax > 0.0)) {
    for (int k = 0; k < steps; ++k) {
      coef[2 * k] = 0.0;
      coef[2 * k + 1] = omega;
    }
  } else {
    const double lmin = lmax / ratio;
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    coef[0] = 0.0;
    coef[1] = 1.0 / theta;
    for (int k = 1; k < steps; ++k) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      coef[2 * k] = rn * rho;
      coef[2 * k + 1] = 2.0 * rn / delta;
      rho = rn;
    }
  }
  if (coef32)
    for (int k = 0; k < 2 * steps; ++k) coef32[k] = (float)coef[k];
  coef[2 * kMaxSmoothSteps] = lmax;
}

void setup_smoothers(tobk_handle* h) {
  cudaStream_t s = h->stream;
  const int steps = std::max(h->desc.nu_pre, h->desc.nu_post);
  const bool cheb = h->desc.smoother == TOBK_SMOOTHER_CHEBYSHEV;
  const bool mixed = h->desc.precision == TOBK_FP32_VCYCLE;
  double* nrm2 = h->dscal + 1002;
  for (int j = 0; j + 1 < h->L; ++j) {
    Level& L = h->lv[j];
    const int64_t n = L.g.n;
    if (cheb) {
      double* v = h->cg.z;   // scratch (the CG is not running during set-up)
      double* y = h->cg.zt;
      const unsigned nb = (unsigned)((n + 255) / 256);
      note_launch();
      k_fill_hash<<<nb, 256, 0, s>>>(v, L.fixed, n, 0x12345ull + (uint64_t)j);
      const LevelOpDesc op = level_op(h, j);
      const unsigned rb = (unsigned)std::min<int64_t>(nb, 608);
      for (int it = 0; it < 12; ++it) {
        launch_apply(op, APPLY_KV, v, nullptr, nullptr, y, SmoothArgs<double>{}, 1, n, s);
        note_launch();
        k_dinv_scale_norm<<<rb, 256, 0, s>>>(y, L.dinv, n, h->cg.partial, h->cg.counters + 5 * kMaxRhs, nrm2);
        note_launch();
        k_normalize<<<nb, 256, 0, s>>>(y, v, n, nrm2);
      }
    }
    note_launch();
    k_smoother_coefs<<<1, 1, 0, s>>>(nrm2, steps, cheb ? 1 : 0, h->desc.cheb_ratio, h->desc.omega, L.coef,
                                     mixed ? L.coef32 : nullptr);
  }
}

}  // namespace tobk
