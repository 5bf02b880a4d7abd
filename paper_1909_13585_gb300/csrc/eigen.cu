// Block eigensolver for the buckling pencil (K + lambda G) phi = 0 on one level of the hierarchy
// (paper eq. eigenvalueProblem0 on Omega_1, eq. eigenvalueProblemCoarseScale on Omega_l).
//
// With mu = 1/lambda the pencil reads -G phi = mu K phi: the q lowest positive lambda are the q
// largest positive mu of the operator T = K^{-1}(-G), which is self-adjoint in the K inner product.
// The paper solves this problem with Krylov-Schur to a residual of 1e-8 (Appendix A).  Here a
// block Krylov/Davidson iteration with explicit Rayleigh-Ritz is used: the basis V is kept
// K-orthonormal, each outer step appends T applied to the unconverged Ritz vectors (one multi-RHS
// mgPCG solve on the sub-hierarchy below the level), and the projected pencil (V^T(-G)V, V^T K V)
// is solved densely in a single thread block.  Convergence: ||(K + lambda G) x|| / ||K x|| <= tol.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "handle.h"

namespace tobk {

// ------------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Start block: independent uniform(-1, 1) entries from a counter-based hash, zero at fixed DOFs.
__global__ void k_random_block(double* X, int64_t n, int64_t stride, const uint8_t* fixed, uint64_t seed) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = blockIdx.y;
  const uint64_t r = splitmix64(seed ^ ((uint64_t)c * 0x100000001B3ull + (uint64_t)i));
  const double u = (double)(r >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
  X[(int64_t)c * stride + i] = fixed[i] ? 0.0 : u;
}

// H[i][col0 + j] = H[col0 + j][i] = sign * C[i][j]  for i < rows, j < cols
__global__ void k_scatter_sym(const double* C, int rows, int cols, int col0, double sign, double* H, int ld) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const int i = t / cols, j = t % cols;
  const double v = sign * C[t];
  H[(size_t)i * ld + col0 + j] = v;
  H[(size_t)(col0 + j) * ld + i] = v;
}

// Cholesky M = R^T R of a small SPD matrix (k <= 32) and Rinv = R^{-1} (upper triangular).
// info[0] = 0 on success, 1 when a pivot is not positive.
__global__ void k_small_cholinv(const double* M, int k, double* Rinv, double* info) {
  __shared__ double L[32 * 32];
  __shared__ double Li[32 * 32];
  __shared__ int bad;
  const int t = threadIdx.x;
  if (t == 0) bad = 0;
  for (int q = t; q < k * k; q += blockDim.x) {
    L[q] = M[q];
    Li[q] = 0.0;
  }
  __syncthreads();
  // lower Cholesky L L^T = M (so R = L^T)
  for (int j = 0; j < k; ++j) {
    if (t == 0) {
      double d = L[j * k + j];
      for (int p = 0; p < j; ++p) d -= L[j * k + p] * L[j * k + p];
      if (!(d > 0.0)) {
        bad = 1;
        d = 1e-300;
      }
      L[j * k + j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + t; i < k; i += blockDim.x) {
      double s = L[i * k + j];
      for (int p = 0; p < j; ++p) s -= L[i * k + p] * L[j * k + p];
      L[i * k + j] = s / L[j * k + j];
    }
    __syncthreads();
  }
  // Linv (lower) by forward substitution, one column per thread
  for (int c = t; c < k; c += blockDim.x) {
    for (int i = 0; i < k; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int p = c; p < i; ++p) s -= L[i * k + p] * Li[p * k + c];
      Li[i * k + c] = (i < c) ? 0.0 : s / L[i * k + i];
    }
  }
  __syncthreads();
  // Rinv = (L^T)^{-1} = (Linv)^T
  for (int q = t; q < k * k; q += blockDim.x) {
    const int i = q / k, j = q % k;
    Rinv[q] = Li[j * k + i];
  }
  if (t == 0) info[0] = bad ? 1.0 : 0.0;
}

// Dense Rayleigh-Ritz of the projected pencil: H y = theta B y, B SPD, size m <= 64.
// Output: theta descending, Y (ld = ldy) with Y^T B Y = I.  One thread block, FP64.
constexpr int kRRMax = 64;

__global__ void __launch_bounds__(512) k_small_rr(const double* H, const double* B, int m, int ld, double* theta,
                                                  double* Y, int ldy, double* info, int max_sweeps) {
  extern __shared__ double sm[];
  double* L = sm;                   // [m*m]  Cholesky factor of B (lower)
  double* Cm = sm + m * m;          // [m*m]  L^{-1} H L^{-T}, then rotated
  double* Vv = sm + 2 * m * m;      // [m*m]  accumulated rotations
  double* rc = sm + 3 * m * m;      // [kRRMax] cosines
  double* rs = rc + kRRMax;         // [kRRMax] sines
  double* red = rs + kRRMax;        // [64] reduction scratch
  __shared__ int s_bad;
  __shared__ double s_off, s_tot;
  const int t = threadIdx.x, nt = blockDim.x;
  if (t == 0) s_bad = 0;
  for (int q = t; q < m * m; q += nt) {
    const int i = q / m, j = q % m;
    L[q] = B[(size_t)i * ld + j];
    Cm[q] = H[(size_t)i * ld + j];
    Vv[q] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (t == 0) {
      double d = L[j * m + j];
      for (int p = 0; p < j; ++p) d -= L[j * m + p] * L[j * m + p];
      if (!(d > 0.0)) {
        s_bad = 1;
        d = 1e-300;
      }
      L[j * m + j] = sqrt(d);
    }
    __syncthreads();
    for (int i = j + 1 + t; i < m; i += nt) {
      double s = L[i * m + j];
      for (int p = 0; p < j; ++p) s -= L[i * m + p] * L[j * m + p];
      L[i * m + j] = s / L[j * m + j];
    }
    __syncthreads();
  }
  // Cm <- L^{-1} Cm (columns)
  for (int c = t; c < m; c += nt) {
    for (int i = 0; i < m; ++i) {
      double s = Cm[i * m + c];
      for (int p = 0; p < i; ++p) s -= L[i * m + p] * Cm[p * m + c];
      Cm[i * m + c] = s / L[i * m + i];
    }
  }
  __syncthreads();
  // Cm <- Cm L^{-T} (rows)
  for (int r = t; r < m; r += nt) {
    for (int i = 0; i < m; ++i) {
      double s = Cm[r * m + i];
      for (int p = 0; p < i; ++p) s -= Cm[r * m + p] * L[i * m + p];
      Cm[r * m + i] = s / L[i * m + i];
    }
  }
  __syncthreads();
  for (int q = t; q < m * m; q += nt) {
    const int i = q / m, j = q % m;
    if (i < j) {
      const double a = 0.5 * (Cm[i * m + j] + Cm[j * m + i]);
      Cm[i * m + j] = a;
      Cm[j * m + i] = a;
    }
  }
  __syncthreads();
  // parallel cyclic Jacobi with a round-robin pairing (mp players, mp even)
  const int mp = (m + 1) & ~1;
  int sweeps = 0;
  for (; sweeps < max_sweeps; ++sweeps) {
    double off = 0.0, tot = 0.0;
    for (int q = t; q < m * m; q += nt) {
      const double v = Cm[q] * Cm[q];
      tot += v;
      if (q / m != q % m) off += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if ((t & 31) == 0) {
      red[(t >> 5) * 2] = off;
      red[(t >> 5) * 2 + 1] = tot;
    }
    __syncthreads();
    if (t == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) {
        a += red[2 * w];
        b += red[2 * w + 1];
      }
      s_off = a;
      s_tot = b;
    }
    __syncthreads();
    if (!(s_off > 1e-30 * s_tot)) break;
    for (int round = 0; round < mp - 1; ++round) {
      for (int pr = t; pr < mp / 2; pr += nt) {
        int p, q;
        if (pr == 0) {
          p = mp - 1;
          q = round;
        } else {
          p = (round + pr) % (mp - 1);
          q = (round - pr + (mp - 1)) % (mp - 1);
        }
        double c = 1.0, s = 0.0;
        if (p < m && q < m) {
          const double apq = Cm[p * m + q];
          if (apq != 0.0) {
            const double tau = (Cm[q * m + q] - Cm[p * m + p]) / (2.0 * apq);
            const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + tt * tt);
            s = tt * c;
          }
        }
        rc[pr] = c;
        rs[pr] = s;
      }
      __syncthreads();
      // rows p, q
      for (int w = t; w < (mp / 2) * m; w += nt) {
        const int pr = w / m, k = w % m;
        int p, q;
        if (pr == 0) {
          p = mp - 1;
          q = round;
        } else {
          p = (round + pr) % (mp - 1);
          q = (round - pr + (mp - 1)) % (mp - 1);
        }
        if (p >= m || q >= m) continue;
        const double c = rc[pr], s = rs[pr];
        const double xp = Cm[p * m + k], xq = Cm[q * m + k];
        Cm[p * m + k] = c * xp - s * xq;
        Cm[q * m + k] = s * xp + c * xq;
      }
      __syncthreads();
      // columns p, q (and the eigenvector accumulation)
      for (int w = t; w < (mp / 2) * m; w += nt) {
        const int pr = w / m, k = w % m;
        int p, q;
        if (pr == 0) {
          p = mp - 1;
          q = round;
        } else {
          p = (round + pr) % (mp - 1);
          q = (round - pr + (mp - 1)) % (mp - 1);
        }
        if (p >= m || q >= m) continue;
        const double c = rc[pr], s = rs[pr];
        const double xp = Cm[k * m + p], xq = Cm[k * m + q];
        Cm[k * m + p] = c * xp - s * xq;
        Cm[k * m + q] = s * xp + c * xq;
        const double vp = Vv[k * m + p], vq = Vv[k * m + q];
        Vv[k * m + p] = c * vp - s * vq;
        Vv[k * m + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  // back-transform Y = L^{-T} V (columns)
  for (int c = t; c < m; c += nt) {
    for (int i = m - 1; i >= 0; --i) {
      double s = Vv[i * m + c];
      for (int p = i + 1; p < m; ++p) s -= L[p * m + i] * Vv[p * m + c];
      Vv[i * m + c] = s / L[i * m + i];
    }
  }
  __syncthreads();
  // sort descending by theta (selection by rank; ties broken by index)
  for (int c = t; c < m; c += nt) {
    const double tc = Cm[c * m + c];
    int rank = 0;
    for (int o = 0; o < m; ++o) {
      const double to = Cm[o * m + o];
      if (to > tc || (to == tc && o < c)) ++rank;
    }
    theta[rank] = tc;
    for (int i = 0; i < m; ++i) Y[(size_t)i * ldy + rank] = Vv[i * m + c];
  }
  if (t == 0) {
    info[0] = s_bad ? 1.0 : 0.0;
    info[1] = (double)sweeps;
  }
}

// Column-wise dot products out[i] = sum_k A_i[k] B_i[k] (two stage, deterministic).
constexpr int kColChunk = 2048;
__global__ void k_coldots_partial(const double* A, const double* B, int64_t n, int64_t stride, double* partial) {
  __shared__ double red[32];
  const int col = blockIdx.y;
  const int64_t k0 = (int64_t)blockIdx.x * kColChunk;
  double s = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < n && k < k0 + kColChunk; k += blockDim.x)
    s += A[(int64_t)col * stride + k] * B[(int64_t)col * stride + k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
    partial[(size_t)col * gridDim.x + blockIdx.x] = a;
  }
}
__global__ void k_coldots_final(const double* partial, int chunks, int ncols, double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double s = 0.0;
  for (int b = 0; b < chunks; ++b) s += partial[(size_t)c * chunks + b];
  out[c] = s;
}

void launch_coldots(const double* A, const double* B, int ncols, int64_t n, int64_t stride, double* out,
                    double* partial, cudaStream_t s) {
  const int chunks = (int)((n + kColChunk - 1) / kColChunk);
  ::tobk::note_launch(), k_coldots_partial<<<dim3(chunks, ncols), 256, 0, s>>>(A, B, n, stride, partial);
  ::tobk::note_launch(), k_coldots_final<<<(ncols + 63) / 64, 64, 0, s>>>(partial, chunks, ncols, out);
}

// R_i = KX_i + (1/theta_i) GX_i written to R (i < q)
__global__ void k_eig_residual_vec(const double* KX, const double* GX, const double* theta, double* R, int64_t n,
                                   int64_t stride) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = blockIdx.y;
  const double th = theta[i];
  const double lam = th != 0.0 ? 1.0 / th : 0.0;
  R[(int64_t)i * stride + k] = KX[(int64_t)i * stride + k] + lam * GX[(int64_t)i * stride + k];
}

// W_c = -GX_{sel[c]}
__global__ void k_gather_neg(const double* GX, const int* sel, int nsel, double* W, int64_t n, int64_t stride) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int c = blockIdx.y;
  W[(int64_t)c * stride + k] = -GX[(int64_t)sel[c] * stride + k];
}

// ------------------------------------------------------------------------------------------------
// driver
// ------------------------------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int eigen_solve(tobk_handle* h, int j, int q, double* out_modes, double* out_lam_host, tobk_solve_info* info) {
  cudaStream_t st = h->stream;
  const int64_t n = h->lv[j].g.n;
  const int64_t sd = n;
  const int nb = h->eig_nb, mmax = h->eig_mmax;
  const double tol = h->desc.eig_tol;
  double* X = h->EW;
  double* KX = h->EW + (size_t)nb * n;
  double* GX = h->EW + (size_t)2 * nb * n;
  double* W = h->EW + (size_t)3 * nb * n;
  double* KW = h->EKW;
  double* Tb = h->EKW + (size_t)nb * n;
  double* GW = h->EGW;
  double* theta = h->dscal;          // [mmax]
  double* resn = h->dscal + 128;     // [q]  ||r_i||^2
  double* kxn = h->dscal + 256;      // [q]  ||K x_i||^2
  double* sinfo = h->dscal + 384;    // small-kernel status
  int* dsel = (int*)(h->dscal + 512);
  double* Cs = h->Cs;
  double* M = h->Cs + (size_t)mmax * nb;  // nb x nb block Gram
  double* Rinv = M + (size_t)nb * nb;
  const size_t rr_smem = sizeof(double) * (3 * (size_t)kRRMax * kRRMax + 2 * kRRMax + 64);
  static bool rr_configured = false;
  if (!rr_configured) {
    cudaFuncSetAttribute(k_small_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rr_smem);
    rr_configured = true;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);

  ::tobk::note_launch(), k_random_block<<<dim3(nblk(n), nb), 256, 0, st>>>(W, n, sd, h->lv[j].fixed, 0x5EEDull + 977ull * j);
  int nadd = nb, m = 0, it = 0, inner_total = 0;
  bool converged = false;
  double worst = INFINITY;
  std::vector<double> hth(mmax), hres(q), hkx(q);
  int rc = TOBK_OK;
  for (it = 0; it < h->desc.eig_max_iter; ++it) {
    // ---- K-orthogonalise the new block against the basis (classical Gram-Schmidt, twice)
    for (int pass = 0; pass < 2 && m > 0; ++pass) {
      launch_gram(h->KV, m, W, nadd, n, sd, Cs, h->gram_partial, st);
      launch_combine(h->V, m, Cs, nadd, nadd, -1.0, 1.0, W, n, sd, st);
    }
    // ---- K-orthonormalise within the block (Cholesky QR, twice)
    for (int pass = 0; pass < 2; ++pass) {
      apply_K_level(h, j, W, KW, nadd, sd);
      launch_gram(W, nadd, KW, nadd, n, sd, M, h->gram_partial, st);
      ::tobk::note_launch(), k_small_cholinv<<<1, 256, 0, st>>>(M, nadd, Rinv, sinfo);
      launch_combine(W, nadd, Rinv, nadd, nadd, 1.0, 0.0, Tb, n, sd, st);
      cudaMemcpyAsync(W, Tb, sizeof(double) * nadd * n, cudaMemcpyDeviceToDevice, st);
    }
    apply_K_level(h, j, W, KW, nadd, sd);
    apply_G_level(h, j, W, GW, nadd, sd);
    // ---- append to the basis
    cudaMemcpyAsync(h->V + (size_t)m * n, W, sizeof(double) * nadd * n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(h->KV + (size_t)m * n, KW, sizeof(double) * nadd * n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(h->GV + (size_t)m * n, GW, sizeof(double) * nadd * n, cudaMemcpyDeviceToDevice, st);
    const int mn = m + nadd;
    launch_gram(h->V, mn, GW, nadd, n, sd, Cs, h->gram_partial, st);
    ::tobk::note_launch(), k_scatter_sym<<<nblk((int64_t)mn * nadd), 256, 0, st>>>(Cs, mn, nadd, m, -1.0, h->Hs, mmax);
    launch_gram(h->V, mn, KW, nadd, n, sd, Cs, h->gram_partial, st);
    ::tobk::note_launch(), k_scatter_sym<<<nblk((int64_t)mn * nadd), 256, 0, st>>>(Cs, mn, nadd, m, 1.0, h->Bs, mmax);
    m = mn;
    // ---- Rayleigh-Ritz
    ::tobk::note_launch(), k_small_rr<<<1, 512, rr_smem, st>>>(h->Hs, h->Bs, m, mmax, theta, h->Ys, mmax, sinfo + 2, 40);
    const int kk = std::min(nb, m);
    launch_combine(h->V, m, h->Ys, mmax, kk, 1.0, 0.0, X, n, sd, st);
    launch_combine(h->KV, m, h->Ys, mmax, kk, 1.0, 0.0, KX, n, sd, st);
    launch_combine(h->GV, m, h->Ys, mmax, kk, 1.0, 0.0, GX, n, sd, st);
    ::tobk::note_launch(), k_eig_residual_vec<<<dim3(nblk(n), q), 256, 0, st>>>(KX, GX, theta, Tb, n, sd);
    launch_coldots(Tb, Tb, q, n, sd, resn, h->gram_partial, st);
    launch_coldots(KX, KX, q, n, sd, kxn, h->gram_partial, st);
    cudaMemcpyAsync(h->hscal, h->dscal, sizeof(double) * 512, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    rc = check_cuda(h, "eigen_solve");
    if (rc) break;
    for (int i = 0; i < kk; ++i) hth[i] = h->hscal[i];
    worst = 0.0;
    std::vector<int> sel;
    for (int i = 0; i < kk; ++i) {
      bool ok = false;
      if (i < q) {
        const double res = std::sqrt(h->hscal[128 + i] / std::max(h->hscal[256 + i], 1e-300));
        ok = hth[i] > 0.0 && res <= tol;
        worst = std::max(worst, hth[i] > 0.0 ? res : INFINITY);
      }
      if (!ok) sel.push_back(i);
    }
    converged = true;
    for (int i = 0; i < q; ++i) {
      const double res = std::sqrt(h->hscal[128 + i] / std::max(h->hscal[256 + i], 1e-300));
      if (!(hth[i] > 0.0 && res <= tol)) converged = false;
    }
    if (converged) break;
    // ---- expansion block W = T X_sel = K^{-1} (-G X_sel)
    nadd = (int)sel.size();
    cudaMemcpyAsync(dsel, sel.data(), sizeof(int) * nadd, cudaMemcpyHostToDevice, st);
    ::tobk::note_launch(), k_gather_neg<<<dim3(nblk(n), nadd), 256, 0, st>>>(GX, dsel, nadd, Tb, n, sd);
    tobk_solve_info si{};
    int src = pcg_solve(h, j, Tb, W, nadd, 1e-10, h->desc.max_iter, false, TOBK_FP64, &si);
    inner_total += si.iterations;
    if (src && src != TOBK_E_NOT_CONVERGED) {
      rc = src;
      break;
    }
    // ---- thick restart: keep the kk Ritz vectors
    if (m + nadd > mmax) {
      cudaMemcpyAsync(h->V, X, sizeof(double) * kk * n, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(h->KV, KX, sizeof(double) * kk * n, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(h->GV, GX, sizeof(double) * kk * n, cudaMemcpyDeviceToDevice, st);
      launch_gram(h->V, kk, h->GV, kk, n, sd, Cs, h->gram_partial, st);
      ::tobk::note_launch(), k_scatter_sym<<<nblk((int64_t)kk * kk), 256, 0, st>>>(Cs, kk, kk, 0, -1.0, h->Hs, mmax);
      launch_gram(h->V, kk, h->KV, kk, n, sd, Cs, h->gram_partial, st);
      ::tobk::note_launch(), k_scatter_sym<<<nblk((int64_t)kk * kk), 256, 0, st>>>(Cs, kk, kk, 0, 1.0, h->Bs, mmax);
      m = kk;
    }
  }
  if (rc == TOBK_OK) {
    // load factors as Rayleigh quotients of the final Ritz vectors: lambda = -x^T K x / x^T G x
    launch_coldots(X, KX, q, n, sd, resn, h->gram_partial, st);
    launch_coldots(X, GX, q, n, sd, kxn, h->gram_partial, st);
    cudaMemcpyAsync(h->hscal, h->dscal, sizeof(double) * 512, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(out_modes, X, sizeof(double) * q * n, cudaMemcpyDeviceToDevice, st);
    cudaStreamSynchronize(st);
    for (int i = 0; i < q; ++i) out_lam_host[i] = -h->hscal[128 + i] / h->hscal[256 + i];
    rc = check_cuda(h, "eigen_solve");
  }
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    info->iterations = it + 1;
    info->converged = converged ? 1 : 0;
    info->num_rhs = q;
    info->rel_residual = worst;
    info->time_ms = ms;
    info->status_detail = inner_total;
  }
  if (rc == TOBK_OK && !converged) rc = fail(h, TOBK_E_NOT_CONVERGED, "eigensolver did not reach eig_tol");
  return rc;
}

}  // namespace tobk
