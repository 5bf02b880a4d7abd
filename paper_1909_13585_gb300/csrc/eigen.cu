// Block eigensolver for the buckling pencil (K + lambda G) phi = 0 on one level of the hierarchy
// (paper eq. eigenvalueProblem0 on Omega_1, eq. eigenvalueProblemCoarseScale on Omega_l).
//
// With mu = 1/lambda the pencil reads -G phi = mu K phi: the q lowest positive lambda are the q
// largest positive mu of the operator T = K^{-1}(-G), which is self-adjoint in the K inner product.
// The paper solves this problem with Krylov-Schur to a residual of 1e-8 (Appendix A).  Here a
// block generalised-Davidson iteration with explicit Rayleigh-Ritz is used: the basis V is kept
// K-orthonormal, each outer step appends the multigrid-preconditioned residuals
// M(-G x_i - theta_i K x_i) of the unconverged Ritz pairs (one V-cycle for all of them, on the
// sub-hierarchy below the level), and the projected problem V^T(-G)V is solved densely in a single
// thread block.  Convergence: ||(K + lambda G) x|| / ||K x|| <= tol for the q wanted pairs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "handle.h"
#include "small_dense.cuh"

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

// H[i][col0 + j] = H[col0 + j][i] = sign * C[i][j]  for i < rows, j < cols.  Inside the square block
// i >= col0 both C[i][j] and C[col0 + j][i - col0] name the same pair; the one with i <= col0 + j is
// used, so that H is exactly symmetric and every entry has a single writer.
__global__ void k_scatter_sym(const double* C, int rows, int cols, int col0, double sign, double* H, int ld) {
  pdl_wait();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const int i = t / cols, j = t % cols;
  if (i >= col0 && i > col0 + j) return;
  const double v = sign * C[t];
  H[(size_t)i * ld + col0 + j] = v;
  H[(size_t)(col0 + j) * ld + i] = v;
}

// Cholesky M = R^T R of a small SPD matrix (k <= 32) and Rinv = R^{-1} (upper triangular), by one
// warp.  Lower factor L = R^T, right-looking: at pivot j one rsqrt of the updated diagonal gives both
// L_jj = d rsqrt(d) and 1 / L_jj, lane i > j scales its entry of column j and updates its row of the
// trailing block (independent multiply-adds, no dependent dot-product chain).  The inverse Linv is
// formed by forward substitution with lane c owning column c (rows updated right-looking, so a lane
// never waits for another).  A chain of FP64 operations on one SM is latency-bound; this keeps it at
// about 2k dependent steps.  info[0] is set to 1 when a pivot is not positive (left unchanged
// otherwise).
__global__ void __launch_bounds__(32) k_small_cholinv(const double* M, int k, double* Rinv, double* info) {
  pdl_wait();
  __shared__ double A[32][33];   // lower triangle of M, overwritten by L
  __shared__ double B[32][33];   // B[r][c]: Linv, column c in lane c
  __shared__ double dinv[32];
  const int t = threadIdx.x;
  if (t < k)
    for (int l = 0; l <= t; ++l) A[t][l] = M[t * k + l];
  __syncwarp();
  bool bad = false;
  for (int j = 0; j < k; ++j) {
    double d = A[j][j];
    if (!(d > 0.0)) {
      bad = true;
      d = 1e-300;
    }
    const double r = rsqrt(d);
    double lij = 0.0;
    if (t > j && t < k) lij = A[t][j] * r;
    __syncwarp();
    if (t > j && t < k) A[t][j] = lij;
    if (t == j) {
      A[j][j] = d * r;
      dinv[j] = r;
    }
    __syncwarp();
    if (t > j && t < k)
      for (int l = j + 1; l <= t; ++l) A[t][l] -= lij * A[l][j];
    __syncwarp();
  }
  if (t < k) {
    for (int r = 0; r < k; ++r) B[r][t] = r == t ? 1.0 : 0.0;
    for (int i = t; i < k; ++i) {  // rows above t stay 0
      const double li = B[i][t] * dinv[i];
      B[i][t] = li;
      for (int r = i + 1; r < k; ++r) B[r][t] -= A[r][i] * li;
    }
  }
  __syncwarp();
  // Rinv = (L^T)^{-1} = (Linv)^T
  for (int q = t; q < k * k; q += 32) {
    const int i = q / k, j = q % k;
    Rinv[q] = B[j][i];
  }
  if (t == 0 && bad) info[0] = 1.0;
}

// Column-wise dot products out[i] = sum_k A_i[k] B_i[k] (two stage, deterministic).
constexpr int kColChunk = 2048;
__global__ void k_coldots_partial(const double* A, const double* B, int64_t n, int64_t stride, double* partial) {
  pdl_wait();
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
  pdl_wait();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double s = 0.0;
  for (int b = 0; b < chunks; ++b) s += partial[(size_t)c * chunks + b];
  out[c] = s;
}

void launch_coldots(const double* A, const double* B, int ncols, int64_t n, int64_t stride, double* out,
                    double* partial, cudaStream_t s) {
  const int chunks = (int)((n + kColChunk - 1) / kColChunk);
  launch_pdl(k_coldots_partial, dim3(dim3(chunks, ncols)), dim3(256), 0, s, A, B, n, stride, partial);
  launch_pdl(k_coldots_final, dim3((ncols + 63) / 64), dim3(64), 0, s, partial, chunks, ncols, out);
}

// Squared norms of the pencil residuals and of K x for the Ritz pairs i < ncols (two stages,
// deterministic): resn[i] = ||KX_i + (1/theta_i) GX_i||^2, kxn[i] = ||KX_i||^2.
__global__ void k_resnorm_partial(const double* KX, const double* GX, const double* theta, int64_t n, int64_t stride,
                                  double* partial) {
  pdl_wait();
  __shared__ double red[2][32];
  const int col = blockIdx.y;
  const double th = theta[col];
  const double lam = th != 0.0 ? 1.0 / th : 0.0;
  const int64_t k0 = (int64_t)blockIdx.x * kColChunk;
  double sr = 0.0, sk = 0.0;
  for (int64_t k = k0 + threadIdx.x; k < n && k < k0 + kColChunk; k += blockDim.x) {
    const double kx = KX[(int64_t)col * stride + k];
    const double r = kx + lam * GX[(int64_t)col * stride + k];
    sr += r * r;
    sk += kx * kx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    sk += __shfl_xor_sync(0xffffffffu, sk, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sr;
    red[1][threadIdx.x >> 5] = sk;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    partial[2 * ((size_t)col * gridDim.x + blockIdx.x)] = a;
    partial[2 * ((size_t)col * gridDim.x + blockIdx.x) + 1] = b;
  }
}
__global__ void k_resnorm_final(const double* partial, int chunks, int ncols, double* resn, double* kxn) {
  pdl_wait();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double a = 0.0, b = 0.0;
  for (int k = 0; k < chunks; ++k) {
    a += partial[2 * ((size_t)c * chunks + k)];
    b += partial[2 * ((size_t)c * chunks + k) + 1];
  }
  resn[c] = a;
  kxn[c] = b;
}

static void launch_resnorms(const double* KX, const double* GX, const double* theta, int ncols, int64_t n,
                            int64_t stride, double* resn, double* kxn, double* partial, cudaStream_t s) {
  const int chunks = (int)((n + kColChunk - 1) / kColChunk);
  launch_pdl(k_resnorm_partial, dim3(dim3(chunks, ncols)), dim3(256), 0, s, KX, GX, theta, n, stride, partial);
  launch_pdl(k_resnorm_final, dim3((ncols + 63) / 64), dim3(64), 0, s, partial, chunks, ncols, resn, kxn);
}

// W_c = -GX_{s} - theta_s KX_{s}, s = sel[c]: the residual of the pencil -G x = mu K x at the Ritz
// pair (theta_s, x_s)
__global__ void k_gather_residual(const double* GX, const double* KX, const double* theta, const int* sel,
                                  double* W, int64_t n, int64_t stride) {
  pdl_wait();
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int c = blockIdx.y;
  const int s = sel[c];
  W[(int64_t)c * stride + k] = -GX[(int64_t)s * stride + k] - theta[s] * KX[(int64_t)s * stride + k];
}

// Gram product of the eigensolver: tensor cores (FP64-accurate splitting, gram_tc.cu) for vectors of
// the eigen level, FP64 CUDA cores otherwise.
static void eig_gram(tobk_handle* h, const double* A, int na, const double* B, int nb, int64_t n, int64_t stride,
                     double* C) {
  if (h->gtc_err && na <= 64 && nb <= 64 && n <= h->gtc_nmax)
    launch_gram_tc(A, na, B, nb, n, stride, C, h->gram_partial, h->gtc_err, h->stream);
  else
    launch_gram(A, na, B, nb, n, stride, C, h->gram_partial, h->stream);
}

// TOBK_OK, or the status of a failed tensor-core Gram product (flags copied to the host at byte offset
// 8000 of hscal by the last synchronised step)
static int gram_tc_status(tobk_handle* h) {
  if (!h->gtc_err) return TOBK_OK;
  unsigned f[2];
  std::memcpy(f, reinterpret_cast<const char*>(h->hscal) + 8000, sizeof(f));
  if (f[0]) return fail(h, TOBK_E_TIMEOUT, "tensor-core Gram product: a bounded wait gave up");
  if (f[1]) return fail(h, TOBK_E_NONFINITE, "non-finite value in the eigensolver basis");
  return TOBK_OK;
}

// ------------------------------------------------------------------------------------------------
// driver
// ------------------------------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

int eigen_solve(tobk_handle* h, int j, int q, double* out_modes, double* out_lam_host, tobk_solve_info* info,
                EigenHook* hook) {
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
  double* theta = h->dscal;          // [mmax]
  double* resn = h->dscal + 128;     // [q]  ||r_i||^2
  double* kxn = h->dscal + 256;      // [q]  ||K x_i||^2
  double* sinfo = h->dscal + 384;    // small-kernel status
  int* dsel = (int*)(h->dscal + 512);
  double* Cs = h->Cs;
  double* M = h->Cs + (size_t)mmax * nb;  // nb x nb block Gram
  double* Rinv = M + (size_t)nb * nb;
  static bool rr_configured = false;
  if (!rr_configured) {
    cudaFuncSetAttribute(k_rr_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)rr_finish_smem_bytes(kRRMax, kRRMax));
    rr_configured = true;
  }
  const int keep_max = std::min(2 * nb, mmax - nb);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);

  ::tobk::note_launch(), k_random_block<<<dim3(nblk(n), nb), 256, 0, st>>>(W, n, sd, h->lv[j].fixed, 0x5EEDull + 977ull * j);
  int nadd = nb, m = 0, it = 0, inner_total = 0;
  bool converged = false;
  double worst = INFINITY;
  std::vector<double> hth(mmax);
  // Rayleigh-Ritz scratch: FP32-stage eigenvectors, refined eigenvectors, S, R, wanted columns
  double* rrX0 = h->tri;
  double* rrX1 = rrX0 + (size_t)mmax * mmax;
  double* rrS = rrX1 + (size_t)mmax * mmax;
  double* rrR = rrS + (size_t)mmax * mmax;
  double* rrXw = rrR + (size_t)mmax * mmax;
  double* rrLam = rrXw + (size_t)mmax * mmax;
  double* rrDelta = rrLam + mmax;
  int rr_prev = 0;  // size of the previous projected problem whose eigenvectors are in rrX1 (0: none)
  cudaMemsetAsync(sinfo, 0, sizeof(double), st);  // Cholesky breakdown flag (sticky)
  if (h->gtc_err) cudaMemsetAsync(h->gtc_err, 0, 2 * sizeof(unsigned), st);
  const bool trace = std::getenv("TOBK_EIG_TRACE") != nullptr;
  int rc = TOBK_OK;
  PhaseMarks pm(h);
  std::vector<std::pair<int, int>> pre_marks, rr_marks;
  for (it = 0; it < h->desc.eig_max_iter; ++it) {
    // ---- K-orthogonalise the new block against the basis (classical Gram-Schmidt, twice)
    prof_begin(h, TOBK_KC_EIGEN_BLOCK, (double)nadd * n);
    for (int pass = 0; pass < 2 && m > 0; ++pass) {
      eig_gram(h, h->KV, m, W, nadd, n, sd, Cs);
      launch_combine(h->V, m, Cs, nadd, nadd, -1.0, 1.0, W, n, sd, st);
    }
    prof_end(h);
    // ---- K-orthonormalise within the block (Cholesky QR, twice: W -> Tb -> the basis columns
    // m .. m + nadd - 1, which the block's K and G images join)
    double* Vn = h->V + (size_t)m * n;
    double* KVn = h->KV + (size_t)m * n;
    double* GVn = h->GV + (size_t)m * n;
    for (int pass = 0; pass < 2; ++pass) {
      const double* src = pass == 0 ? W : Tb;
      double* dst = pass == 0 ? Tb : Vn;
      apply_K_level(h, j, src, KW, nadd, sd);
      prof_begin(h, TOBK_KC_EIGEN_BLOCK, (double)nadd * n);
      eig_gram(h, src, nadd, KW, nadd, n, sd, M);
      prof_end(h);
      prof_begin(h, TOBK_KC_EIGEN_DENSE, (double)nadd);
      launch_pdl(k_small_cholinv, dim3(1), dim3(32), 0, st, M, nadd, Rinv, sinfo);
      prof_end(h);
      prof_begin(h, TOBK_KC_EIGEN_BLOCK, (double)nadd * n);
      launch_combine(src, nadd, Rinv, nadd, nadd, 1.0, 0.0, dst, n, sd, st);
      prof_end(h);
    }
    apply_K_level(h, j, Vn, KVn, nadd, sd);
    apply_G_level(h, j, Vn, GVn, nadd, sd);
    const int mn = m + nadd;
    prof_begin(h, TOBK_KC_EIGEN_BLOCK, (double)mn * n);
    eig_gram(h, h->V, mn, GVn, nadd, n, sd, Cs);
    launch_pdl(k_scatter_sym, dim3(nblk((int64_t)mn * nadd)), dim3(256), 0, st, Cs, mn, nadd, m, -1.0, h->Hs, mmax);
    prof_end(h);
    m = mn;
    // ---- Rayleigh-Ritz (the basis is K-orthonormal, so V^T K V = I): the leading eigenpairs of
    // the projected matrix, FP32 decomposition + two FP64 refinement steps (small_dense.cuh)
    const int nvec = std::min(m, keep_max);
    const int rr0 = pm.mark();
    prof_begin(h, TOBK_KC_EIGEN_DENSE, (double)m);
    // warm start from the previous refined eigenvectors while the basis only grew since then
    launch_rr_eig32(h->Hs, m, mmax, rrX1, rr_prev, rrX0, sinfo + 2, st);
    // refinement: X0 -> X1 -> X0 ... (the last step writes the nvec wanted columns to Xw); the error
    // bound of the FP32 result decides the clusters of every step and of the finish
    for (int step = 0; step < kRRRefineSteps; ++step) {
      const bool last = step == kRRRefineSteps - 1;
      double* xin = (step & 1) ? rrX1 : rrX0;
      double* xout = last ? rrXw : ((step & 1) ? rrX0 : rrX1);
      launch_pdl(k_rr_oa_products, dim3(m), dim3(kOAThreads), 0, st, h->Hs, mmax, xin, m, rrS, rrR);
      launch_pdl(k_rr_oa_update, dim3(last ? nvec : m), dim3(kOAThreads), 0, st, xin, rrS, rrR, m, xout, last ? mmax : m,
                                                                           last ? rrLam : nullptr, rrDelta, step == 0);
    }
    launch_pdl(k_rr_finish, dim3(1), dim3(256), rr_finish_smem_bytes(m, nvec), st, 
        h->Hs, mmax, m, nvec, rrXw, mmax, rrLam, rrDelta, theta, h->Ys, mmax);
    prof_end(h);
    rr_marks.emplace_back(rr0, pm.mark());
    rr_prev = m;
    const int kk = std::min(nb, m);
    prof_begin(h, TOBK_KC_EIGEN_BLOCK, (double)m * n);
    launch_combine3(h->V, h->KV, h->GV, m, h->Ys, mmax, kk, X, KX, GX, n, sd, st);
    launch_resnorms(KX, GX, theta, q, n, sd, resn, kxn, h->gram_partial, st);
    prof_end(h);
    cudaMemcpyAsync(h->hscal, h->dscal, sizeof(double) * 512, cudaMemcpyDeviceToHost, st);
    if (h->gtc_err)
      cudaMemcpyAsync(reinterpret_cast<char*>(h->hscal) + 8000, h->gtc_err, 2 * sizeof(unsigned),
                      cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    rc = check_cuda(h, "eigen_solve");
    if (rc) break;
    rc = gram_tc_status(h);
    if (rc) break;
    if (h->hscal[384] != 0.0) {  // the K-orthonormalised expansion lost rank
      rc = fail(h, TOBK_E_BREAKDOWN,
                "eigensolver basis lost rank (the level has fewer free DOFs than the block of q vectors needs)");
      break;
    }
    for (int i = 0; i < kk; ++i) hth[i] = h->hscal[i];
    if (trace)
      std::fprintf(stderr, "[tobk eig] level %d it %d m %d nadd %d theta0 %.9e thetaq %.9e fp32 sweeps %g\n", j, it, m,
                   nadd, hth[0], hth[std::min(q, kk) - 1], h->hscal[386]);
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
    if (trace) std::fprintf(stderr, "[tobk eig]   worst residual %.3e, unconverged %d\n", worst, (int)sel.size());
    converged = true;
    bool conv[64];
    for (int i = 0; i < q; ++i) {
      const double res = std::sqrt(h->hscal[128 + i] / std::max(h->hscal[256 + i], 1e-300));
      conv[i] = hth[i] > 0.0 && res <= tol;
      if (!conv[i]) converged = false;
    }
    if (converged) break;
    if (hook) hook->iteration(X, n, hth.data(), conv, q);
    // ---- expansion block (generalised Davidson): W = M r_s, r_s = -G x_s - theta_s K x_s for the
    // selected Ritz pairs, M = one multigrid V-cycle for K on this level and below
    nadd = (int)sel.size();
    cudaMemcpyAsync(dsel, sel.data(), sizeof(int) * nadd, cudaMemcpyHostToDevice, st);
    launch_pdl(k_gather_residual, dim3(dim3(nblk(n), nadd)), dim3(256), 0, st, GX, KX, theta, dsel, Tb, n, sd);
    const int pre0 = pm.mark();
    if (h->desc.eig_inner_iters <= 0) {
      apply_vcycle(h, j, nadd, Tb, W);
      ++inner_total;
    } else {
      // a few mgPCG iterations on K w = r (a better approximation of K^{-1} r than one V-cycle;
      // the iteration limit is the point, so "not converged" is the expected status)
      tobk_solve_info si{};
      const int src =
          pcg_solve(h, j, Tb, W, nadd, 1e-300, h->desc.eig_inner_iters, false, h->desc.precision, &si, true);
      if (src && src != TOBK_E_NOT_CONVERGED) {
        rc = src;
        break;
      }
      inner_total += si.status_detail;
    }
    pre_marks.emplace_back(pre0, pm.mark());
    // ---- thick restart: keep the kk Ritz vectors (FP64-accurate, hence K-orthonormal)
    if (m + nadd > mmax) {
      // keep the leading min(2 nb, mmax - nb) Ritz vectors (and their K and G images)
      const int keep = std::min(std::min(2 * nb, mmax - nb), m);
      double* tmp = h->EW + (size_t)4 * nb * n;
      double* bases[3] = {h->V, h->KV, h->GV};
      for (double* bsp : bases) {
        launch_combine(bsp, m, h->Ys, mmax, keep, 1.0, 0.0, tmp, n, sd, st);
        cudaMemcpyAsync(bsp, tmp, sizeof(double) * keep * n, cudaMemcpyDeviceToDevice, st);
      }
      eig_gram(h, h->V, keep, h->GV, keep, n, sd, Cs);
      launch_pdl(k_scatter_sym, dim3(nblk((int64_t)keep * keep)), dim3(256), 0, st, Cs, keep, keep, 0, -1.0, h->Hs,
                                                                                       mmax);
      m = keep;
      rr_prev = 0;  // the basis was replaced by Ritz vectors: its projected matrix is diagonal
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
  if (h->phase_on) {
    double tp = 0.0, tr = 0.0;
    for (auto& pr : pre_marks) tp += pm.ms(pr.first, pr.second);
    for (auto& pr : rr_marks) tr += pm.ms(pr.first, pr.second);
    h->phase_ms[TOBK_PHASE_EIGEN_PRECOND] = tp;
    h->phase_ms[TOBK_PHASE_EIGEN_RR] = tr;
    h->phase_ms[TOBK_PHASE_EIGEN_ITERS] = it + 1;
  }
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

// Rayleigh-Ritz of (K^j, G^j) on span Psi at level j (Algorithm 2, 'R[Psi]'): K-orthonormalise the
// q columns (Cholesky QR, twice), project H = Psi^T (-G) Psi, decompose it with the dense
// Rayleigh-Ritz kernels of the eigensolver (FP32 Jacobi + FP64 refinement), rotate Psi onto the
// Ritz vectors.  Scratch: the level's V-cycle vectors z, t, r (each [rmax][n_j], rmax >= q).
int ritz_level(tobk_handle* h, int j, int q, double* Psi, double* lam_host) {
  cudaStream_t st = h->stream;
  const int64_t n = h->lv[j].g.n;
  const int nb = h->eig_nb, mmax = h->eig_mmax;
  if (q > nb || q > kRRMax) return fail(h, TOBK_E_ARG, "ritz_level: too many vectors");
  double* KW = h->lv[j].z;
  double* Tb = h->lv[j].t;
  double* GW = h->lv[j].r;
  double* theta = h->dscal;
  double* sinfo = h->dscal + 384;
  double* Cs = h->Cs;
  double* M = h->Cs + (size_t)mmax * nb;
  double* Rinv = M + (size_t)nb * nb;
  double* rrX0 = h->tri;
  double* rrX1 = rrX0 + (size_t)mmax * mmax;
  double* rrS = rrX1 + (size_t)mmax * mmax;
  double* rrR = rrS + (size_t)mmax * mmax;
  double* rrXw = rrR + (size_t)mmax * mmax;
  double* rrLam = rrXw + (size_t)mmax * mmax;
  double* rrDelta = rrLam + mmax;
  cudaFuncSetAttribute(k_rr_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)rr_finish_smem_bytes(kRRMax, kRRMax));
  cudaMemsetAsync(sinfo, 0, sizeof(double), st);
  for (int pass = 0; pass < 2; ++pass) {
    apply_K_level(h, j, Psi, KW, q, n);
    eig_gram(h, Psi, q, KW, q, n, n, M);
    launch_pdl(k_small_cholinv, dim3(1), dim3(32), 0, st, M, q, Rinv, sinfo);
    launch_combine(Psi, q, Rinv, q, q, 1.0, 0.0, Tb, n, n, st);
    cudaMemcpyAsync(Psi, Tb, sizeof(double) * q * n, cudaMemcpyDeviceToDevice, st);
  }
  apply_G_level(h, j, Psi, GW, q, n);
  eig_gram(h, Psi, q, GW, q, n, n, Cs);
  launch_pdl(k_scatter_sym, dim3(nblk((int64_t)q * q)), dim3(256), 0, st, Cs, q, q, 0, -1.0, h->Hs, mmax);
  launch_rr_eig32(h->Hs, q, mmax, nullptr, 0, rrX0, sinfo + 2, st);
  for (int step = 0; step < kRRRefineSteps; ++step) {
    const bool last = step == kRRRefineSteps - 1;
    double* xin = (step & 1) ? rrX1 : rrX0;
    double* xout = last ? rrXw : ((step & 1) ? rrX0 : rrX1);
    launch_pdl(k_rr_oa_products, dim3(q), dim3(kOAThreads), 0, st, h->Hs, mmax, xin, q, rrS, rrR);
    launch_pdl(k_rr_oa_update, dim3(q), dim3(kOAThreads), 0, st, xin, rrS, rrR, q, xout, last ? mmax : q,
                                                            last ? rrLam : nullptr, rrDelta, step == 0);
  }
  launch_pdl(k_rr_finish, dim3(1), dim3(256), rr_finish_smem_bytes(q, q), st, h->Hs, mmax, q, q, rrXw, mmax, rrLam,
                                                                                 rrDelta, theta, h->Ys, mmax);
  launch_combine(Psi, q, h->Ys, mmax, q, 1.0, 0.0, Tb, n, n, st);
  cudaMemcpyAsync(Psi, Tb, sizeof(double) * q * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(h->hscal, h->dscal, sizeof(double) * 512, cudaMemcpyDeviceToHost, st);
  if (h->gtc_err)
    cudaMemcpyAsync(reinterpret_cast<char*>(h->hscal) + 8000, h->gtc_err, 2 * sizeof(unsigned),
                    cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  int rc = check_cuda(h, "ritz_level");
  if (rc) return rc;
  rc = gram_tc_status(h);
  if (rc) return rc;
  if (h->hscal[384] != 0.0) return fail(h, TOBK_E_BREAKDOWN, "Ritz projection: the prolongated modes lost rank");
  for (int i = 0; i < q; ++i) {
    const double th = h->hscal[i];
    if (!(th > 0.0) || !std::isfinite(th))
      return fail(h, TOBK_E_BREAKDOWN, "Ritz projection lost a positive load factor on level " + std::to_string(j + 1));
    lam_host[i] = 1.0 / th;
  }
  return TOBK_OK;
}

}  // namespace tobk
