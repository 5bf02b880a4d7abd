// Dense Rayleigh-Ritz of the projected buckling pencil in one thread block (included by eigen.cu).
//
// The eigensolver keeps its basis K-orthonormal, so the projected problem is the standard
// symmetric eigenproblem H y = theta y with H = V^T (-G) V (size m <= 64).  GB300 executes FP64 at
// 1/64 of its FP32 rate, so the cyclic Jacobi sweeps run in FP32 first (to ~1e-6 relative
// off-diagonal mass); when full accuracy is requested, the FP32 eigenvectors are refined in FP64:
// C = V^T H V (nearly diagonal), followed by FP64 Jacobi sweeps, which converge quadratically from
// there.  Eigenpairs are returned sorted by descending theta.
#pragma once
#include <cuda_runtime.h>

namespace tobk {

constexpr int kRRMax = 64;

// Round-robin pairing of mp (even) indices: round r, pair slot k -> (p, q).
__device__ __forceinline__ void rr_pair(int mp, int round, int k, int& p, int& q) {
  if (k == 0) {
    p = mp - 1;
    q = round;
  } else {
    p = (round + k) % (mp - 1);
    q = (round - k + (mp - 1)) % (mp - 1);
  }
}

// One cyclic Jacobi sweep (all pairs once, m/2 disjoint rotations per round) on C (m x m, row-major)
// with the rotations accumulated into V.  rc/rs: per-pair cosines and sines (T precision).
template <typename T>
__device__ void jacobi_sweep(T* C, T* V, int m, T* rc, T* rs) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int mp = (m + 1) & ~1;
  for (int round = 0; round < mp - 1; ++round) {
    for (int k = t; k < mp / 2; k += nt) {
      int p, q;
      rr_pair(mp, round, k, p, q);
      T c = T(1), s = T(0);
      if (p < m && q < m) {
        const T apq = C[p * m + q];
        if (apq != T(0)) {
          const T tau = (C[q * m + q] - C[p * m + p]) / (T(2) * apq);
          const T tt = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
          c = T(1) / sqrt(T(1) + tt * tt);
          s = tt * c;
        }
      }
      rc[k] = c;
      rs[k] = s;
    }
    __syncthreads();
    for (int w = t; w < (mp / 2) * m; w += nt) {  // rows p, q
      const int k = w / m, col = w % m;
      int p, q;
      rr_pair(mp, round, k, p, q);
      if (p >= m || q >= m || rs[k] == T(0)) continue;
      const T c = rc[k], s = rs[k];
      const T xp = C[p * m + col], xq = C[q * m + col];
      C[p * m + col] = c * xp - s * xq;
      C[q * m + col] = s * xp + c * xq;
    }
    __syncthreads();
    for (int w = t; w < (mp / 2) * m; w += nt) {  // columns p, q and the accumulated rotations
      const int k = w / m, row = w % m;
      int p, q;
      rr_pair(mp, round, k, p, q);
      if (p >= m || q >= m || rs[k] == T(0)) continue;
      const T c = rc[k], s = rs[k];
      const T xp = C[row * m + p], xq = C[row * m + q];
      C[row * m + p] = c * xp - s * xq;
      C[row * m + q] = s * xp + c * xq;
      const T vp = V[row * m + p], vq = V[row * m + q];
      V[row * m + p] = c * vp - s * vq;
      V[row * m + q] = s * vp + c * vq;
    }
    __syncthreads();
  }
}

// off-diagonal and total squared Frobenius mass of C (result valid in all threads)
template <typename T>
__device__ void offdiag_mass(const T* C, int m, double* red, double& off, double& tot) {
  const int t = threadIdx.x, nt = blockDim.x;
  double o = 0.0, a = 0.0;
  for (int q = t; q < m * m; q += nt) {
    const double v = (double)C[q] * (double)C[q];
    a += v;
    if (q / m != q % m) o += v;
  }
  for (int s = 16; s > 0; s >>= 1) {
    o += __shfl_xor_sync(0xffffffffu, o, s);
    a += __shfl_xor_sync(0xffffffffu, a, s);
  }
  __syncthreads();
  if ((t & 31) == 0) {
    red[2 * (t >> 5)] = o;
    red[2 * (t >> 5) + 1] = a;
  }
  __syncthreads();
  o = 0.0;
  a = 0.0;
  for (int w = 0; w < (nt + 31) / 32; ++w) {
    o += red[2 * w];
    a += red[2 * w + 1];
  }
  off = o;
  tot = a;
  __syncthreads();
}

// H: [m][ld] symmetric (only the leading m x m block is read).  full_precision != 0 adds the FP64
// refinement.  Outputs theta[m] (descending) and Y (column i = eigenvector i, ld = ldy);
// info[0] = FP32 sweeps, info[1] = FP64 sweeps.
__global__ void __launch_bounds__(512) k_small_rr(const double* H, int m, int ld, double* theta, double* Y, int ldy,
                                                  double* info, int full_precision) {
  extern __shared__ double sm[];
  double* C64 = sm;                       // [m*m]
  double* V64 = C64 + m * m;              // [m*m]
  double* T64 = V64 + m * m;              // [m*m]
  double* rc64 = T64 + m * m;             // [kRRMax]
  double* rs64 = rc64 + kRRMax;           // [kRRMax]
  double* red = rs64 + kRRMax;            // [64]
  float* C32 = reinterpret_cast<float*>(red + 64);  // [m*m]
  float* V32 = C32 + m * m;                         // [m*m]
  float* rc32 = V32 + m * m;                        // [kRRMax]
  float* rs32 = rc32 + kRRMax;                      // [kRRMax]
  const int t = threadIdx.x, nt = blockDim.x;
  for (int q = t; q < m * m; q += nt) {
    const int i = q / m, j = q % m;
    const double a = 0.5 * (H[(size_t)i * ld + j] + H[(size_t)j * ld + i]);
    C64[q] = a;
    C32[q] = (float)a;
    V32[q] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  double off, tot;
  int s32 = 0, s64 = 0;
  for (; s32 < 30; ++s32) {
    offdiag_mass(C32, m, red, off, tot);
    if (!(off > 1e-11 * tot)) break;
    jacobi_sweep<float>(C32, V32, m, rc32, rs32);
  }
  for (int q = t; q < m * m; q += nt) V64[q] = (double)V32[q];
  __syncthreads();
  if (full_precision) {
    // The FP32 rotations leave V64 orthonormal only to ~1e-7: re-orthonormalise its columns in FP64
    // (classical Gram-Schmidt, column by column; T64 holds the projection coefficients).
    for (int col = 0; col < m; ++col) {
      for (int i = t; i < col; i += nt) {
        double s = 0.0;
        for (int r = 0; r < m; ++r) s += V64[r * m + i] * V64[r * m + col];
        T64[i] = s;
      }
      __syncthreads();
      for (int r = t; r < m; r += nt) {
        double s = V64[r * m + col];
        for (int i = 0; i < col; ++i) s -= T64[i] * V64[r * m + i];
        V64[r * m + col] = s;
      }
      __syncthreads();
      if (t < 32) {
        double s = 0.0;
        for (int r = t; r < m; r += 32) s += V64[r * m + col] * V64[r * m + col];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (t == 0) T64[m] = 1.0 / sqrt(s);
      }
      __syncthreads();
      for (int r = t; r < m; r += nt) V64[r * m + col] *= T64[m];
      __syncthreads();
    }
    // T = C64 V64, then C64 = V64^T T  (the FP32 basis makes C64 nearly diagonal)
    for (int q = t; q < m * m; q += nt) {
      const int i = q / m, j = q % m;
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += C64[i * m + k] * V64[k * m + j];
      T64[q] = s;
    }
    __syncthreads();
    for (int q = t; q < m * m; q += nt) {
      const int i = q / m, j = q % m;
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += V64[k * m + i] * T64[k * m + j];
      C64[q] = s;
    }
    __syncthreads();
    for (int q = t; q < m * m; q += nt) {
      const int i = q / m, j = q % m;
      if (i < j) {
        const double a = 0.5 * (C64[i * m + j] + C64[j * m + i]);
        C64[i * m + j] = a;
        C64[j * m + i] = a;
      }
    }
    __syncthreads();
    for (; s64 < 6; ++s64) {
      offdiag_mass(C64, m, red, off, tot);
      if (!(off > 1e-30 * tot)) break;
      jacobi_sweep<double>(C64, V64, m, rc64, rs64);
    }
  } else {
    for (int q = t; q < m * m; q += nt) C64[q] = (double)C32[q];
    __syncthreads();
  }
  // sort descending by theta (rank by comparison; ties by index)
  for (int c = t; c < m; c += nt) {
    const double tc = C64[c * m + c];
    int rank = 0;
    for (int o = 0; o < m; ++o) {
      const double to = C64[o * m + o];
      if (to > tc || (to == tc && o < c)) ++rank;
    }
    theta[rank] = tc;
    for (int i = 0; i < m; ++i) Y[(size_t)i * ldy + rank] = V64[i * m + c];
  }
  if (t == 0) {
    info[0] = (double)s32;
    info[1] = (double)s64;
  }
}

// ------------------------------------------------------------------------------------------------
// Top-nvec eigenpairs of a small symmetric matrix in FP64 with few block-wide barriers:
// Householder tridiagonalisation (about 5 barriers per column), then, one thread per wanted
// eigenvalue, Sturm-sequence bisection and inverse iteration with a partially pivoted tridiagonal
// solve, re-orthogonalisation inside clusters, and the back-transformation by the reflectors.
// ------------------------------------------------------------------------------------------------
constexpr int kTriMaxVec = 48;

__device__ int sturm_count(const double* d, const double* e, int m, double x) {
  double q = d[0] - x;
  int cnt = q < 0.0 ? 1 : 0;
  for (int i = 1; i < m; ++i) {
    if (q == 0.0) q = 1e-300;
    q = d[i] - x - e[i - 1] * e[i - 1] / q;
    cnt += q < 0.0 ? 1 : 0;
  }
  return cnt;
}

// In-place solve of (tridiag(e, dd, e)) x = b with partial pivoting; dd, b overwritten; work
// arrays dl, du, du2 of length m.
__device__ void tridiag_solve_pivoted(const double* e, double* dd, double* b, double* dl, double* du, double* du2,
                                      int n, double tiny) {
  for (int i = 0; i < n - 1; ++i) {
    dl[i] = e[i];
    du[i] = e[i];
  }
  for (int i = 0; i < n - 1; ++i) {
    if (fabs(dd[i]) >= fabs(dl[i])) {
      if (dd[i] == 0.0) dd[i] = tiny;
      const double f = dl[i] / dd[i];
      dd[i + 1] -= f * du[i];
      b[i + 1] -= f * b[i];
      if (i < n - 2) du2[i] = 0.0;
    } else {
      const double f = dd[i] / dl[i];
      dd[i] = dl[i];
      const double tmp = dd[i + 1];
      dd[i + 1] = du[i] - f * tmp;
      if (i < n - 2) {
        du2[i] = du[i + 1];
        du[i + 1] = -f * du2[i];
      }
      du[i] = tmp;
      const double tb = b[i];
      b[i] = b[i + 1];
      b[i + 1] = tb - f * b[i + 1];
    }
  }
  if (dd[n - 1] == 0.0) dd[n - 1] = tiny;
  b[n - 1] /= dd[n - 1];
  if (n > 1) b[n - 2] = (b[n - 2] - du[n - 2] * b[n - 1]) / dd[n - 2];
  for (int i = n - 3; i >= 0; --i) b[i] = (b[i] - du[i] * b[i + 1] - du2[i] * b[i + 2]) / dd[i];
}

// H [m][ld] symmetric; returns the nvec (<= kTriMaxVec) largest eigenvalues in theta (descending)
// and their orthonormal eigenvectors in the first nvec columns of Y (ld = ldy).
__global__ void __launch_bounds__(256) k_small_eig_tridiag(const double* H, int m, int ld, int nvec, double* theta,
                                                           double* Y, int ldy, double* info) {
  extern __shared__ double sm[];
  double* A = sm;                  // [m*m]; column k below the diagonal stores reflector k
  double* d = A + m * m;           // [m] diagonal of T
  double* e = d + m;               // [m] sub-diagonal of T
  double* beta = e + m;            // [m]
  double* p = beta + m;            // [m]
  double* lam = p + m;             // [kTriMaxVec]
  double* Z = lam + kTriMaxVec;    // [kTriMaxVec][m] eigenvectors of T, then of H
  double* red = Z + kTriMaxVec * m;  // [64]
  const int t = threadIdx.x, nt = blockDim.x;
  for (int q = t; q < m * m; q += nt) {
    const int i = q / m, j = q % m;
    A[q] = 0.5 * (H[(size_t)i * ld + j] + H[(size_t)j * ld + i]);
  }
  __syncthreads();
  // ---- Householder tridiagonalisation
  for (int k = 0; k < m - 2; ++k) {
    const int s = m - k - 1;
    double* colk = A + (size_t)(k + 1) * m + k;  // x_i = colk[i * m]
    if (t < 32) {
      double sig = 0.0;
      for (int i = 1 + t; i < s; i += 32) sig += colk[i * m] * colk[i * m];
      for (int o = 16; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
      if (t == 0) {
        const double x0 = colk[0];
        if (sig == 0.0) {
          beta[k] = 0.0;
          e[k] = x0;
          red[0] = 1.0;  // v0 (no scaling of the tail)
        } else {
          const double mu = sqrt(x0 * x0 + sig);
          const double v0 = x0 <= 0.0 ? x0 - mu : -sig / (x0 + mu);
          beta[k] = 2.0 * v0 * v0 / (sig + v0 * v0);
          e[k] = mu;
          red[0] = v0;
        }
      }
    }
    __syncthreads();
    const double v0 = red[0], bk = beta[k];
    for (int i = 1 + t; i < s; i += nt) colk[i * m] /= v0;  // v = x / v0, v_0 = 1 (implicit)
    __syncthreads();
    if (bk != 0.0) {
      double* A22 = A + (size_t)(k + 1) * m + (k + 1);
      for (int i = t; i < s; i += nt) {
        double acc = 0.0;
        for (int j = 0; j < s; ++j) acc += A22[(size_t)i * m + j] * (j == 0 ? 1.0 : colk[j * m]);
        p[i] = bk * acc;
      }
      __syncthreads();
      if (t < 32) {
        double kk = 0.0;
        for (int i = t; i < s; i += 32) kk += p[i] * (i == 0 ? 1.0 : colk[i * m]);
        for (int o = 16; o > 0; o >>= 1) kk += __shfl_xor_sync(0xffffffffu, kk, o);
        if (t == 0) red[1] = 0.5 * bk * kk;
      }
      __syncthreads();
      const double K = red[1];
      for (int i = t; i < s; i += nt) p[i] -= K * (i == 0 ? 1.0 : colk[i * m]);
      __syncthreads();
      for (int q = t; q < s * s; q += nt) {
        const int i = q / s, j = q % s;
        const double vi = i == 0 ? 1.0 : colk[i * m], vj = j == 0 ? 1.0 : colk[j * m];
        A22[(size_t)i * m + j] -= vi * p[j] + p[i] * vj;
      }
    }
    __syncthreads();
  }
  for (int i = t; i < m; i += nt) d[i] = A[(size_t)i * m + i];
  if (t == 0 && m >= 2) e[m - 2] = A[(size_t)(m - 1) * m + (m - 2)];
  __syncthreads();
  // ---- eigenvalues (bisection) and eigenvectors (inverse iteration) of T, one thread each
  double tnorm = 0.0;
  for (int i = 0; i < m; ++i) {
    const double r = fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < m - 1 ? fabs(e[i]) : 0.0);
    tnorm = fmax(tnorm, r);
  }
  if (t < nvec) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
      const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < m - 1 ? fabs(e[i]) : 0.0);
      lo = fmin(lo, d[i] - r);
      hi = fmax(hi, d[i] + r);
    }
    const int rnk = m - 1 - t;
    for (int it = 0; it < 200; ++it) {
      if (hi - lo <= 2.2e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
      const double mid = 0.5 * (lo + hi);
      if (sturm_count(d, e, m, mid) <= rnk)
        lo = mid;
      else
        hi = mid;
    }
    const double l = 0.5 * (lo + hi);
    lam[t] = l;
    double dd[kRRMax], dl[kRRMax], du[kRRMax], du2[kRRMax];
    double* x = Z + (size_t)t * m;
    for (int i = 0; i < m; ++i) x[i] = 1.0 + 0.1 * (double)((i * 7919 + t * 31) % 13) / 13.0;
    for (int it = 0; it < 3; ++it) {
      for (int i = 0; i < m; ++i) dd[i] = d[i] - l;
      tridiag_solve_pivoted(e, dd, x, dl, du, du2, m, 2.2e-16 * tnorm);
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
      nrm = 1.0 / sqrt(nrm);
      for (int i = 0; i < m; ++i) x[i] *= nrm;
    }
  }
  __syncthreads();
  // ---- re-orthogonalise eigenvectors inside clusters of close eigenvalues (serial, small)
  if (t == 0) {
    for (int c = 1; c < nvec; ++c) {
      int c0 = c;
      while (c0 > 0 && fabs(lam[c0 - 1] - lam[c]) < 1e-6 * tnorm) --c0;
      if (c0 == c) continue;
      double* x = Z + (size_t)c * m;
      for (int jv = c0; jv < c; ++jv) {
        const double* y = Z + (size_t)jv * m;
        double dot = 0.0;
        for (int i = 0; i < m; ++i) dot += y[i] * x[i];
        for (int i = 0; i < m; ++i) x[i] -= dot * y[i];
      }
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
      nrm = 1.0 / sqrt(nrm);
      for (int i = 0; i < m; ++i) x[i] *= nrm;
    }
  }
  __syncthreads();
  // ---- back-transformation y = H_0 H_1 ... H_{m-3} z, one thread per vector
  if (t < nvec) {
    double* x = Z + (size_t)t * m;
    for (int k = m - 3; k >= 0; --k) {
      const double bk = beta[k];
      if (bk == 0.0) continue;
      double dot = x[k + 1];
      for (int i = k + 2; i < m; ++i) dot += A[(size_t)i * m + k] * x[i];
      dot *= bk;
      x[k + 1] -= dot;
      for (int i = k + 2; i < m; ++i) x[i] -= dot * A[(size_t)i * m + k];
    }
    theta[t] = lam[t];
  }
  __syncthreads();
  for (int q = t; q < m * nvec; q += nt) {
    const int i = q / nvec, c = q % nvec;
    Y[(size_t)i * ldy + c] = Z[(size_t)c * m + i];
  }
  if (t == 0) {
    info[0] = 0.0;
    info[1] = 0.0;
  }
}

// ------------------------------------------------------------------------------------------------
// The same method split over several thread blocks, so that the FP64 work of the per-eigenvalue
// bisection and inverse iteration (the dominant part at GB300's FP64 rate) runs on one SM per
// eigenvalue.  Scratch layout in global memory (tri, doubles):
//   [0, m*m)            reflectors (column k below the diagonal), as in k_small_eig_tridiag
//   d [m], e [m], beta [m], lam [kTriMaxVec], Z [kTriMaxVec][m]
// ------------------------------------------------------------------------------------------------
struct TriScratch {
  double *A, *d, *e, *beta, *lam, *Z;
  __host__ __device__ static TriScratch at(double* base, int mmax) {
    TriScratch s;
    s.A = base;
    s.d = base + (size_t)mmax * mmax;
    s.e = s.d + mmax;
    s.beta = s.e + mmax;
    s.lam = s.beta + mmax;
    s.Z = s.lam + kTriMaxVec;
    return s;
  }
  static size_t doubles(int mmax) { return (size_t)mmax * mmax + 3 * (size_t)mmax + kTriMaxVec + (size_t)kTriMaxVec * mmax; }
};

// Stage 1 (one block): Householder tridiagonalisation of H into the scratch.
__global__ void __launch_bounds__(256) k_tri_reduce(const double* H, int m, int ld, double* scratch, int mmax) {
  extern __shared__ double sm[];
  double* A = sm;           // [m*m]
  double* p = A + m * m;    // [m]
  double* beta = p + m;     // [m]
  double* e = beta + m;     // [m]
  double* red = e + m;      // [8]
  const int t = threadIdx.x, nt = blockDim.x;
  for (int q = t; q < m * m; q += nt) {
    const int i = q / m, j = q % m;
    A[q] = 0.5 * (H[(size_t)i * ld + j] + H[(size_t)j * ld + i]);
  }
  __syncthreads();
  for (int k = 0; k < m - 2; ++k) {
    const int s = m - k - 1;
    double* colk = A + (size_t)(k + 1) * m + k;
    if (t < 32) {
      double sig = 0.0;
      for (int i = 1 + t; i < s; i += 32) sig += colk[i * m] * colk[i * m];
      for (int o = 16; o > 0; o >>= 1) sig += __shfl_xor_sync(0xffffffffu, sig, o);
      if (t == 0) {
        const double x0 = colk[0];
        if (sig == 0.0) {
          beta[k] = 0.0;
          e[k] = x0;
          red[0] = 1.0;
        } else {
          const double mu = sqrt(x0 * x0 + sig);
          const double v0 = x0 <= 0.0 ? x0 - mu : -sig / (x0 + mu);
          beta[k] = 2.0 * v0 * v0 / (sig + v0 * v0);
          e[k] = mu;
          red[0] = v0;
        }
      }
    }
    __syncthreads();
    const double v0 = red[0], bk = beta[k];
    for (int i = 1 + t; i < s; i += nt) colk[i * m] /= v0;
    __syncthreads();
    if (bk != 0.0) {
      const double* A22 = A + (size_t)(k + 1) * m + (k + 1);
      // p = bk A22 v, reading A22 by columns (symmetric) so that neighbouring threads touch
      // neighbouring words
      for (int i = t; i < s; i += nt) {
        double acc = 0.0;
        for (int j = 0; j < s; ++j) acc += A22[(size_t)j * m + i] * (j == 0 ? 1.0 : colk[j * m]);
        p[i] = bk * acc;
      }
      __syncthreads();
      if (t < 32) {
        double kk = 0.0;
        for (int i = t; i < s; i += 32) kk += p[i] * (i == 0 ? 1.0 : colk[i * m]);
        for (int o = 16; o > 0; o >>= 1) kk += __shfl_xor_sync(0xffffffffu, kk, o);
        if (t == 0) red[1] = 0.5 * bk * kk;
      }
      __syncthreads();
      const double K = red[1];
      for (int i = t; i < s; i += nt) p[i] -= K * (i == 0 ? 1.0 : colk[i * m]);
      __syncthreads();
      double* A22w = A + (size_t)(k + 1) * m + (k + 1);
      for (int q = t; q < s * s; q += nt) {
        const int i = q / s, j = q % s;
        const double vi = i == 0 ? 1.0 : colk[i * m], vj = j == 0 ? 1.0 : colk[j * m];
        A22w[(size_t)i * m + j] -= vi * p[j] + p[i] * vj;
      }
    }
    __syncthreads();
  }
  TriScratch S = TriScratch::at(scratch, mmax);
  for (int q = t; q < m * m; q += nt) S.A[q] = A[q];
  for (int i = t; i < m; i += nt) {
    S.d[i] = A[(size_t)i * m + i];
    S.beta[i] = i < m - 2 ? beta[i] : 0.0;
    S.e[i] = i < m - 2 ? e[i] : (i == m - 2 ? A[(size_t)(m - 1) * m + (m - 2)] : 0.0);
  }
}

// Stage 2 (one block of 64 threads per wanted eigenvalue c): the c-th largest eigenvalue of T by
// multisection (64 Sturm counts per round), then its eigenvector by inverse iteration.
__global__ void __launch_bounds__(64) k_tri_eigvec(double* scratch, int mmax, int m) {
  const TriScratch S = TriScratch::at(scratch, mmax);
  __shared__ double d[kRRMax], e[kRRMax];
  __shared__ double lo_s, hi_s;
  __shared__ int cnt[64];
  const int t = threadIdx.x, c = blockIdx.x;
  for (int i = t; i < m; i += blockDim.x) {
    d[i] = S.d[i];
    e[i] = S.e[i];
  }
  __syncthreads();
  double tnorm = 0.0, lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < m - 1 ? fabs(e[i]) : 0.0);
    tnorm = fmax(tnorm, fabs(d[i]) + r);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
  }
  const int rnk = m - 1 - c;  // rank among the ascending eigenvalues
  for (int round = 0; round < 40; ++round) {
    if (hi - lo <= 2.2e-16 * fmax(fabs(lo), fabs(hi)) + 1e-300) break;
    const double x = lo + (hi - lo) * (double)(t + 1) / (double)(blockDim.x + 1);
    cnt[t] = sturm_count(d, e, m, x);
    __syncthreads();
    if (t == 0) {
      // sample points x_1 < ... < x_64; keep the sub-interval whose ends bracket rank rnk
      double nlo = lo, nhi = hi;
      for (int k = 0; k < (int)blockDim.x; ++k) {
        const double xk = lo + (hi - lo) * (double)(k + 1) / (double)(blockDim.x + 1);
        if (cnt[k] <= rnk)
          nlo = xk;
        else {
          nhi = xk;
          break;
        }
      }
      lo_s = nlo;
      hi_s = nhi;
    }
    __syncthreads();
    lo = lo_s;
    hi = hi_s;
    __syncthreads();
  }
  if (t != 0) return;
  const double l = 0.5 * (lo + hi);
  S.lam[c] = l;
  double dd[kRRMax], dl[kRRMax], du[kRRMax], du2[kRRMax];
  double* x = S.Z + (size_t)c * m;
  for (int i = 0; i < m; ++i) x[i] = 1.0 + 0.1 * (double)((i * 7919 + c * 31) % 13) / 13.0;
  for (int it = 0; it < 3; ++it) {
    for (int i = 0; i < m; ++i) dd[i] = d[i] - l;
    tridiag_solve_pivoted(e, dd, x, dl, du, du2, m, 2.2e-16 * tnorm);
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
    nrm = 1.0 / sqrt(nrm);
    for (int i = 0; i < m; ++i) x[i] *= nrm;
  }
}

// Stage 3 (one block): re-orthogonalisation inside clusters, back-transformation, output.
__global__ void __launch_bounds__(256) k_tri_finish(double* scratch, int mmax, int m, int nvec, double* theta,
                                                    double* Y, int ldy) {
  const TriScratch S = TriScratch::at(scratch, mmax);
  extern __shared__ double sm[];
  double* Z = sm;                       // [nvec][m]
  double* A = Z + (size_t)nvec * m;     // [m*m] reflectors
  double* dots = A + (size_t)m * m;     // [kTriMaxVec]
  const int t = threadIdx.x, nt = blockDim.x;
  for (int q = t; q < nvec * m; q += nt) Z[q] = S.Z[q];
  for (int q = t; q < m * m; q += nt) A[q] = S.A[q];
  double tnorm = 0.0;
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(S.e[i - 1]) : 0.0) + (i < m - 1 ? fabs(S.e[i]) : 0.0);
    tnorm = fmax(tnorm, fabs(S.d[i]) + r);
  }
  __syncthreads();
  for (int cc = 1; cc < nvec; ++cc) {
    int c0 = cc;
    while (c0 > 0 && fabs(S.lam[c0 - 1] - S.lam[cc]) < 1e-6 * tnorm) --c0;
    if (c0 == cc) continue;  // uniform across the block
    double* x = Z + (size_t)cc * m;
    const int w = t >> 5, lane = t & 31;
    for (int jv = c0 + w; jv < cc; jv += nt >> 5) {  // one warp per previous cluster member
      const double* y = Z + (size_t)jv * m;
      double s = 0.0;
      for (int i = lane; i < m; i += 32) s += y[i] * x[i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) dots[jv] = s;
    }
    __syncthreads();
    for (int i = t; i < m; i += nt) {
      double v = x[i];
      for (int jv = c0; jv < cc; ++jv) v -= dots[jv] * Z[(size_t)jv * m + i];
      x[i] = v;
    }
    __syncthreads();
    if (t < 32) {
      double s = 0.0;
      for (int i = t; i < m; i += 32) s += x[i] * x[i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (t == 0) dots[kTriMaxVec - 1] = 1.0 / sqrt(s);
    }
    __syncthreads();
    const double sc = dots[kTriMaxVec - 1];
    for (int i = t; i < m; i += nt) x[i] *= sc;
    __syncthreads();
  }
  // back-transformation, one thread per vector
  if (t < nvec) {
    double* x = Z + (size_t)t * m;
    for (int k = m - 3; k >= 0; --k) {
      const double bk = S.beta[k];
      if (bk == 0.0) continue;
      double dot = x[k + 1];
      for (int i = k + 2; i < m; ++i) dot += A[(size_t)i * m + k] * x[i];
      dot *= bk;
      x[k + 1] -= dot;
      for (int i = k + 2; i < m; ++i) x[i] -= dot * A[(size_t)i * m + k];
    }
    theta[t] = S.lam[t];
  }
  __syncthreads();
  for (int q = t; q < m * nvec; q += nt) {
    const int i = q / nvec, c = q % nvec;
    Y[(size_t)i * ldy + c] = Z[(size_t)c * m + i];
  }
}

inline size_t tri_reduce_smem_bytes() { return sizeof(double) * ((size_t)kRRMax * kRRMax + 3 * (size_t)kRRMax + 8); }
inline size_t tri_finish_smem_bytes() {
  return sizeof(double) * ((size_t)kTriMaxVec * kRRMax + (size_t)kRRMax * kRRMax + kTriMaxVec);
}

inline size_t small_eig_tridiag_smem_bytes() {
  return sizeof(double) * ((size_t)kRRMax * kRRMax + 4 * (size_t)kRRMax + kTriMaxVec + (size_t)kTriMaxVec * kRRMax + 64);
}

inline size_t small_rr_smem_bytes() {
  return sizeof(double) * (3 * (size_t)kRRMax * kRRMax + 2 * kRRMax + 64) +
         sizeof(float) * (2 * (size_t)kRRMax * kRRMax + 2 * kRRMax);
}

}  // namespace tobk
