// Dense Rayleigh-Ritz of the projected buckling pencil (included by eigen.cu), the dense step of
// the coarse eigenproblem (eq. eigenvalueProblemCoarseScale; solved to a residual of 1e-8, Appendix A).
//
// The eigensolver keeps its basis K-orthonormal, so the projected problem is the standard
// symmetric eigenproblem H y = theta y with H = V^T (-G) V (size m <= kRRMax; the eigensolver writes
// every entry pair H[i][j], H[j][i] with one value, so H is exactly symmetric and the kernels below
// read one triangle's order only).  A dense eigensolver
// is a long chain of dependent steps confined to one SM, and GB300 executes FP64 at 1/64 of its
// FP32 rate (2 FP64 FMA per clock per SM), so the O(m^3) work of the decomposition is done in FP32
// and FP64 accuracy is recovered by a refinement made only of matrix products, spread over one
// thread block per column:
//   1. k_rr_eig32 (one block): all m eigenvectors of H by cyclic Jacobi sweeps in FP32.
//   2. kRRRefineSteps refinement steps in FP64 (Ogita & Aishima, "Iterative refinement for symmetric
//      eigenvalue decomposition", Japan J. Indust. Appl. Math. 35 (2018)): with X the current
//      eigenvector matrix, R = I - X^T X, S = X^T H X, lambda_i = s_ii / (1 - r_ii),
//      E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) for i != j, E_ii = r_ii / 2, and
//      X <- X + X E; each step squares the error.  Pairs closer than the step's error bound delta
//      get E_ij = r_ij / 2, which refines their common subspace but not its split.
//   3. k_rr_finish (one block): the wanted columns sorted by lambda; every cluster of wanted
//      eigenvalues closer than delta is split by FP64 Jacobi rotations of its small block of
//      X^T H X.
// Eigenpairs are returned sorted by descending theta.
#pragma once
#include <cuda_runtime.h>

namespace tobk {

constexpr int kRRMax = 64;  // largest projected problem (the FP32 stage pads to it)
// FP32 stage stopping rule: off-diagonal mass below this fraction of the total (off-diagonal entries
// about 3e-5 of the norm); each of the kRRRefineSteps FP64 refinement steps then squares the error
// (3e-5 -> 1e-9 -> 1e-18).
constexpr double kRRJacobiTol2 = 1e-9;
constexpr int kRRRefineSteps = 2;
static_assert(kRRRefineSteps >= 2, "the eigensolver's warm start reads the first refined X");

// Stage 1.  All m eigenvectors of H [m][ld] (symmetric) in FP32 by cyclic Jacobi, written in
// FP64 to X [m][m] (column c = eigenvector of the c-th largest eigenvalue).  The matrix is padded
// to P (a multiple of 8, P >= m; padding rows are never rotated).  One round applies P/2 disjoint
// rotations J_k (round-robin pairing of the P indices) as C <- J C J^T, as independent 2 x 2
// blocks.  Warp w owns the row slots A = w and A = w + P/4 of a round; lane B < P/2 owns column slot
// B: the thread updates the blocks (A, B) of C and rows B and B + P/2 of the accumulated rotation's
// columns p_A, q_A.  Lane k of every warp computes the rotation of slot k from the diagonal block of C
// (the same arithmetic on the same values in every warp) and the warp's row rotations are broadcast
// by shuffles.  C is double-buffered (a round reads one copy and writes the other), so a round costs
// one barrier and no thread waits for another's rotation.  The rotations only steer the FP32 stage
// (the FP64 refinement below fixes the digits), so they use fast reciprocal / square-root
// approximations.  Shared arrays have the odd row stride P + 1.  Warm start: when mprev > 0, Xp
// [mprev][mprev] (the previous eigenvectors of the leading mprev x mprev block, FP64) starts the
// accumulated rotation V = diag(Xp, I), so that the old block is already nearly diagonal.
// info[0] = sweeps.
namespace rr_detail {
// Round-robin (circle) pairing of P indices: in round r (0 <= r < P - 1), slot k pairs (p, q); every
// index appears in exactly one slot of a round and every pair in exactly one round of a sweep.
template <int P>
__device__ __forceinline__ void pair_of(int r, int k, int& p, int& q) {
  if (k == 0) {
    p = P - 1;
    q = r;
  } else {
    p = r + k;
    if (p >= P - 1) p -= P - 1;
    q = r - k;
    if (q < 0) q += P - 1;
  }
}

// Rotation (c, s) that zeroes C[p][q] when rows and columns p, q are replaced by c p - s q and
// s p + c q: t = s / c is the smaller root of t^2 + 2 tau t - 1 = 0, tau = (a_qq - a_pp) / (2 a_pq).
__device__ __forceinline__ void jacobi_rotation(float app, float aqq, float apq, float& c, float& s) {
  c = 1.f;
  s = 0.f;
  if (apq != 0.f) {
    const float tau = __fdividef(aqq - app, 2.f * apq);
    const float at = fabsf(tau);
    // tan of the rotation angle, 1 / (|tau| + sqrt(1 + tau^2)), signed like tau
    float tt = at < 1e18f ? __fdividef(1.f, at + (1.f + at * at) * rsqrtf(1.f + at * at)) : __fdividef(0.5f, at);
    tt = tau >= 0.f ? tt : -tt;
    c = rsqrtf(1.f + tt * tt);
    s = tt * c;
  }
}

// The 2 x 2 block of C at rows (pa, qa), columns (pb, qb) rotated on both sides, Cc -> Cn.
template <int LD>
__device__ __forceinline__ void rotate_block(const float* Cc, float* Cn, int pa, int qa, float ca, float sa, int pb,
                                             int qb, float cb, float sb) {
  const float b00 = Cc[pa * LD + pb], b01 = Cc[pa * LD + qb], b10 = Cc[qa * LD + pb], b11 = Cc[qa * LD + qb];
  const float l00 = ca * b00 - sa * b10, l01 = ca * b01 - sa * b11;
  const float l10 = sa * b00 + ca * b10, l11 = sa * b01 + ca * b11;
  Cn[pa * LD + pb] = cb * l00 - sb * l01;
  Cn[pa * LD + qb] = sb * l00 + cb * l01;
  Cn[qa * LD + pb] = cb * l10 - sb * l11;
  Cn[qa * LD + qb] = sb * l10 + cb * l11;
}

// Accumulated rotation V <- V J^T on columns pa, qa (stored as rows of V), at rows r0 and r1.
template <int LD>
__device__ __forceinline__ void rotate_vcols(float* V, int pa, int qa, float ca, float sa, int r0, int r1) {
  float* vp = V + pa * LD;
  float* vq = V + qa * LD;
  const float p0 = vp[r0], p1 = vp[r1], q0 = vq[r0], q1 = vq[r1];
  vp[r0] = ca * p0 - sa * q0;
  vp[r1] = ca * p1 - sa * q1;
  vq[r0] = sa * p0 + ca * q0;
  vq[r1] = sa * p1 + ca * q1;
}
}  // namespace rr_detail

template <int P>
__global__ void __launch_bounds__(8 * P) k_rr_eig32(const double* H, int m, int ld, const double* Xp, int mprev,
                                                    double* X, double* info, double tol2) {
  pdl_wait();
  static_assert(P % 8 == 0 && P <= kRRMax, "padded size");
  constexpr int NP = P / 2;    // rotations per round (column slots, one per lane)
  constexpr int NW = NP / 2;   // warps; warp w owns row slots w and w + NW
  constexpr int NT = 32 * NW;
  constexpr int LD = P + 1;
  constexpr int SZ = P * LD;
  extern __shared__ float sm32[];
  float* Cc = sm32;          // current copy of the rotated matrix
  float* Cn = sm32 + SZ;     // next copy (and the warm start's scratch)
  float* V = sm32 + 2 * SZ;  // accumulated rotations, transposed: V[col * LD + row]
  __shared__ unsigned short ptab[(P - 1) * NP];  // round r, slot k -> p | q << 8
  __shared__ double red[2 * NW];
  __shared__ double hmax_s;
  __shared__ int done_s;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const bool own = lane < NP;
  for (int q = t; q < (P - 1) * NP; q += NT) {
    int p, r;
    rr_detail::pair_of<P>(q / NP, q % NP, p, r);
    ptab[q] = (unsigned short)(p | (r << 8));
  }
  // scale by max |H| so that the FP32 working range holds any problem scaling
  double mx = 0.0;
  for (int q = t; q < m * m; q += NT) mx = fmax(mx, fabs(H[(size_t)(q / m) * ld + q % m]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (t == 0) {
    double a = 0.0;
    for (int w = 0; w < NW; ++w) a = fmax(a, red[w]);
    hmax_s = a > 0.0 ? a : 1.0;
  }
  __syncthreads();
  const float inv = (float)(1.0 / hmax_s);
  for (int q = t; q < P * P; q += NT) {
    const int i = q / P, j = q % P;
    float h = 0.f, v = (i == j) ? 1.f : 0.f;
    if (i < m && j < m) h = inv * (float)H[(size_t)i * ld + j];
    if (i < mprev && j < mprev) v = (float)Xp[(size_t)i * mprev + j];
    Cc[i * LD + j] = h;
    V[j * LD + i] = v;
  }
  __syncthreads();
  if (mprev > 0) {  // C <- V^T C V in 2 x 2 register tiles (rows 2A, 2A + 1, columns 2B, 2B + 1)
    const int j0 = 2 * lane;
    for (int pass = 0; pass < 2; ++pass) {
      const float* Lm = pass == 0 ? Cc : V;  // left factor rows:  C[i][k]  |  V^T[i][k] = V[i * LD + k]
      const float* Rm = pass == 0 ? V : Cn;  // right factor:      V[j][k] (= V(k, j))  |  T[k][j]
      float* Out = pass == 0 ? Cn : Cc;
      if (own) {
        for (int half = 0; half < 2; ++half) {
          const int i0 = 2 * (warp + half * NW);
          float a00 = 0.f, a01 = 0.f, a10 = 0.f, a11 = 0.f;
#pragma unroll 8
          for (int k = 0; k < P; ++k) {
            const float l0 = Lm[i0 * LD + k], l1 = Lm[(i0 + 1) * LD + k];
            const float r0 = pass == 0 ? Rm[j0 * LD + k] : Rm[k * LD + j0];
            const float r1 = pass == 0 ? Rm[(j0 + 1) * LD + k] : Rm[k * LD + j0 + 1];
            a00 += l0 * r0;
            a01 += l0 * r1;
            a10 += l1 * r0;
            a11 += l1 * r1;
          }
          Out[i0 * LD + j0] = a00;
          Out[i0 * LD + j0 + 1] = a01;
          Out[(i0 + 1) * LD + j0] = a10;
          Out[(i0 + 1) * LD + j0 + 1] = a11;
        }
      }
      __syncthreads();
    }
  }
  int sweeps = 0;
  for (; sweeps < 30; ++sweeps) {
    // convergence: off-diagonal mass below tol2 of the total
    float o = 0.f, a = 0.f;
    for (int q = t; q < P * P; q += NT) {
      const int i = q / P, j = q % P;
      const float v = Cc[i * LD + j] * Cc[i * LD + j];
      a += v;
      if (i != j) o += v;
    }
    for (int s = 16; s > 0; s >>= 1) {
      o += __shfl_xor_sync(0xffffffffu, o, s);
      a += __shfl_xor_sync(0xffffffffu, a, s);
    }
    if (lane == 0) {
      red[2 * warp] = o;
      red[2 * warp + 1] = a;
    }
    __syncthreads();
    if (t == 0) {
      double oo = 0.0, aa = 0.0;
      for (int w = 0; w < NW; ++w) {
        oo += red[2 * w];
        aa += red[2 * w + 1];
      }
      done_s = !(oo > tol2 * aa);
    }
    __syncthreads();
    if (done_s) break;
    for (int round = 0; round < P - 1; ++round) {
      // rotation of column slot `lane` (lanes >= NP hold the identity)
      int pq = 0;
      float cB = 1.f, sB = 0.f;
      if (own) {
        pq = ptab[round * NP + lane];
        const int pB = pq & 255, qB = pq >> 8;
        if (pB < m && qB < m)
          rr_detail::jacobi_rotation(Cc[pB * LD + pB], Cc[qB * LD + qB], Cc[pB * LD + qB], cB, sB);
      }
      // row slots warp and warp + NW: rotations and pairs from those lanes
      const int A0 = warp, A1 = warp + NW;
      const float cA0 = __shfl_sync(0xffffffffu, cB, A0), sA0 = __shfl_sync(0xffffffffu, sB, A0);
      const float cA1 = __shfl_sync(0xffffffffu, cB, A1), sA1 = __shfl_sync(0xffffffffu, sB, A1);
      const int pqA0 = __shfl_sync(0xffffffffu, pq, A0), pqA1 = __shfl_sync(0xffffffffu, pq, A1);
      if (own) {
        const int pB = pq & 255, qB = pq >> 8;
        const int pA0 = pqA0 & 255, qA0 = pqA0 >> 8, pA1 = pqA1 & 255, qA1 = pqA1 >> 8;
        rr_detail::rotate_block<LD>(Cc, Cn, pA0, qA0, cA0, sA0, pB, qB, cB, sB);
        rr_detail::rotate_block<LD>(Cc, Cn, pA1, qA1, cA1, sA1, pB, qB, cB, sB);
        rr_detail::rotate_vcols<LD>(V, pA0, qA0, cA0, sA0, lane, lane + NP);
        rr_detail::rotate_vcols<LD>(V, pA1, qA1, cA1, sA1, lane, lane + NP);
      }
      __syncthreads();
      float* tmp = Cc;
      Cc = Cn;
      Cn = tmp;
    }
  }
  // descending order of the diagonal (ties by index); padding rows excluded
  for (int c = t; c < m; c += NT) {
    const float tc = Cc[c * LD + c];
    int rank = 0;
    for (int o = 0; o < m; ++o) {
      const float to = Cc[o * LD + o];
      if (to > tc || (to == tc && o < c)) ++rank;
    }
    for (int i = 0; i < m; ++i) X[(size_t)i * m + rank] = (double)V[c * LD + i];
  }
  if (t == 0) info[0] = (double)sweeps;
}

template <int P>
inline size_t rr_eig32_smem_bytes() {
  return sizeof(float) * 3 * (size_t)P * (P + 1);
}

// Stage 1 launch: the smallest padded size (a multiple of 8) that holds m.
template <int P>
inline void rr_eig32_launch(const double* H, int m, int ld, const double* Xp, int mprev, double* X, double* info,
                            double tol2, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_rr_eig32<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rr_eig32_smem_bytes<P>());
    configured = true;
  }
  launch_pdl(k_rr_eig32<P>, dim3(1), dim3(8 * P), rr_eig32_smem_bytes<P>(), st, H, m, ld, Xp, mprev, X, info, tol2);
}

inline void launch_rr_eig32(const double* H, int m, int ld, const double* Xp, int mprev, double* X, double* info,
                            cudaStream_t st, double tol2 = kRRJacobiTol2) {
  switch ((m + 7) / 8) {
    case 0:
    case 1:
    case 2: rr_eig32_launch<16>(H, m, ld, Xp, mprev, X, info, tol2, st); break;
    case 3: rr_eig32_launch<24>(H, m, ld, Xp, mprev, X, info, tol2, st); break;
    case 4: rr_eig32_launch<32>(H, m, ld, Xp, mprev, X, info, tol2, st); break;
    case 5: rr_eig32_launch<40>(H, m, ld, Xp, mprev, X, info, tol2, st); break;
    case 6: rr_eig32_launch<48>(H, m, ld, Xp, mprev, X, info, tol2, st); break;
    case 7: rr_eig32_launch<56>(H, m, ld, Xp, mprev, X, info, tol2, st); break;
    default: rr_eig32_launch<64>(H, m, ld, Xp, mprev, X, info, tol2, st); break;
  }
}

// Stage 2a.  S = X^T H X and R = I - X^T X ([m][m] each); block j computes column j.  256 threads:
// four groups of 64 take every fourth term of each dot product (four times the loads in flight of
// one thread per row) and the four partial sums are added in a fixed order.
constexpr int kOAThreads = 256;
__global__ void __launch_bounds__(kOAThreads) k_rr_oa_products(const double* H, int ld, const double* X, int m,
                                                               double* S, double* R) {
  pdl_wait();
  __shared__ double xj[kRRMax], pj[kRRMax];
  __shared__ double part[3][4][kRRMax];
  const int j = blockIdx.x, t = threadIdx.x;
  const int g = t >> 6, i = t & 63;
  if (t < m) xj[t] = X[(size_t)t * m + j];
  __syncthreads();
  if (i < m) {
    double s = 0.0;
    for (int k = g; k < m; k += 4) s += H[(size_t)k * ld + i] * xj[k];
    part[0][g][i] = s;
  }
  __syncthreads();
  if (t < m) pj[t] = ((part[0][0][t] + part[0][1][t]) + part[0][2][t]) + part[0][3][t];
  __syncthreads();
  if (i < m) {
    double s = 0.0, r = 0.0;
    for (int k = g; k < m; k += 4) {
      const double xki = X[(size_t)k * m + i];
      s += xki * pj[k];
      r += xki * xj[k];
    }
    part[1][g][i] = s;
    part[2][g][i] = r;
  }
  __syncthreads();
  if (t < m) {
    const double sv = ((part[1][0][t] + part[1][1][t]) + part[1][2][t]) + part[1][3][t];
    const double rv = ((part[2][0][t] + part[2][1][t]) + part[2][2][t]) + part[2][3][t];
    S[(size_t)t * m + j] = sv;
    R[(size_t)t * m + j] = (t == j ? 1.0 : 0.0) - rv;
  }
}

// Stage 2b.  One refinement step for columns j < gridDim.x (block j, 256 threads):
// Xout[:, j] = X[:, j] + X E[:, j] (ldo = leading dimension of Xout) and lam_out[j].
// set_delta != 0: the step's error bound delta = 2 (||S - diag(lambda)||_F + max|lambda| ||R||_F)
// is computed (by every block, identically) and block 0 stores it in *delta; otherwise *delta is
// read.
__global__ void __launch_bounds__(kOAThreads) k_rr_oa_update(const double* X, const double* S, const double* R, int m,
                                                             double* Xout, int ldo, double* lam_out, double* delta,
                                                             int set_delta) {
  pdl_wait();
  constexpr int NW = kOAThreads / 32;
  __shared__ double lam[kRRMax], e[kRRMax], red[3 * NW];
  __shared__ double part[4][kRRMax];
  const int j = blockIdx.x, t = threadIdx.x, nt = blockDim.x;
  if (t < m) lam[t] = S[(size_t)t * m + t] / (1.0 - R[(size_t)t * m + t]);
  __syncthreads();
  double dl;
  if (set_delta) {
    double so = 0.0, ro = 0.0, lm = 0.0;
    for (int q = t; q < m * m; q += nt) {
      const int i = q / m, k = q % m;
      const double sv = S[q] - (i == k ? lam[i] : 0.0);
      so += sv * sv;
      ro += R[q] * R[q];
    }
    if (t < m) lm = fabs(lam[t]);
    for (int o = 16; o > 0; o >>= 1) {
      so += __shfl_xor_sync(0xffffffffu, so, o);
      ro += __shfl_xor_sync(0xffffffffu, ro, o);
      lm = fmax(lm, __shfl_xor_sync(0xffffffffu, lm, o));
    }
    if ((t & 31) == 0) {
      red[3 * (t >> 5)] = so;
      red[3 * (t >> 5) + 1] = ro;
      red[3 * (t >> 5) + 2] = lm;
    }
    __syncthreads();
    so = 0.0;
    ro = 0.0;
    lm = 0.0;
    for (int w = 0; w < NW; ++w) {
      so += red[3 * w];
      ro += red[3 * w + 1];
      lm = fmax(lm, red[3 * w + 2]);
    }
    dl = 2.0 * (sqrt(so) + lm * sqrt(ro));
    if (j == 0 && t == 0) *delta = dl;
  } else {
    dl = *delta;
  }
  if (t < m) {
    const double rij = R[(size_t)t * m + j];
    double eij = 0.5 * rij;
    if (t != j && fabs(lam[j] - lam[t]) > dl) eij = (S[(size_t)t * m + j] + lam[j] * rij) / (lam[j] - lam[t]);
    e[t] = eij;
  }
  __syncthreads();
  const int g = t >> 6, r = t & 63;
  if (r < m) {
    double s = 0.0;
    for (int i = g; i < m; i += 4) s += X[(size_t)r * m + i] * e[i];
    part[g][r] = s;
  }
  __syncthreads();
  if (t < m) Xout[(size_t)t * ldo + j] = X[(size_t)t * m + j] + (((part[0][t] + part[1][t]) + part[2][t]) + part[3][t]);
  if (t == 0 && lam_out) lam_out[j] = lam[j];
}

// Stage 3 (one block).  The nvec refined columns Xw [m][ldw] with their lam are sorted by
// descending lam; each run of neighbours closer than *delta (a cluster the refinement did not
// split) is diagonalised by FP64 Jacobi rotations of its block B = Z^T H Z.  Outputs
// theta[nvec] (descending) and Y [m][ldy].  Scratch in shared memory (dynamic): Z [nvec][m],
// HZ [kRRClusterMax][m].
constexpr int kRRClusterMax = 16;
__global__ void __launch_bounds__(256) k_rr_finish(const double* H, int ld, int m, int nvec, const double* Xw, int ldw,
                                                   const double* lam_in, const double* delta, double* theta, double* Y,
                                                   int ldy) {
  pdl_wait();
  extern __shared__ double smd[];
  double* Z = smd;                                   // [nvec][m]
  double* HZ = Z + (size_t)nvec * m;                 // [kRRClusterMax][m]
  __shared__ double l[kRRMax], B[kRRClusterMax * kRRClusterMax], Q[kRRClusterMax * kRRClusterMax];
  __shared__ int rk[kRRClusterMax];
  const int t = threadIdx.x, nt = blockDim.x;
  for (int c = t; c < nvec; c += nt) {
    const double lc = lam_in[c];
    int rank = 0;
    for (int o = 0; o < nvec; ++o) {
      const double lo = lam_in[o];
      if (lo > lc || (lo == lc && o < c)) ++rank;
    }
    l[rank] = lc;
    for (int i = 0; i < m; ++i) Z[(size_t)rank * m + i] = Xw[(size_t)i * ldw + c];
  }
  __syncthreads();
  const double dl = *delta;
  int c0 = 0;
  while (c0 < nvec) {
    int c1 = c0 + 1;
    while (c1 < nvec && c1 - c0 < kRRClusterMax && fabs(l[c1 - 1] - l[c1]) <= dl) ++c1;
    const int c = c1 - c0;
    if (c > 1) {
      // HZ = H Z_c, B = Z_c^T HZ
      for (int q = t; q < c * m; q += nt) {
        const int a = q / m, i = q % m;
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += H[(size_t)k * ld + i] * Z[(size_t)(c0 + a) * m + k];
        HZ[(size_t)a * m + i] = s;
      }
      __syncthreads();
      for (int q = t; q < c * c; q += nt) {
        const int a = q / c, b = q % c;
        double s = 0.0;
        for (int k = 0; k < m; ++k) s += Z[(size_t)(c0 + a) * m + k] * HZ[(size_t)b * m + k];
        B[q] = s;
        Q[q] = (a == b) ? 1.0 : 0.0;
      }
      __syncthreads();
      if (t == 0) {
        for (int a = 0; a < c; ++a)
          for (int b = a + 1; b < c; ++b) {
            const double s = 0.5 * (B[a * c + b] + B[b * c + a]);
            B[a * c + b] = s;
            B[b * c + a] = s;
          }
        for (int sweep = 0; sweep < 12; ++sweep) {
          double off = 0.0, tot = 0.0;
          for (int q = 0; q < c * c; ++q) {
            tot += B[q] * B[q];
            if (q / c != q % c) off += B[q] * B[q];
          }
          if (!(off > 1e-32 * tot)) break;
          for (int p = 0; p < c - 1; ++p)
            for (int r = p + 1; r < c; ++r) {
              const double apr = B[p * c + r];
              if (apr == 0.0) continue;
              const double tau = (B[r * c + r] - B[p * c + p]) / (2.0 * apr);
              const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
              const double cs = 1.0 / sqrt(1.0 + tt * tt), sn = tt * cs;
              for (int k = 0; k < c; ++k) {  // rows p, r
                const double xp = B[p * c + k], xr = B[r * c + k];
                B[p * c + k] = cs * xp - sn * xr;
                B[r * c + k] = sn * xp + cs * xr;
              }
              for (int k = 0; k < c; ++k) {  // columns p, r and the rotation
                const double xp = B[k * c + p], xr = B[k * c + r];
                B[k * c + p] = cs * xp - sn * xr;
                B[k * c + r] = sn * xp + cs * xr;
                const double qp = Q[k * c + p], qr = Q[k * c + r];
                Q[k * c + p] = cs * qp - sn * qr;
                Q[k * c + r] = sn * qp + cs * qr;
              }
            }
        }
        // order the cluster's eigenpairs by descending value
        for (int a = 0; a < c; ++a) {
          int rank = 0;
          for (int o = 0; o < c; ++o)
            if (B[o * c + o] > B[a * c + a] || (B[o * c + o] == B[a * c + a] && o < a)) ++rank;
          rk[a] = rank;
        }
        for (int a = 0; a < c; ++a) l[c0 + rk[a]] = B[a * c + a];
      }
      __syncthreads();
      // Z_c <- Z_c Q (columns permuted into descending order), through HZ as scratch
      for (int q = t; q < c * m; q += nt) {
        const int a = q / m, i = q % m;
        double s = 0.0;
        for (int k = 0; k < c; ++k) s += Z[(size_t)(c0 + k) * m + i] * Q[k * c + a];
        HZ[(size_t)rk[a] * m + i] = s;
      }
      __syncthreads();
      for (int q = t; q < c * m; q += nt) Z[(size_t)c0 * m + q] = HZ[q];
      __syncthreads();
    }
    c0 = c1;
  }
  for (int c = t; c < nvec; c += nt) theta[c] = l[c];
  for (int q = t; q < m * nvec; q += nt) {
    const int i = q / nvec, c = q % nvec;
    Y[(size_t)i * ldy + c] = Z[(size_t)c * m + i];
  }
}

inline size_t rr_finish_smem_bytes(int m, int nvec) {
  return sizeof(double) * ((size_t)nvec * m + (size_t)kRRClusterMax * m);
}

}  // namespace tobk
