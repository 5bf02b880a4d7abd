// Many independent designs solved together (the multi-design batching form of the solver path).
//
// Every design keeps its own multigrid hierarchy (a solve-only handle: SIMP moduli, Galerkin levels,
// nodal stencils, smoother coefficients, coarsest inverse), built by the single-design set-up.  The
// solve then runs flexible CG in FP64 on all designs and all right-hand sides at once, with an FP32
// V-cycle (paper Appendix A: mgPCG; the V-cycle in FP32 storage and arithmetic, as in
// TOBK_FP32_VCYCLE).  Each phase of the CG iteration and of the V-cycle is ONE grouped launch over
// a work list of (design, tile) items gathered from every design that takes part in the phase; the
// blocks walk the list with a grid stride (persistent-style, at most a few blocks per SM), so that
// designs of uneven size fill the GPU together.  Two CG iterations are captured into a CUDA graph
// once and replayed; converged (design, RHS) pairs skip their tiles.  The tile shape of the fine
// FP32 smoother and the RHS blocking of the coarse stencil kernel are chosen by a small autotuner
// that times the candidate variants on the batch itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "handle.h"
#include "q4_element.cuh"

namespace tobk {

constexpr int kBatchMaxLevels = 8;

struct BLevel {             // one level of one design
  Grid g;
  const uint8_t* fixed;
  const float* Ek;          // fine level: FP32 moduli
  const float* S;           // coarse levels: FP32 nodal stencil [9*4][nnode]
  const float* dinv;
  const float* coef;        // smoother coefficients [2 * kMaxSmoothSteps]
  float *b, *z, *t, *r;     // V-cycle vectors [nrhs][n]
  float *dA, *dB;           // Chebyshev increments (null for damped Jacobi)
};

struct BDesign {
  int L;                    // multigrid levels
  int64_t nc;               // DOFs of the coarsest level
  const float* Ainv;        // coarsest dense inverse (FP32) [nc][nc]
  const double* Ek;         // fine FP64 moduli (outer CG operator)
  const double* b;          // right-hand sides [nrhs][n] (packed batch input)
  double *x, *r, *z, *p0, *p1, *q;  // outer CG vectors [nrhs][n]
  double* sc;               // [nrhs][kScStride]
  double* partial;          // reduction partials, [nrhs][pstride]
  unsigned* counters;       // [kNumCounterSets][kMaxRhs]
  int64_t pstride;
  BLevel lv[kBatchMaxLevels];
};

struct BItem {
  int d;       // design
  int bx, by;  // block coordinates inside the design's level
  int local;   // index of the item among the design's items of this list
};

// ------------------------------------------------------------------------------------------------
// kernels (blockIdx.y = right-hand side, or RHS group for the stencil kernel)
// ------------------------------------------------------------------------------------------------
constexpr int kBElem = 4096;  // DOFs per item of the elementwise lists (16 per thread: few, long blocks)

__device__ __forceinline__ bool b_active(const BDesign& d, int rhs) { return d.sc[rhs * kScStride + SC_ACTIVE] != 0.0; }

template <typename T>
__device__ __forceinline__ T* b_sel(const BLevel& L, int sel) {
  if constexpr (sizeof(T) == 4) {
    switch (sel) {
      case 0: return (T*)L.z;
      case 1: return (T*)L.t;
      case 2: return (T*)L.dA;
      case 3: return (T*)L.dB;
      case 4: return (T*)L.b;
      default: return (T*)L.r;
    }
  }
  return nullptr;
}
enum { SEL_Z = 0, SEL_T = 1, SEL_DA = 2, SEL_DB = 3, SEL_NONE = -1 };

// lv[0].b = (float) x_cg.r  (cast of the outer residual into the V-cycle)
__global__ void __launch_bounds__(256) kb_to32(const BDesign* __restrict__ D, const BItem* __restrict__ items, int nitems) {
  const int rhs = blockIdx.y;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    if (!b_active(d, rhs)) continue;
    const int64_t n = d.lv[0].g.n, off = (int64_t)rhs * n;
    for (int64_t i = (int64_t)w.bx * kBElem + threadIdx.x; i < n && i < (int64_t)(w.bx + 1) * kBElem; i += blockDim.x)
      d.lv[0].b[off + i] = (float)d.r[off + i];
  }
}

// x_cg.z = (double) result of the V-cycle on the fine level (buffer sel)
__global__ void __launch_bounds__(256) kb_to64(const BDesign* __restrict__ D, const BItem* __restrict__ items, int nitems,
                                               int sel) {
  const int rhs = blockIdx.y;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    if (!b_active(d, rhs)) continue;
    const int64_t n = d.lv[0].g.n, off = (int64_t)rhs * n;
    const float* src = b_sel<float>(d.lv[0], sel);
    for (int64_t i = (int64_t)w.bx * kBElem + threadIdx.x; i < n && i < (int64_t)(w.bx + 1) * kBElem; i += blockDim.x)
      d.z[off + i] = (double)src[off + i];
  }
}

// First smoothing step from a zero guess at one depth: z = c_0[1] dinv b (and dA = z).
__global__ void __launch_bounds__(256) kb_jacobi0(const BDesign* __restrict__ D, const BItem* __restrict__ items, int nitems,
                                                  int depth) {
  const int rhs = blockIdx.y;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    if (!b_active(d, rhs)) continue;
    const BLevel& L = d.lv[depth];
    const int64_t n = L.g.n, off = (int64_t)rhs * n;
    const float c1 = L.coef[1];
    for (int64_t i = (int64_t)w.bx * kBElem + threadIdx.x; i < n && i < (int64_t)(w.bx + 1) * kBElem; i += blockDim.x) {
      const float zi = c1 * L.dinv[i] * L.b[off + i];
      L.z[off + i] = zi;
      if (L.dA) L.dA[off + i] = zi;
    }
  }
}

// Fine-level FP32 smoothing step / residual in factored Q4 form on TX x TY node tiles:
//   MODE APPLY_JAC: dst = src + dn, dn = coef[0] d_in + coef[1] dinv (b - K src), d_out = dn
//   MODE APPLY_RES: r = b - K src
template <int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX* TY) kb_fine_smooth(const BDesign* __restrict__ D, const BItem* __restrict__ items,
                                                         int nitems, Q4Consts<float> cst, int src_sel, int dst_sel,
                                                         int din_sel, int dout_sel, int coef_off) {
  constexpr int EX = TX + 1, EY = TY + 1, NX = TX + 2, NY = TY + 2;
  __shared__ float su[NY][NX], sv[NY][NX];
  __shared__ float fe[EY][EX][8];
  const int rhs = blockIdx.y;
  const int tid = threadIdx.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    if (!b_active(d, rhs)) continue;
    const BLevel& L = d.lv[0];
    const Grid g = L.g;
    const int64_t off = (int64_t)rhs * g.n;
    const float* src = b_sel<float>(L, src_sel) + off;
    const int x0 = w.bx * TX, y0 = w.by * TY;
    const int nnx = g.nn[0], nny = g.nn[1];
    for (int q = tid; q < NX * NY; q += TX * TY) {
      const int lx = q % NX, ly = q / NX;
      const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
      float a = 0.f, c = 0.f;
      if (gx >= 0 && gx < nnx && gy >= 0 && gy < nny) {
        const int64_t node = gx + (int64_t)nnx * gy;
        a = src[2 * node];
        c = src[2 * node + 1];
      }
      su[ly][lx] = a;
      sv[ly][lx] = c;
    }
    __syncthreads();
    for (int q = tid; q < EX * EY; q += TX * TY) {
      const int lx = q % EX, ly = q / EX;
      const int ex = x0 - 1 + lx, ey = y0 - 1 + ly;
      float f[8];
      if (ex >= 0 && ex < g.nel[0] && ey >= 0 && ey < g.nel[1]) {
        q4_forces<float>(su[ly][lx], su[ly][lx + 1], su[ly + 1][lx + 1], su[ly + 1][lx], sv[ly][lx], sv[ly][lx + 1],
                         sv[ly + 1][lx + 1], sv[ly + 1][lx], L.Ek[ex + (int64_t)g.nel[0] * ey], cst, f);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) fe[ly][lx][k] = f[k];
    }
    __syncthreads();
    const int tx = tid % TX, ty = tid / TX;
    const int X = x0 + tx, Y = y0 + ty;
    if (X < nnx && Y < nny) {
      const float fx = fe[ty][tx][4] + fe[ty][tx + 1][6] + fe[ty + 1][tx][2] + fe[ty + 1][tx + 1][0];
      const float fy = fe[ty][tx][5] + fe[ty][tx + 1][7] + fe[ty + 1][tx][3] + fe[ty + 1][tx + 1][1];
      const int64_t node = X + (int64_t)nnx * Y;
      const float acc[2] = {fx, fy};
      const float vloc[2] = {su[ty + 1][tx + 1], sv[ty + 1][tx + 1]};
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int64_t idx = 2 * node + c;
        if (MODE == APPLY_RES) {
          L.r[off + idx] = L.fixed[idx] ? 0.f : L.b[off + idx] - acc[c];
        } else {
          float out = 0.f;
          if (!L.fixed[idx]) {
            const float rr = L.dinv[idx] * (L.b[off + idx] - acc[c]);
            const float* din = din_sel >= 0 ? b_sel<float>(L, din_sel) : nullptr;
            const float dn = (din ? L.coef[coef_off] * din[off + idx] : 0.f) + L.coef[coef_off + 1] * rr;
            if (dout_sel >= 0) b_sel<float>(L, dout_sel)[off + idx] = dn;
            out = vloc[c] + dn;
          } else if (dout_sel >= 0) {
            b_sel<float>(L, dout_sel)[off + idx] = 0.f;
          }
          b_sel<float>(L, dst_sel)[off + idx] = out;
        }
      }
    }
    __syncthreads();
  }
}

// Coarse-level FP32 smoothing step / residual with the assembled 9-point stencil, R RHS per thread.
template <int MODE, int R>
__global__ void __launch_bounds__(256) kb_coarse_smooth(const BDesign* __restrict__ D, const BItem* __restrict__ items,
                                                        int nitems, int depth, int nrhs, int src_sel, int dst_sel,
                                                        int din_sel, int dout_sel, int coef_off) {
  const int r0 = blockIdx.y * R;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    bool any = false;
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (r0 + r < nrhs && b_active(d, r0 + r)) any = true;
    if (!any) continue;
    const BLevel& L = d.lv[depth];
    const Grid g = L.g;
    const int64_t node = (int64_t)w.bx * blockDim.x + threadIdx.x;
    if (node >= g.nnode) continue;
    const int i = (int)(node % g.nn[0]), j = (int)(node / g.nn[0]);
    const int64_t nn = g.nnode, n = g.n;
    const float* src = b_sel<float>(L, src_sel);
    float acc[R][2];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r][0] = acc[r][1] = 0.f;
#pragma unroll
    for (int nbr = 0; nbr < 9; ++nbr) {
      const int dx = nbr % 3 - 1, dy = nbr / 3 - 1;
      if (i + dx < 0 || i + dx >= g.nn[0] || j + dy < 0 || j + dy >= g.nn[1]) continue;
      const int64_t nb = node + dx + (int64_t)g.nn[0] * dy;
      float blk[2][2];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) blk[c][cc] = L.S[(int64_t)((nbr * 2 + c) * 2 + cc) * nn + node];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        if (r0 + r >= nrhs) break;
        const float* vr = src + (int64_t)(r0 + r) * n + 2 * nb;
        const float v0 = vr[0], v1 = vr[1];
        acc[r][0] += blk[0][0] * v0 + blk[0][1] * v1;
        acc[r][1] += blk[1][0] * v0 + blk[1][1] * v1;
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r0 + r >= nrhs) break;
      const int64_t off = (int64_t)(r0 + r) * n;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int64_t idx = 2 * node + c;
        if (MODE == APPLY_RES) {
          L.r[off + idx] = L.fixed[idx] ? 0.f : L.b[off + idx] - acc[r][c];
        } else {
          float out = 0.f;
          float dn = 0.f;
          if (!L.fixed[idx]) {
            const float rr = L.dinv[idx] * (L.b[off + idx] - acc[r][c]);
            const float* din = din_sel >= 0 ? b_sel<float>(L, din_sel) : nullptr;
            dn = (din ? L.coef[coef_off] * din[off + idx] : 0.f) + L.coef[coef_off + 1] * rr;
            out = src[off + idx] + dn;
          }
          if (dout_sel >= 0) b_sel<float>(L, dout_sel)[off + idx] = dn;
          b_sel<float>(L, dst_sel)[off + idx] = out;
        }
      }
    }
  }
}

// lv[depth+1].b = P^T lv[depth].r (masked), one coarse node per thread
__global__ void __launch_bounds__(256) kb_restrict(const BDesign* __restrict__ D, const BItem* __restrict__ items, int nitems,
                                                   int depth) {
  const int rhs = blockIdx.y;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    if (!b_active(d, rhs)) continue;
    const BLevel& F = d.lv[depth];
    const BLevel& C = d.lv[depth + 1];
    const int64_t cn = (int64_t)w.bx * blockDim.x + threadIdx.x;
    if (cn >= C.g.nnode) continue;
    const int I = (int)(cn % C.g.nn[0]), J = (int)(cn / C.g.nn[0]);
    const float* rf = F.r + (int64_t)rhs * F.g.n;
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int fj = 2 * J + dy;
      if (fj < 0 || fj >= F.g.nn[1]) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int fi = 2 * I + dx;
        if (fi < 0 || fi >= F.g.nn[0]) continue;
        const float wgt = (dx == 0 ? 1.f : 0.5f) * (dy == 0 ? 1.f : 0.5f);
        const int64_t fn = fi + (int64_t)F.g.nn[0] * fj;
        a0 += wgt * rf[2 * fn];
        a1 += wgt * rf[2 * fn + 1];
      }
    }
    float* bc = C.b + (int64_t)rhs * C.g.n;
    bc[2 * cn] = C.fixed[2 * cn] ? 0.f : a0;
    bc[2 * cn + 1] = C.fixed[2 * cn + 1] ? 0.f : a1;
  }
}

// lv[depth].sel += P (coarse result), one fine node per thread.  The coarse result is lv[depth+1].z
// on the design's coarsest level, else the buffer the coarse level's smoothing ended in.
__global__ void __launch_bounds__(256) kb_prolong(const BDesign* __restrict__ D, const BItem* __restrict__ items, int nitems,
                                                  int depth, int fine_sel, int coarse_sel) {
  const int rhs = blockIdx.y;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    if (!b_active(d, rhs)) continue;
    const BLevel& F = d.lv[depth];
    const BLevel& C = d.lv[depth + 1];
    const int64_t fn = (int64_t)w.bx * blockDim.x + threadIdx.x;
    if (fn >= F.g.nnode) continue;
    const int i = (int)(fn % F.g.nn[0]), j = (int)(fn / F.g.nn[0]);
    const float* zc = (depth + 1 == d.L - 1 ? C.z : b_sel<float>(C, coarse_sel)) + (int64_t)rhs * C.g.n;
    float* zf = b_sel<float>(F, fine_sel) + (int64_t)rhs * F.g.n;
    const int ix0 = i >> 1, ix1 = (i + 1) >> 1, iy0 = j >> 1, iy1 = (j + 1) >> 1;
    const float wx = (i & 1) ? 0.5f : 1.f, wy = (j & 1) ? 0.5f : 1.f;
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int by = 0; by < 2; ++by) {
      if (by == 1 && !(j & 1)) continue;
#pragma unroll
      for (int bx = 0; bx < 2; ++bx) {
        if (bx == 1 && !(i & 1)) continue;
        const int64_t cn = (bx ? ix1 : ix0) + (int64_t)C.g.nn[0] * (by ? iy1 : iy0);
        a0 += wx * wy * zc[2 * cn];
        a1 += wx * wy * zc[2 * cn + 1];
      }
    }
    if (!F.fixed[2 * fn]) zf[2 * fn] += a0;
    if (!F.fixed[2 * fn + 1]) zf[2 * fn + 1] += a1;
  }
}

// Coarsest level of every design: z = Ainv b, one warp per row (items: 8 rows each).
__global__ void __launch_bounds__(256) kb_coarsest(const BDesign* __restrict__ D, const BItem* __restrict__ items, int nitems) {
  const int rhs = blockIdx.y;
  const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    if (!b_active(d, rhs)) continue;
    const BLevel& C = d.lv[d.L - 1];
    const int64_t row = (int64_t)w.bx * 8 + wrp, n = d.nc;
    if (row >= n) continue;
    const float* a = d.Ainv + row * n;
    const float* b = C.b + (int64_t)rhs * n;
    float s = 0.f;
    for (int64_t k = lane; k < n; k += 32) s += a[k] * b[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) C.z[(int64_t)rhs * n + row] = s;
  }
}

// ---- outer flexible CG (FP64), same recurrences and scalar slots as the single-design solver ----
template <int NV>
__device__ __forceinline__ bool b_reduce(const BDesign& d, int rhs, int slot, const BItem& w, int nlocal,
                                         double (&v)[NV], double (&tot)[NV], double* smem) {
  return grid_sum_last_idx<NV>(v, d.partial + (int64_t)rhs * d.pstride, d.counters + slot * kMaxRhs + rhs, tot, smem,
                               (unsigned)w.local, (unsigned)nlocal);
}

// x = 0, r = b (masked), b.b, r.r, scalar state (every (design, RHS) restarts)
__global__ void __launch_bounds__(256) kb_cg_init(const BDesign* __restrict__ D, const BItem* __restrict__ items, int nitems,
                                                  const int* __restrict__ nloc, double rtol) {
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    const BLevel& L = d.lv[0];
    const int64_t n = L.g.n, off = (int64_t)rhs * n;
    double v[1] = {0.0};
    for (int64_t i = (int64_t)w.bx * kBElem + threadIdx.x; i < n && i < (int64_t)(w.bx + 1) * kBElem; i += blockDim.x) {
      const double bi = L.fixed[i] ? 0.0 : d.b[off + i];
      d.r[off + i] = bi;
      d.x[off + i] = 0.0;
      d.p0[off + i] = 0.0;
      d.q[off + i] = 0.0;
      v[0] += bi * bi;
    }
    double tot[1];
    if (b_reduce<1>(d, rhs, 0, w, nloc[w.d], v, tot, smem) && threadIdx.x == 0) {
      double* s = d.sc + rhs * kScStride;
      for (int k = 0; k < kScStride; ++k) s[k] = 0.0;
      s[SC_BB] = tot[0];
      s[SC_RR] = tot[0];
      s[SC_RTOL] = rtol;
      s[SC_ZR_OLD] = 1.0;
      s[SC_PQ] = 1.0;
      s[SC_RELRES] = tot[0] > 0.0 ? 1.0 : 0.0;
      s[SC_ACTIVE] = tot[0] > 0.0 ? 1.0 : 0.0;
      if (!isfinite(tot[0])) {
        s[SC_STATUS] = 2.0;
        s[SC_ACTIVE] = 0.0;
      }
    }
    __syncthreads();
  }
}

// z.r, z.q_old, p_old.r and the flexible beta
__global__ void __launch_bounds__(256) kb_cg_dots(const BDesign* __restrict__ D, const BItem* __restrict__ items, int nitems,
                                                  const int* __restrict__ nloc, int pold) {
  __shared__ double smem[96];
  const int rhs = blockIdx.y;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    if (!b_active(d, rhs)) continue;
    const int64_t n = d.lv[0].g.n, off = (int64_t)rhs * n;
    const double* p = pold ? d.p1 : d.p0;
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t i = (int64_t)w.bx * kBElem + threadIdx.x; i < n && i < (int64_t)(w.bx + 1) * kBElem; i += blockDim.x) {
      const double zi = d.z[off + i], ri = d.r[off + i];
      v[0] += zi * ri;
      v[1] += zi * d.q[off + i];
      v[2] += p[off + i] * ri;
    }
    double tot[3];
    if (b_reduce<3>(d, rhs, 1, w, nloc[w.d], v, tot, smem) && threadIdx.x == 0) {
      double* s = d.sc + rhs * kScStride;
      const double zr = tot[0], zq = tot[1], pr = tot[2];
      const double beta = s[SC_ITERS] > 0.0 ? -zq / s[SC_PQ] : 0.0;
      s[SC_BETA] = beta;
      s[SC_ZR] = zr;
      s[SC_ZR_OLD] = zr;
      s[SC_PR] = zr + beta * pr;
      if (!isfinite(beta) || !isfinite(zr)) {
        s[SC_STATUS] = 2.0;
        s[SC_ACTIVE] = 0.0;
      }
    }
    __syncthreads();
  }
}

// p_new = z + beta p_old, q = K p_new (factored Q4, FP64), p.q and alpha; 32 x 8 node tiles
constexpr int kBTX = 32, kBTY = 8;
__global__ void __launch_bounds__(kBTX* kBTY) kb_cg_direction(const BDesign* __restrict__ D, const BItem* __restrict__ items,
                                                              int nitems, const int* __restrict__ nloc,
                                                              Q4Consts<double> cst, int pold) {
  constexpr int TX = kBTX, TY = kBTY, EX = TX + 1, EY = TY + 1, NX = TX + 2, NY = TY + 2;
  __shared__ double su[NY][NX], sv[NY][NX];
  __shared__ double fe[EY][EX][8];
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  const int tid = threadIdx.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    double* s = d.sc + rhs * kScStride;
    if (s[SC_ACTIVE] == 0.0) continue;
    const double beta = s[SC_BETA];
    const BLevel& L = d.lv[0];
    const Grid g = L.g;
    const int64_t off = (int64_t)rhs * g.n;
    const double* po = (pold ? d.p1 : d.p0) + off;
    double* pn = (pold ? d.p0 : d.p1) + off;
    const double* z = d.z + off;
    const int x0 = w.bx * TX, y0 = w.by * TY;
    const int nnx = g.nn[0], nny = g.nn[1];
    for (int t = tid; t < NX * NY; t += TX * TY) {
      const int lx = t % NX, ly = t / NX;
      const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
      double a = 0.0, c = 0.0;
      if (gx >= 0 && gx < nnx && gy >= 0 && gy < nny) {
        const int64_t i0 = 2 * (gx + (int64_t)nnx * gy);
        a = L.fixed[i0] ? 0.0 : z[i0] + beta * po[i0];
        c = L.fixed[i0 + 1] ? 0.0 : z[i0 + 1] + beta * po[i0 + 1];
      }
      su[ly][lx] = a;
      sv[ly][lx] = c;
    }
    __syncthreads();
    for (int t = tid; t < EX * EY; t += TX * TY) {
      const int lx = t % EX, ly = t / EX;
      const int ex = x0 - 1 + lx, ey = y0 - 1 + ly;
      double f[8];
      if (ex >= 0 && ex < g.nel[0] && ey >= 0 && ey < g.nel[1]) {
        q4_forces<double>(su[ly][lx], su[ly][lx + 1], su[ly + 1][lx + 1], su[ly + 1][lx], sv[ly][lx], sv[ly][lx + 1],
                          sv[ly + 1][lx + 1], sv[ly + 1][lx], d.Ek[ex + (int64_t)g.nel[0] * ey], cst, f);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) fe[ly][lx][k] = f[k];
    }
    __syncthreads();
    const int tx = tid % TX, ty = tid / TX;
    const int X = x0 + tx, Y = y0 + ty;
    double v[1] = {0.0};
    if (X < nnx && Y < nny) {
      const double fx = fe[ty][tx][4] + fe[ty][tx + 1][6] + fe[ty + 1][tx][2] + fe[ty + 1][tx + 1][0];
      const double fy = fe[ty][tx][5] + fe[ty][tx + 1][7] + fe[ty + 1][tx][3] + fe[ty + 1][tx + 1][1];
      const int64_t idx = 2 * (X + (int64_t)nnx * Y);
      const double px = su[ty + 1][tx + 1], py = sv[ty + 1][tx + 1];
      const double qx = L.fixed[idx] ? 0.0 : fx, qy = L.fixed[idx + 1] ? 0.0 : fy;
      pn[idx] = px;
      pn[idx + 1] = py;
      d.q[off + idx] = qx;
      d.q[off + idx + 1] = qy;
      v[0] = px * qx + py * qy;
    }
    double tot[1];
    if (b_reduce<1>(d, rhs, 2, w, nloc[w.d], v, tot, smem) && tid == 0) {
      const double pq = tot[0];
      s[SC_PQ] = pq;
      if (!(pq > 0.0) || !isfinite(pq)) {
        s[SC_STATUS] = 1.0;
        s[SC_ACTIVE] = 0.0;
        s[SC_ALPHA] = 0.0;
      } else {
        s[SC_ALPHA] = s[SC_PR] / pq;
      }
    }
    __syncthreads();
  }
}

// x += alpha p, r -= alpha q, r.r and the convergence test
__global__ void __launch_bounds__(256) kb_cg_update(const BDesign* __restrict__ D, const BItem* __restrict__ items, int nitems,
                                                    const int* __restrict__ nloc, int pnew) {
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    double* s = d.sc + rhs * kScStride;
    if (s[SC_ACTIVE] == 0.0) continue;
    const int64_t n = d.lv[0].g.n, off = (int64_t)rhs * n;
    const double alpha = s[SC_ALPHA];
    const double* p = pnew ? d.p1 : d.p0;
    double v[1] = {0.0};
    for (int64_t i = (int64_t)w.bx * kBElem + threadIdx.x; i < n && i < (int64_t)(w.bx + 1) * kBElem; i += blockDim.x) {
      d.x[off + i] += alpha * p[off + i];
      const double ri = d.r[off + i] - alpha * d.q[off + i];
      d.r[off + i] = ri;
      v[0] += ri * ri;
    }
    double tot[1];
    if (b_reduce<1>(d, rhs, 3, w, nloc[w.d], v, tot, smem) && threadIdx.x == 0) {
      s[SC_RR] = tot[0];
      const double rel = sqrt(tot[0] / s[SC_BB]);
      s[SC_RELRES] = rel;
      s[SC_ITERS] += 1.0;
      if (!isfinite(rel)) {
        s[SC_STATUS] = 2.0;
        s[SC_ACTIVE] = 0.0;
      } else if (rel <= s[SC_RTOL]) {
        s[SC_ACTIVE] = 0.0;
      }
    }
    __syncthreads();
  }
}

// True residual at exit: ||b - K x|| / ||b|| into sc[SC_RELRES] (FP64 factored Q4, 32 x 8 tiles).
__global__ void __launch_bounds__(kBTX* kBTY) kb_true_residual(const BDesign* __restrict__ D, const BItem* __restrict__ items,
                                                               int nitems, const int* __restrict__ nloc,
                                                               Q4Consts<double> cst) {
  constexpr int TX = kBTX, TY = kBTY, EX = TX + 1, EY = TY + 1, NX = TX + 2, NY = TY + 2;
  __shared__ double su[NY][NX], sv[NY][NX];
  __shared__ double fe[EY][EX][8];
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  const int tid = threadIdx.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const BItem w = items[it];
    const BDesign& d = D[w.d];
    const BLevel& L = d.lv[0];
    const Grid g = L.g;
    const int64_t off = (int64_t)rhs * g.n;
    const double* x = d.x + off;
    const int x0 = w.bx * TX, y0 = w.by * TY;
    const int nnx = g.nn[0], nny = g.nn[1];
    for (int t = tid; t < NX * NY; t += TX * TY) {
      const int lx = t % NX, ly = t / NX;
      const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
      double a = 0.0, c = 0.0;
      if (gx >= 0 && gx < nnx && gy >= 0 && gy < nny) {
        const int64_t i0 = 2 * (gx + (int64_t)nnx * gy);
        a = x[i0];
        c = x[i0 + 1];
      }
      su[ly][lx] = a;
      sv[ly][lx] = c;
    }
    __syncthreads();
    for (int t = tid; t < EX * EY; t += TX * TY) {
      const int lx = t % EX, ly = t / EX;
      const int ex = x0 - 1 + lx, ey = y0 - 1 + ly;
      double f[8];
      if (ex >= 0 && ex < g.nel[0] && ey >= 0 && ey < g.nel[1]) {
        q4_forces<double>(su[ly][lx], su[ly][lx + 1], su[ly + 1][lx + 1], su[ly + 1][lx], sv[ly][lx], sv[ly][lx + 1],
                          sv[ly + 1][lx + 1], sv[ly + 1][lx], d.Ek[ex + (int64_t)g.nel[0] * ey], cst, f);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) f[k] = 0.0;
      }
#pragma unroll
      for (int k = 0; k < 8; ++k) fe[ly][lx][k] = f[k];
    }
    __syncthreads();
    const int tx = tid % TX, ty = tid / TX;
    const int X = x0 + tx, Y = y0 + ty;
    double v[2] = {0.0, 0.0};
    if (X < nnx && Y < nny) {
      const double fx = fe[ty][tx][4] + fe[ty][tx + 1][6] + fe[ty + 1][tx][2] + fe[ty + 1][tx + 1][0];
      const double fy = fe[ty][tx][5] + fe[ty][tx + 1][7] + fe[ty + 1][tx][3] + fe[ty + 1][tx + 1][1];
      const int64_t idx = 2 * (X + (int64_t)nnx * Y);
      const double bx = L.fixed[idx] ? 0.0 : d.b[off + idx], by = L.fixed[idx + 1] ? 0.0 : d.b[off + idx + 1];
      const double rx = L.fixed[idx] ? 0.0 : bx - fx, ry = L.fixed[idx + 1] ? 0.0 : by - fy;
      v[0] = rx * rx + ry * ry;
      v[1] = bx * bx + by * by;
    }
    double tot[2];
    if (b_reduce<2>(d, rhs, 0, w, nloc[w.d], v, tot, smem) && tid == 0) {
      double* s = d.sc + rhs * kScStride;
      s[SC_RR] = tot[0];
      s[SC_BB] = tot[1];
      s[SC_RELRES] = tot[1] > 0.0 ? sqrt(tot[0] / tot[1]) : sqrt(tot[0]);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
namespace {

struct WorkList {
  BItem* items = nullptr;  // device
  int* nloc = nullptr;     // device, items per design
  int count = 0;
};

// Variants the autotuner chooses between.
constexpr int kFineVariants = 4;   // node tiles 32x8, 32x4, 64x4, 16x16 of the FP32 fine smoother
constexpr int kCoarseVariants = 3; // 1, 2, 4 right-hand sides per thread in the coarse stencil kernel
const int kFineTX[kFineVariants] = {32, 32, 64, 16};
const int kFineTY[kFineVariants] = {8, 4, 4, 16};

}  // namespace
}  // namespace tobk

struct tobk_batch {
  int nd = 0, nrhs = 1, dim = 2, Lmax = 1;
  tobk_desc desc0{};
  cudaStream_t stream = nullptr;
  std::vector<tobk_handle*> h;
  std::vector<int64_t> dof_off, elem_off;  // [nd + 1]
  // device memory owned by the batch
  char* arena = nullptr;
  tobk::BDesign* dD = nullptr;
  double *B = nullptr, *X = nullptr;  // packed [design][rhs][n_d]
  double* sc = nullptr;               // [nd][nrhs][kScStride]
  double* host_sc = nullptr;          // pinned
  std::vector<float*> ainv32;
  // work lists
  tobk::WorkList vec0;                              // fine DOF chunks (outer CG, casts)
  tobk::WorkList cgtile;                            // fine 32x8 FP64 tiles (CG direction, residual)
  tobk::WorkList fine[tobk::kFineVariants];         // fine FP32 smoother tiles per variant
  std::vector<tobk::WorkList> elem;                 // [depth] DOF chunks of designs smoothing at depth
  std::vector<tobk::WorkList> nodes;                // [depth] node blocks of designs smoothing at depth
  std::vector<tobk::WorkList> rnodes;               // [depth] coarse node blocks (restriction into depth+1)
  tobk::WorkList coarsest;                          // row blocks of every design's coarsest level
  std::vector<char*> list_mem;
  int fine_variant = 0, coarse_variant = 2;
  bool tuned = false, have_designs = false;
  cudaGraphExec_t graph = nullptr;
  long long graph_kernels = 0;
  int sm_count = 152;
  std::string err;
};

namespace tobk {
namespace {

int bfail(tobk_batch* b, int code, const std::string& m) {
  b->err = m;
  return code;
}

unsigned grid_cap(const tobk_batch* b, int count, int per_sm) {
  return (unsigned)std::max(1, std::min(count, per_sm * b->sm_count));
}

WorkList upload_list(tobk_batch* b, const std::vector<BItem>& items, const std::vector<int>& nloc) {
  WorkList w;
  w.count = (int)items.size();
  const size_t bytes = sizeof(BItem) * std::max<size_t>(1, items.size()) + sizeof(int) * nloc.size();
  char* mem = nullptr;
  if (cudaMalloc(&mem, bytes) != cudaSuccess) return w;
  b->list_mem.push_back(mem);
  w.items = reinterpret_cast<BItem*>(mem);
  w.nloc = reinterpret_cast<int*>(mem + sizeof(BItem) * std::max<size_t>(1, items.size()));
  if (!items.empty()) cudaMemcpy(w.items, items.data(), sizeof(BItem) * items.size(), cudaMemcpyHostToDevice);
  cudaMemcpy(w.nloc, nloc.data(), sizeof(int) * nloc.size(), cudaMemcpyHostToDevice);
  return w;
}

// items over DOF chunks of level `depth` of the designs selected by take(d)
template <class F>
WorkList chunk_list(tobk_batch* b, int depth, F take) {
  std::vector<BItem> it;
  std::vector<int> nloc(b->nd, 0);
  for (int d = 0; d < b->nd; ++d) {
    if (!take(d)) continue;
    const int64_t n = b->h[d]->lv[depth].g.n;
    for (int64_t c = 0; c * kBElem < n; ++c) it.push_back({d, (int)c, 0, nloc[d]++});
  }
  return upload_list(b, it, nloc);
}

template <class F>
WorkList node_list(tobk_batch* b, int depth, F take) {
  std::vector<BItem> it;
  std::vector<int> nloc(b->nd, 0);
  for (int d = 0; d < b->nd; ++d) {
    if (!take(d)) continue;
    const int64_t nn = b->h[d]->lv[depth].g.nnode;
    for (int64_t c = 0; c * 256 < nn; ++c) it.push_back({d, (int)c, 0, nloc[d]++});
  }
  return upload_list(b, it, nloc);
}

WorkList tile_list(tobk_batch* b, int tx, int ty) {
  std::vector<BItem> it;
  std::vector<int> nloc(b->nd, 0);
  for (int d = 0; d < b->nd; ++d) {
    const Grid& g = b->h[d]->lv[0].g;
    for (int y = 0; y * ty < g.nn[1]; ++y)
      for (int x = 0; x * tx < g.nn[0]; ++x) it.push_back({d, x, y, nloc[d]++});
  }
  return upload_list(b, it, nloc);
}

template <int TX, int TY>
void launch_fine_variant(tobk_batch* b, const WorkList& w, int mode, int src, int dst, int din, int dout, int coef_off,
                         const Q4Consts<float>& cst) {
  dim3 grid(grid_cap(b, w.count, 2048 / (TX * TY)), b->nrhs);
  note_launch();
  if (mode == APPLY_RES)
    kb_fine_smooth<TX, TY, APPLY_RES><<<grid, TX * TY, 0, b->stream>>>(b->dD, w.items, w.count, cst, src, dst, din, dout,
                                                                      coef_off);
  else
    kb_fine_smooth<TX, TY, APPLY_JAC><<<grid, TX * TY, 0, b->stream>>>(b->dD, w.items, w.count, cst, src, dst, din, dout,
                                                                      coef_off);
}

void launch_fine(tobk_batch* b, int variant, int mode, int src, int dst, int din, int dout, int coef_off) {
  const Q4Consts<float> cst = q4_consts<float>(b->h[0]->tab.Ke0.data());
  const WorkList& w = b->fine[variant];
  switch (variant) {
    case 0: launch_fine_variant<32, 8>(b, w, mode, src, dst, din, dout, coef_off, cst); break;
    case 1: launch_fine_variant<32, 4>(b, w, mode, src, dst, din, dout, coef_off, cst); break;
    case 2: launch_fine_variant<64, 4>(b, w, mode, src, dst, din, dout, coef_off, cst); break;
    default: launch_fine_variant<16, 16>(b, w, mode, src, dst, din, dout, coef_off, cst); break;
  }
}

template <int R>
void launch_coarse_r(tobk_batch* b, int depth, int mode, int src, int dst, int din, int dout, int coef_off) {
  const WorkList& w = b->nodes[depth];
  if (w.count == 0) return;
  dim3 grid(grid_cap(b, w.count, 8), (b->nrhs + R - 1) / R);
  note_launch();
  if (mode == APPLY_RES)
    kb_coarse_smooth<APPLY_RES, R><<<grid, 256, 0, b->stream>>>(b->dD, w.items, w.count, depth, b->nrhs, src, dst, din,
                                                                dout, coef_off);
  else
    kb_coarse_smooth<APPLY_JAC, R><<<grid, 256, 0, b->stream>>>(b->dD, w.items, w.count, depth, b->nrhs, src, dst, din,
                                                                dout, coef_off);
}

void launch_coarse(tobk_batch* b, int variant, int depth, int mode, int src, int dst, int din, int dout, int coef_off) {
  switch (variant) {
    case 0: launch_coarse_r<1>(b, depth, mode, src, dst, din, dout, coef_off); break;
    case 1: launch_coarse_r<2>(b, depth, mode, src, dst, din, dout, coef_off); break;
    default: launch_coarse_r<4>(b, depth, mode, src, dst, din, dout, coef_off); break;
  }
}

void launch_smooth(tobk_batch* b, int depth, int mode, int src, int dst, int din, int dout, int coef_off) {
  if (depth == 0)
    launch_fine(b, b->fine_variant, mode, src, dst, din, dout, coef_off);
  else
    launch_coarse(b, b->coarse_variant, depth, mode, src, dst, din, dout, coef_off);
}

// One V-cycle of every design on its FP32 hierarchy: lv[0].b -> result buffer of level 0 (returned
// selector).  The buffer roles follow the same sequence as the single-design vcycle32.
int enqueue_vcycle(tobk_batch* b) {
  cudaStream_t s = b->stream;
  const int npre = b->desc0.nu_pre, npost = b->desc0.nu_post;
  const bool cheb = b->desc0.smoother == TOBK_SMOOTHER_CHEBYSHEV;
  const int Jm = b->Lmax - 1;  // depths that smooth: 0 .. Jm-1
  std::vector<int> cur(Jm, SEL_Z), dA(Jm, SEL_DA), dB(Jm, SEL_DB);
  for (int j = 0; j < Jm; ++j) {
    const WorkList& e = b->elem[j];
    if (e.count == 0) continue;
    note_launch();
    kb_jacobi0<<<dim3(grid_cap(b, e.count, 8), b->nrhs), 256, 0, s>>>(b->dD, e.items, e.count, j);
    int z = SEL_Z, t = SEL_T, a = SEL_DA, bb = SEL_DB;
    for (int it = 1; it < npre; ++it) {
      launch_smooth(b, j, APPLY_JAC, z, t, cheb ? a : SEL_NONE, cheb ? bb : SEL_NONE, 2 * it);
      std::swap(z, t);
      std::swap(a, bb);
    }
    launch_smooth(b, j, APPLY_RES, z, z, SEL_NONE, SEL_NONE, 0);
    const WorkList& r = b->rnodes[j];
    note_launch();
    kb_restrict<<<dim3(grid_cap(b, r.count, 8), b->nrhs), 256, 0, s>>>(b->dD, r.items, r.count, j);
    cur[j] = z;
    dA[j] = a;
    dB[j] = bb;
  }
  note_launch();
  kb_coarsest<<<dim3(grid_cap(b, b->coarsest.count, 8), b->nrhs), 256, 0, s>>>(b->dD, b->coarsest.items,
                                                                              b->coarsest.count);
  const int coarse_sel = ((npre - 1 + npost) & 1) ? SEL_T : SEL_Z;  // where a smoothed level's result ends
  for (int j = Jm - 1; j >= 0; --j) {
    const WorkList& nl = b->nodes[j];
    if (nl.count == 0) continue;
    int z = cur[j], t = z == SEL_Z ? SEL_T : SEL_Z, a = dA[j], bb = dB[j];
    note_launch();
    kb_prolong<<<dim3(grid_cap(b, nl.count, 8), b->nrhs), 256, 0, s>>>(b->dD, nl.items, nl.count, j, z, coarse_sel);
    for (int it = 0; it < npost; ++it) {
      launch_smooth(b, j, APPLY_JAC, z, t, (cheb && it > 0) ? a : SEL_NONE, cheb ? bb : SEL_NONE, 2 * it);
      std::swap(z, t);
      std::swap(a, bb);
    }
    cur[j] = z;
  }
  return cur[0];
}

void enqueue_cg_pair(tobk_batch* b) {
  cudaStream_t s = b->stream;
  const Q4Consts<double> cst = q4_consts<double>(b->h[0]->tab.Ke0.data());
  const WorkList& v = b->vec0;
  const WorkList& t = b->cgtile;
  for (int k = 0; k < 2; ++k) {
    const int pold = k;  // iteration 0: p_old = p0 -> p_new = p1; iteration 1: the reverse
    note_launch();
    kb_to32<<<dim3(grid_cap(b, v.count, 8), b->nrhs), 256, 0, s>>>(b->dD, v.items, v.count);
    const int zsel = enqueue_vcycle(b);
    note_launch();
    kb_to64<<<dim3(grid_cap(b, v.count, 8), b->nrhs), 256, 0, s>>>(b->dD, v.items, v.count, zsel);
    note_launch();
    kb_cg_dots<<<dim3(v.count, b->nrhs), 256, 0, s>>>(b->dD, v.items, v.count, v.nloc, pold);
    note_launch();
    kb_cg_direction<<<dim3(t.count, b->nrhs), kBTX * kBTY, 0, s>>>(b->dD, t.items, t.count, t.nloc, cst, pold);
    note_launch();
    kb_cg_update<<<dim3(v.count, b->nrhs), 256, 0, s>>>(b->dD, v.items, v.count, v.nloc, 1 - pold);
  }
}

void destroy_graph(tobk_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

int run_pair(tobk_batch* b) {
  if (b->stream == nullptr) {  // the legacy default stream cannot be captured: launch directly
    enqueue_cg_pair(b);
    return TOBK_OK;
  }
  if (!b->graph) {
    cudaGraph_t g = nullptr;
    const long long c0 = g_launch_count.load();
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return bfail(b, TOBK_E_CUDA, "batch graph capture failed");
    enqueue_cg_pair(b);
    if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess) return bfail(b, TOBK_E_CUDA, "batch graph capture failed");
    b->graph_kernels = g_launch_count.load() - c0;
    g_launch_count.fetch_sub(b->graph_kernels);
    if (cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      return bfail(b, TOBK_E_CUDA, "batch graph instantiate failed");
    }
    cudaGraphDestroy(g);
  }
  cudaGraphLaunch(b->graph, b->stream);
  g_launch_count.fetch_add(b->graph_kernels);
  return TOBK_OK;
}

}  // namespace
}  // namespace tobk

using namespace tobk;

extern "C" {

int tobk_batch_create(const tobk_desc* descs, int ndesigns, int nrhs, void* cuda_stream, tobk_batch** out) {
  if (!descs || !out || ndesigns < 1 || nrhs < 1 || nrhs > kMaxRhs) return TOBK_E_ARG;
  *out = nullptr;
  const tobk_desc& d0 = descs[0];
  for (int d = 0; d < ndesigns; ++d) {
    const tobk_desc& dd = descs[d];
    if (dd.dim != 2 || dd.nu != d0.nu || dd.nu_pre != d0.nu_pre || dd.nu_post != d0.nu_post ||
        dd.smoother != d0.smoother || dd.mg_levels < 2 || dd.mg_levels > kBatchMaxLevels)
      return TOBK_E_ARG;
  }
  tobk_batch* b = new tobk_batch();
  b->nd = ndesigns;
  b->nrhs = nrhs;
  b->desc0 = d0;
  b->stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
  b->dof_off.assign(ndesigns + 1, 0);
  b->elem_off.assign(ndesigns + 1, 0);
  for (int d = 0; d < ndesigns; ++d) {
    tobk_desc dd = descs[d];
    dd.precision = TOBK_FP32_VCYCLE;
    dd.max_rhs = std::max(dd.max_rhs, nrhs);
    dd.num_modes = 1;
    dd.eig_level = 1;
    tobk_handle* h = nullptr;
    const int rc = create_handle(&dd, cuda_stream, &h, true);
    if (rc != TOBK_OK) {
      for (auto* x : b->h) destroy_handle(x);
      delete b;
      return rc;
    }
    b->h.push_back(h);
    b->dof_off[d + 1] = b->dof_off[d] + h->lv[0].g.n;
    b->elem_off[d + 1] = b->elem_off[d] + h->lv[0].g.m;
    b->Lmax = std::max(b->Lmax, h->L);
  }
  // batch-owned device memory: design table, packed B and X, scalar state, FP32 coarsest inverses
  const int64_t ntot = b->dof_off[ndesigns];
  size_t bytes = sizeof(BDesign) * ndesigns + 2 * sizeof(double) * nrhs * ntot +
                 sizeof(double) * (size_t)ndesigns * nrhs * kScStride + 256 * 8;
  for (auto* h : b->h) bytes += sizeof(float) * (size_t)h->lv[h->L - 1].g.n * h->lv[h->L - 1].g.n + 256;
  if (cudaMalloc(&b->arena, bytes) != cudaSuccess || cudaMallocHost(&b->host_sc, sizeof(double) * ndesigns * nrhs * kScStride) != cudaSuccess) {
    cudaGetLastError();
    tobk_batch_destroy(b);
    return TOBK_E_NOMEM;
  }
  Arena a;
  a.base = b->arena;
  a.cap = bytes;
  b->dD = a.take<BDesign>(ndesigns);
  b->B = a.take<double>((size_t)nrhs * ntot);
  b->X = a.take<double>((size_t)nrhs * ntot);
  b->sc = a.take<double>((size_t)ndesigns * nrhs * kScStride);
  for (auto* h : b->h) b->ainv32.push_back(a.take<float>((size_t)h->lv[h->L - 1].g.n * h->lv[h->L - 1].g.n));
  cudaMemsetAsync(b->sc, 0, sizeof(double) * ndesigns * nrhs * kScStride, b->stream);
  // design table (pointers into the member handles)
  std::vector<BDesign> hd(ndesigns);
  for (int d = 0; d < ndesigns; ++d) {
    tobk_handle* h = b->h[d];
    BDesign& D = hd[d];
    std::memset(&D, 0, sizeof(D));
    D.L = h->L;
    D.nc = h->lv[h->L - 1].g.n;
    D.Ainv = b->ainv32[d];
    D.Ek = h->Ek;
    D.b = b->B + (size_t)nrhs * b->dof_off[d];
    D.x = h->cg.x;
    D.r = h->cg.r;
    D.z = h->cg.z;
    D.p0 = h->cg.p0;
    D.p1 = h->cg.p1;
    D.q = h->cg.q;
    D.sc = b->sc + (size_t)d * nrhs * kScStride;
    D.partial = h->cg.partial;
    D.counters = h->cg.counters;
    D.pstride = cg_partial_stride(h->lv[0].g);
    for (int j = 0; j < h->L; ++j) {
      const Level& L = h->lv[j];
      BLevel& B = D.lv[j];
      B.g = L.g;
      B.fixed = L.fixed;
      B.Ek = j == 0 ? h->Ek32 : nullptr;
      B.S = L.S32;
      B.dinv = L.dinv32;
      B.coef = L.coef32;
      B.b = L.b32;
      B.z = L.z32;
      B.t = L.t32;
      B.r = L.r32;
      B.dA = L.dA32;
      B.dB = L.dB32;
    }
  }
  cudaMemcpyAsync(b->dD, hd.data(), sizeof(BDesign) * ndesigns, cudaMemcpyHostToDevice, b->stream);
  // work lists
  b->vec0 = chunk_list(b, 0, [](int) { return true; });
  b->cgtile = tile_list(b, kBTX, kBTY);
  for (int v = 0; v < kFineVariants; ++v) b->fine[v] = tile_list(b, kFineTX[v], kFineTY[v]);
  for (int j = 0; j + 1 < b->Lmax; ++j) {
    auto smooths = [b, j](int d) { return j < b->h[d]->L - 1; };
    b->elem.push_back(chunk_list(b, j, smooths));
    b->nodes.push_back(node_list(b, j, smooths));
    // restriction into level j+1: coarse node blocks
    std::vector<BItem> it;
    std::vector<int> nloc(b->nd, 0);
    for (int d = 0; d < b->nd; ++d) {
      if (!smooths(d)) continue;
      const int64_t nn = b->h[d]->lv[j + 1].g.nnode;
      for (int64_t c = 0; c * 256 < nn; ++c) it.push_back({d, (int)c, 0, nloc[d]++});
    }
    b->rnodes.push_back(upload_list(b, it, nloc));
  }
  {
    std::vector<BItem> it;
    std::vector<int> nloc(b->nd, 0);
    for (int d = 0; d < b->nd; ++d) {
      const int64_t nc = b->h[d]->lv[b->h[d]->L - 1].g.n;
      for (int64_t c = 0; c * 8 < nc; ++c) it.push_back({d, (int)c, 0, nloc[d]++});
    }
    b->coarsest = upload_list(b, it, nloc);
  }
  cudaStreamSynchronize(b->stream);
  if (cudaGetLastError() != cudaSuccess) {
    tobk_batch_destroy(b);
    return TOBK_E_CUDA;
  }
  *out = b;
  return TOBK_OK;
}

void tobk_batch_destroy(tobk_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  destroy_graph(b);
  for (char* m : b->list_mem) cudaFree(m);
  for (auto* h : b->h) destroy_handle(h);
  if (b->arena) cudaFree(b->arena);
  if (b->host_sc) cudaFreeHost(b->host_sc);
  delete b;
}

const char* tobk_batch_last_error(const tobk_batch* b) { return b ? b->err.c_str() : "null batch"; }

int tobk_batch_layout(const tobk_batch* b, int64_t* dof_offsets, int64_t* elem_offsets) {
  if (!b) return TOBK_E_ARG;
  for (int d = 0; d <= b->nd; ++d) {
    if (dof_offsets) dof_offsets[d] = b->dof_off[d];
    if (elem_offsets) elem_offsets[d] = b->elem_off[d];
  }
  return TOBK_OK;
}

int tobk_batch_set_designs(tobk_batch* b, const double* x, const uint8_t* fixed, int on_device) {
  if (!b || !x || !fixed) return TOBK_E_ARG;
  for (int d = 0; d < b->nd; ++d) {
    tobk_handle* h = b->h[d];
    int rc = set_fixed(h, fixed + b->dof_off[d], on_device != 0);
    if (!rc) rc = set_densities(h, x + b->elem_off[d], on_device != 0);
    if (!rc) rc = setup_hierarchy(h);
    if (rc) return bfail(b, rc, "design " + std::to_string(d) + ": " + h->err);
    const int64_t nc = h->lv[h->L - 1].g.n;
    launch_f64_to_f32(h->Ainv, b->ainv32[d], nc * nc, b->stream);
  }
  if (cudaGetLastError() != cudaSuccess) return bfail(b, TOBK_E_CUDA, "set_designs: launch failed");
  b->have_designs = true;
  return TOBK_OK;
}

int tobk_batch_solve(tobk_batch* b, const double* B, double* X, int on_device, tobk_solve_info* infos) {
  if (!b || !B || !X) return TOBK_E_ARG;
  if (!b->have_designs) return bfail(b, TOBK_E_STATE, "designs not set");
  cudaStream_t s = b->stream;
  const int64_t ntot = b->dof_off[b->nd];
  const size_t vbytes = sizeof(double) * b->nrhs * ntot;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaMemcpyAsync(b->B, B, vbytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  const double rtol = b->desc0.rtol;
  const int max_iter = b->desc0.max_iter;
  const WorkList& v = b->vec0;
  note_launch();
  kb_cg_init<<<dim3(v.count, b->nrhs), 256, 0, s>>>(b->dD, v.items, v.count, v.nloc, rtol);
  const size_t scb = sizeof(double) * b->nd * b->nrhs * kScStride;
  int pairs = 0, rc = TOBK_OK;
  while (2 * pairs < max_iter) {
    rc = run_pair(b);
    if (rc) break;
    ++pairs;
    cudaMemcpyAsync(b->host_sc, b->sc, scb, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    bool any = false;
    for (int k = 0; k < b->nd * b->nrhs; ++k) any |= b->host_sc[(size_t)k * kScStride + SC_ACTIVE] != 0.0;
    if (!any) break;
  }
  const int64_t status_iters = 2 * pairs;
  std::vector<double> iters(b->nd * b->nrhs), status(b->nd * b->nrhs);
  for (int k = 0; k < b->nd * b->nrhs; ++k) {
    iters[k] = b->host_sc[(size_t)k * kScStride + SC_ITERS];
    status[k] = b->host_sc[(size_t)k * kScStride + SC_STATUS];
  }
  // true residuals at exit and the packed solution
  const WorkList& t = b->cgtile;
  const Q4Consts<double> cst = q4_consts<double>(b->h[0]->tab.Ke0.data());
  note_launch();
  kb_true_residual<<<dim3(t.count, b->nrhs), kBTX * kBTY, 0, s>>>(b->dD, t.items, t.count, t.nloc, cst);
  for (int d = 0; d < b->nd; ++d)
    cudaMemcpyAsync(b->X + (size_t)b->nrhs * b->dof_off[d], b->h[d]->cg.x, sizeof(double) * b->nrhs * b->h[d]->lv[0].g.n,
                    cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(X, b->X, vbytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(b->host_sc, b->sc, scb, cudaMemcpyDeviceToHost, s);
  cudaEventRecord(e1, s);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return bfail(b, TOBK_E_CUDA, "batch solve: CUDA error");
  bool all_conv = true;
  int worst_status = 0;
  for (int d = 0; d < b->nd; ++d) {
    double worst = 0.0;
    int it = 0;
    bool conv = true;
    for (int r = 0; r < b->nrhs; ++r) {
      const size_t k = (size_t)d * b->nrhs + r;
      const double rel = b->host_sc[k * kScStride + SC_RELRES];
      worst = std::max(worst, std::isfinite(rel) ? rel : INFINITY);
      it = std::max(it, (int)iters[k]);
      worst_status = std::max(worst_status, (int)status[k]);
      if (!(rel <= rtol)) conv = false;
    }
    all_conv &= conv;
    if (infos) {
      infos[d].iterations = it;
      infos[d].converged = conv ? 1 : 0;
      infos[d].num_rhs = b->nrhs;
      infos[d].rel_residual = worst;
      infos[d].time_ms = ms;
      infos[d].status_detail = (int)status_iters;
    }
  }
  if (rc) return rc;
  if (worst_status == 1) return bfail(b, TOBK_E_BREAKDOWN, "CG breakdown: p^T K p <= 0");
  if (worst_status == 2) return bfail(b, TOBK_E_NONFINITE, "non-finite value in CG");
  if (!all_conv) return bfail(b, TOBK_E_NOT_CONVERGED, "CG iteration limit reached (or true residual above rtol)");
  return TOBK_OK;
}

int tobk_batch_autotune(tobk_batch* b, int* fine_variant, int* coarse_variant) {
  if (!b) return TOBK_E_ARG;
  if (!b->have_designs) return bfail(b, TOBK_E_STATE, "designs not set");
  cudaStream_t s = b->stream;
  // make every (design, RHS) active with a nonzero right-hand side in the V-cycle inputs
  std::vector<double> one((size_t)b->nd * b->nrhs * kScStride, 0.0);
  for (size_t k = 0; k < (size_t)b->nd * b->nrhs; ++k) one[k * kScStride + SC_ACTIVE] = 1.0;
  cudaMemcpyAsync(b->sc, one.data(), sizeof(double) * one.size(), cudaMemcpyHostToDevice, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int reps = 5;
  float best = 1e30f;
  for (int v = 0; v < kFineVariants; ++v) {
    for (int r = 0; r < 2; ++r) launch_fine(b, v, APPLY_RES, SEL_Z, SEL_Z, SEL_NONE, SEL_NONE, 0);  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps; ++r) launch_fine(b, v, APPLY_RES, SEL_Z, SEL_Z, SEL_NONE, SEL_NONE, 0);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      b->fine_variant = v;
    }
  }
  best = 1e30f;
  for (int v = 0; v < kCoarseVariants; ++v) {
    float total = 0.f;
    for (int j = 1; j < (int)b->nodes.size(); ++j) {
      for (int r = 0; r < 2; ++r) launch_coarse(b, v, j, APPLY_RES, SEL_Z, SEL_Z, SEL_NONE, SEL_NONE, 0);
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps; ++r) launch_coarse(b, v, j, APPLY_RES, SEL_Z, SEL_Z, SEL_NONE, SEL_NONE, 0);
      cudaEventRecord(e1, s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      total += ms;
    }
    if (total < best) {
      best = total;
      b->coarse_variant = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaMemsetAsync(b->sc, 0, sizeof(double) * one.size(), s);
  cudaStreamSynchronize(s);
  destroy_graph(b);  // the captured iteration used the previous choice
  b->tuned = true;
  if (fine_variant) *fine_variant = b->fine_variant;
  if (coarse_variant) *coarse_variant = b->coarse_variant;
  if (cudaGetLastError() != cudaSuccess) return bfail(b, TOBK_E_CUDA, "autotune: CUDA error");
  return TOBK_OK;
}

int tobk_batch_set_variants(tobk_batch* b, int fine_variant, int coarse_variant) {
  if (!b || fine_variant < 0 || fine_variant >= kFineVariants || coarse_variant < 0 || coarse_variant >= kCoarseVariants)
    return TOBK_E_ARG;
  b->fine_variant = fine_variant;
  b->coarse_variant = coarse_variant;
  destroy_graph(b);
  return TOBK_OK;
}

}  // extern "C"
