// Coarse-level operators as assembled nodal stencils.
//
// On a Galerkin level (Sec. 2.1 step 1) the operator K^j is stored element by element.  For the
// smoother and residual sweeps it is cheaper to assemble it once per design into a 3^d-point stencil
// of d x d blocks per node: a row then costs 3^d d^2 multiply-adds (36 in 2D, 243 in 3D) instead of
// the 2^d d (d 2^d) of the element form (64 / 576), and the stencil is read once for a chunk of
// right-hand sides.  Layout (structure of arrays, coalesced across nodes):
//     S[((nbr * d + c) * d + c') * nnode + node],  nbr = (dx+1) + 3 (dy+1) [+ 9 (dz+1)].
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace tobk {

template <int DIM>
struct StencilDims {
  static constexpr int NB = DIM == 2 ? 9 : 27;
  static constexpr int NE = NB * DIM * DIM;
};

template <int DIM>
__global__ void k_stencil_assemble(Grid g, const double* __restrict__ Ke, const uint8_t* __restrict__ fixed,
                                   double* __restrict__ S, float* __restrict__ S32) {
  constexpr int NN = Dims<DIM>::NN, ND = Dims<DIM>::ND, NE = StencilDims<DIM>::NE;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(g, node, i, j, k)) return;
  const int64_t nn = g.nnode;
  for (int q = 0; q < NE; ++q) S[(int64_t)q * nn + node] = 0.0;
  for (int cz = 0; cz < (DIM == 3 ? 2 : 1); ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        const int ei = i - cx, ej = j - cy, ek = k - cz;
        if (ei < 0 || ei >= g.nel[0] || ej < 0 || ej >= g.nel[1]) continue;
        if (DIM == 3 && (ek < 0 || ek >= g.nel[2])) continue;
        const int64_t e = ei + (int64_t)g.nel[0] * (ej + (int64_t)g.nel[1] * ek);
        const int ln = local_node(cx, cy, cz);
        for (int lb = 0; lb < NN; ++lb) {
          const int dx = corner_x(lb) - cx, dy = corner_y(lb) - cy, dz = corner_z(lb) - cz;
          const int nbr = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
          const int64_t nb = node + dx + (int64_t)g.nn[0] * (dy + (int64_t)g.nn[1] * dz);
          for (int c = 0; c < DIM; ++c)
            for (int cc = 0; cc < DIM; ++cc) {
              if (fixed[DIM * node + c] || fixed[DIM * nb + cc]) continue;
              S[(int64_t)((nbr * DIM + c) * DIM + cc) * nn + node] += Ke[e * ND * ND + (ln * DIM + c) * ND + lb * DIM + cc];
            }
        }
      }
  if (S32)
    for (int q = 0; q < NE; ++q) S32[(int64_t)q * nn + node] = (float)S[(int64_t)q * nn + node];
}

void launch_stencil_assemble(const Grid& g, const double* Ke, const uint8_t* fixed, double* S, float* S32,
                             cudaStream_t s) {
  const unsigned grid = (unsigned)((g.nnode + 127) / 128);
  note_launch();
  if (g.dim == 2)
    k_stencil_assemble<2><<<grid, 128, 0, s>>>(g, Ke, fixed, S, S32);
  else
    k_stencil_assemble<3><<<grid, 128, 0, s>>>(g, Ke, fixed, S, S32);
}

// y = K v | b - K v | v + omega dinv (b - K v) for R right-hand sides per thread.
template <int DIM, typename T, int MODE, int R>
__global__ void __launch_bounds__(256) k_apply_stencil(Grid g, const T* __restrict__ S, const uint8_t* __restrict__ fixed,
                                                       const T* __restrict__ v, const T* __restrict__ b,
                                                       const T* __restrict__ dinv, T* __restrict__ y, SmoothArgs<T> sm,
                                                       int nr, int64_t stride, const double* __restrict__ act) {
  pdl_wait();
  constexpr int NB = StencilDims<DIM>::NB;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(g, node, i, j, k)) return;
  const int r0 = blockIdx.y * R;
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r0 + r < nr && !(act && act[(size_t)(r0 + r) * kScStride + SC_ACTIVE] == 0.0)) any = true;
  if (!any) return;
  const int64_t nn = g.nnode;
  T acc[R][DIM];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[r][c] = T(0);
  // straight-line neighbour loop: a neighbour outside the grid reads the node itself and counts as
  // zero (its stencil coefficients are zero as well), so every load is unconditional and all of them
  // can be in flight together
#pragma unroll
  for (int nbr = 0; nbr < NB; ++nbr) {
    const int dx = nbr % 3 - 1, dy = (nbr / 3) % 3 - 1, dz = DIM == 3 ? nbr / 9 - 1 : 0;
    const bool in = i + dx >= 0 && i + dx < g.nn[0] && j + dy >= 0 && j + dy < g.nn[1] &&
                    (DIM == 2 || (k + dz >= 0 && k + dz < g.nn[2]));
    const int64_t nb = in ? node + dx + (int64_t)g.nn[0] * (dy + (int64_t)g.nn[1] * dz) : node;
    T blk[DIM][DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int cc = 0; cc < DIM; ++cc) blk[c][cc] = __ldg(S + (int64_t)((nbr * DIM + c) * DIM + cc) * nn + node);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r0 + r >= nr) break;
      const T* vr = v + (int64_t)(r0 + r) * stride + DIM * nb;
#pragma unroll
      for (int cc = 0; cc < DIM; ++cc) {
        const T vv = in ? __ldg(vr + cc) : T(0);
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[r][c] += blk[c][cc] * vv;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (r0 + r >= nr) break;
    const int64_t off = (int64_t)(r0 + r) * stride;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t idx = DIM * node + c;
      T out;
      if (fixed[idx])
        out = T(0);
      else if (MODE == APPLY_KV)
        out = acc[r][c];
      else if (MODE == APPLY_RES)
        out = b[off + idx] - acc[r][c];
      else
      {
        const T rr = dinv[idx] * (b[off + idx] - acc[r][c]);
        const T dn = (sm.d_in ? sm.coef[0] * sm.d_in[off + idx] : T(0)) + sm.coef[1] * rr;
        if (sm.d_out) sm.d_out[off + idx] = dn;
        out = v[off + idx] + dn;
      }
      y[off + idx] = out;
    }
  }
}

template <int DIM, typename T, int R>
static void stencil_dispatch(const Grid& g, const T* S, const uint8_t* fixed, int mode, const T* v, const T* b,
                             const T* dinv, T* y, SmoothArgs<T> sm, int nr, int64_t stride, cudaStream_t s) {
  // 128-thread blocks: the FP64-bound sweeps of a level with many right-hand sides run at the pace of
  // the SM with the most blocks, and smaller blocks even out the count per SM
  constexpr int kTh = 128;
  dim3 grid((unsigned)((g.nnode + kTh - 1) / kTh), (unsigned)((nr + R - 1) / R));
  const double* act = active_rhs();
  if (mode == APPLY_KV)
    launch_pdl(k_apply_stencil<DIM, T, APPLY_KV, R>, grid, dim3(kTh), 0, s, g, S, fixed, v, b, dinv, y, sm, nr,
               stride, act);
  else if (mode == APPLY_RES)
    launch_pdl(k_apply_stencil<DIM, T, APPLY_RES, R>, grid, dim3(kTh), 0, s, g, S, fixed, v, b, dinv, y, sm, nr,
               stride, act);
  else
    launch_pdl(k_apply_stencil<DIM, T, APPLY_JAC, R>, grid, dim3(kTh), 0, s, g, S, fixed, v, b, dinv, y, sm, nr,
               stride, act);
}

// Right-hand sides per thread: reusing a stencil row across several RHS saves loads on large levels,
// while small levels need every thread they can get (one RHS per thread) to hide load latency.
template <typename T>
void launch_apply_stencil(const Grid& g, const T* S, const uint8_t* fixed, int mode, const T* v, const T* b,
                          const T* dinv, T* y, SmoothArgs<T> sm, int nr, int64_t stride, cudaStream_t s) {
  const int64_t work = g.nnode;
  if (g.dim == 2) {
    if (work <= 8192)
      stencil_dispatch<2, T, 1>(g, S, fixed, mode, v, b, dinv, y, sm, nr, stride, s);
    else if (work <= 32768)
      stencil_dispatch<2, T, 2>(g, S, fixed, mode, v, b, dinv, y, sm, nr, stride, s);
    else
      stencil_dispatch<2, T, 4>(g, S, fixed, mode, v, b, dinv, y, sm, nr, stride, s);
  } else {
    if (work <= 8192)
      stencil_dispatch<3, T, 1>(g, S, fixed, mode, v, b, dinv, y, sm, nr, stride, s);
    else
      stencil_dispatch<3, T, 2>(g, S, fixed, mode, v, b, dinv, y, sm, nr, stride, s);
  }
}

template void launch_apply_stencil<double>(const Grid&, const double*, const uint8_t*, int, const double*,
                                           const double*, const double*, double*, SmoothArgs<double>, int, int64_t,
                                           cudaStream_t);
template void launch_apply_stencil<float>(const Grid&, const float*, const uint8_t*, int, const float*, const float*,
                                          const float*, float*, SmoothArgs<float>, int, int64_t,
                                          cudaStream_t);

// ================================================================================================
// Transfers fused into the stencil sweeps of 2D levels (the V-cycle of Algorithm 1, step 3).
//
// The small levels of a V-cycle are latency-bound: each launch costs a few microseconds whatever its
// work.  Two pairs of consecutive steps are merged into one launch each, on shared-memory node tiles
// with a one-node halo that is recomputed by the neighbouring tiles:
//   * residual + restriction: r = b - K z on the fine nodes under a tile of coarse nodes, then
//     b_c = P^T r (and, when the coarse level smooths, its first damped step z_c = omega D^-1 b_c);
//   * prolongation + first post-smoothing step: v = z + P z_c on the tile and its halo, then one
//     step v + d, d = coef D^-1 (b - K v).
// Both sum in the order of the separate kernels (k_restrict, k_prolong_add, k_apply_stencil), so
// the results are the same bit for bit.
// ================================================================================================

// (P zc)_c at fine node (i, j): bilinear interpolation from the up to four coarse nodes around it.
template <typename T>
__device__ __forceinline__ T prolong_value_2d(const Grid& gc, const T* __restrict__ zc, int i, int j, int c) {
  const int ix0 = i >> 1, ix1 = (i + 1) >> 1;
  const int iy0 = j >> 1, iy1 = (j + 1) >> 1;
  const T wx = (i & 1) ? T(0.5) : T(1), wy = (j & 1) ? T(0.5) : T(1);
  T acc = T(0);
#pragma unroll
  for (int by = 0; by < 2; ++by) {
    if (by == 1 && !(j & 1)) continue;
    const int J = by ? iy1 : iy0;
#pragma unroll
    for (int bx = 0; bx < 2; ++bx) {
      if (bx == 1 && !(i & 1)) continue;
      const int I = bx ? ix1 : ix0;
      const T w = wx * wy;
      acc += w * zc[2 * (I + (int64_t)gc.nn[0] * J) + c];
    }
  }
  return acc;
}

// The 36 stencil coefficients of one node, loaded together (before any barrier, so that their
// latency overlaps the tile loads).  Coefficients toward nodes outside the grid are exactly zero (no
// element couples them), and the tiles hold zeros there, so the sums need no bounds checks.
template <typename T>
__device__ __forceinline__ void load_stencil_2d(const T* __restrict__ S, int64_t nn, int64_t node, T (&st)[36]) {
#pragma unroll
  for (int q = 0; q < 36; ++q) st[q] = __ldg(S + (int64_t)q * nn + node);
}

// y = v + d, d = coef[0] d_in + coef[1] D^-1 (b - K v) with v = z + P zc (P zc skipped at fixed
// DOFs), for R right-hand sides per block (blockIdx.z groups); node tile TX x TY, one node per thread.
template <typename T, int TX, int TY, int R>
__global__ void __launch_bounds__(TX * TY) k_stencil_jac_prolong(Grid g, Grid gc, const T* __restrict__ S,
                                                                 const uint8_t* __restrict__ fixed,
                                                                 const T* __restrict__ z, const T* __restrict__ zc,
                                                                 const T* __restrict__ b, const T* __restrict__ dinv,
                                                                 T* __restrict__ y, SmoothArgs<T> sm, int nr,
                                                                 int64_t stride, int64_t cstride,
                                                                 const double* __restrict__ act) {
  pdl_wait();
  constexpr int NX = TX + 2, NY = TY + 2;
  __shared__ T vs[R][NY][NX][2];
  const int r0 = blockIdx.z * R;
  bool any = false;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (r0 + r < nr && !(act && act[(size_t)(r0 + r) * kScStride + SC_ACTIVE] == 0.0)) any = true;
  if (!any) return;
  const int nnx = g.nn[0], nny = g.nn[1];
  const int64_t nn = g.nnode;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int X = x0 + tx, Y = y0 + ty;
  const bool mine = X < nnx && Y < nny;
  const int64_t node = mine ? X + (int64_t)nnx * Y : 0;
  T st[36];
  load_stencil_2d<T>(S, nn, node, st);
  for (int q = threadIdx.x; q < NX * NY; q += TX * TY) {
    const int lx = q % NX, ly = q / NX;
    const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
    const bool inside = gx >= 0 && gx < nnx && gy >= 0 && gy < nny;
    const int64_t hn = gx + (int64_t)nnx * gy;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        T val = T(0);
        if (inside && r0 + r < nr) {
          val = z[(int64_t)(r0 + r) * stride + 2 * hn + c];
          if (!fixed[2 * hn + c]) val += prolong_value_2d<T>(gc, zc + (int64_t)(r0 + r) * cstride, gx, gy, c);
        }
        vs[r][ly][lx][c] = val;
      }
  }
  __syncthreads();
  if (!mine) return;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if (r0 + r >= nr) break;
    T acc[2] = {T(0), T(0)};
#pragma unroll
    for (int nbr = 0; nbr < 9; ++nbr) {
      const int dx = nbr % 3 - 1, dy = nbr / 3 - 1;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const T vv = vs[r][ty + 1 + dy][tx + 1 + dx][cc];
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[c] += st[(nbr * 2 + c) * 2 + cc] * vv;
      }
    }
    const int64_t off = (int64_t)(r0 + r) * stride;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int64_t idx = 2 * node + c;
      T out;
      if (fixed[idx]) {
        out = T(0);
      } else {
        const T rr = dinv[idx] * (b[off + idx] - acc[c]);
        const T dn = (sm.d_in ? sm.coef[0] * sm.d_in[off + idx] : T(0)) + sm.coef[1] * rr;
        if (sm.d_out) sm.d_out[off + idx] = dn;
        out = vs[r][ty + 1][tx + 1][c] + dn;
      }
      y[off + idx] = out;
    }
  }
}

// b_c = P^T (b - K z) on a CX x CY tile of coarse nodes (one right-hand side per blockIdx.z), and
// when zc != nullptr the coarse level's first damped step z_c = coef_c[1] dinv_c b_c (also into dc).
// One thread per fine node of the residual region ((2 CX + 1) x (2 CY + 1) nodes).
template <typename T, int CX, int CY>
__global__ void __launch_bounds__(((2 * CX + 1) * (2 * CY + 1) + 31) / 32 * 32)
    k_stencil_res_restrict(Grid g, Grid gc, const T* __restrict__ S, const uint8_t* __restrict__ fixed,
                           const T* __restrict__ z, const T* __restrict__ b, int64_t stride,
                           const uint8_t* __restrict__ fixed_c, T* __restrict__ bc, int64_t cstride,
                           const T* __restrict__ dinv_c, const T* __restrict__ coef_c, T* __restrict__ zc,
                           T* __restrict__ dc, const double* __restrict__ act) {
  pdl_wait();
  constexpr int RX = 2 * CX + 1, RY = 2 * CY + 1;  // fine nodes whose residual the tile restricts
  constexpr int ZX = RX + 2, ZY = RY + 2;          // ... and the iterate around them
  constexpr int NTH = (RX * RY + 31) / 32 * 32;
  __shared__ T zs[ZY][ZX][2];
  __shared__ T rs[RY][RX][2];
  const int rhs = blockIdx.z;
  if (act && act[(size_t)rhs * kScStride + SC_ACTIVE] == 0.0) return;
  const int nnx = g.nn[0], nny = g.nn[1];
  const int64_t nn = g.nnode;
  const int I0 = blockIdx.x * CX, J0 = blockIdx.y * CY;
  const int fx0 = 2 * I0 - 1, fy0 = 2 * J0 - 1;  // fine origin of the residual region
  z += (int64_t)rhs * stride;
  b += (int64_t)rhs * stride;
  // this thread's fine node of the residual region: stencil, right-hand side, mask
  const int t = threadIdx.x;
  const int lx = t % RX, ly = t / RX;
  const int gx = fx0 + lx, gy = fy0 + ly;
  const bool mine = t < RX * RY && gx >= 0 && gx < nnx && gy >= 0 && gy < nny;
  const int64_t node = mine ? gx + (int64_t)nnx * gy : 0;
  T st[36];
  load_stencil_2d<T>(S, nn, node, st);
  T b0 = T(0), b1 = T(0);
  bool f0 = true, f1 = true;
  if (mine) {
    b0 = b[2 * node];
    b1 = b[2 * node + 1];
    f0 = fixed[2 * node] != 0;
    f1 = fixed[2 * node + 1] != 0;
  }
  for (int q = t; q < ZX * ZY; q += NTH) {
    const int zx = q % ZX, zy = q / ZX;
    const int hx = fx0 - 1 + zx, hy = fy0 - 1 + zy;
    T a = T(0), c = T(0);
    if (hx >= 0 && hx < nnx && hy >= 0 && hy < nny) {
      const int64_t hn = hx + (int64_t)nnx * hy;
      a = z[2 * hn];
      c = z[2 * hn + 1];
    }
    zs[zy][zx][0] = a;
    zs[zy][zx][1] = c;
  }
  __syncthreads();
  if (t < RX * RY) {
    T acc[2] = {T(0), T(0)};
#pragma unroll
    for (int nbr = 0; nbr < 9; ++nbr) {
      const int dx = nbr % 3 - 1, dy = nbr / 3 - 1;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const T vv = zs[ly + 1 + dy][lx + 1 + dx][cc];
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[c] += st[(nbr * 2 + c) * 2 + cc] * vv;
      }
    }
    rs[ly][lx][0] = f0 ? T(0) : b0 - acc[0];
    rs[ly][lx][1] = f1 ? T(0) : b1 - acc[1];
  }
  __syncthreads();
  for (int q = t; q < CX * CY * 2; q += NTH) {
    const int c = q & 1, cl = q >> 1;
    const int ci = cl % CX, cj = cl / CX;
    const int I = I0 + ci, J = J0 + cj;
    if (I >= gc.nn[0] || J >= gc.nn[1]) continue;
    T acc = T(0);
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int fj = 2 * J + dy;
      if (fj < 0 || fj >= nny) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int fi = 2 * I + dx;
        if (fi < 0 || fi >= nnx) continue;
        const T w = T((dx == 0 ? 1.0 : 0.5) * (dy == 0 ? 1.0 : 0.5));
        acc += w * rs[2 * cj + 1 + dy][2 * ci + 1 + dx][c];
      }
    }
    const int64_t idx = 2 * (I + (int64_t)gc.nn[0] * J) + c;
    const T bi = fixed_c[idx] ? T(0) : acc;
    bc[(int64_t)rhs * cstride + idx] = bi;
    if (zc) {
      const T zi = coef_c[1] * dinv_c[idx] * bi;
      zc[(int64_t)rhs * cstride + idx] = zi;
      if (dc) dc[(int64_t)rhs * cstride + idx] = zi;
    }
  }
}

// CG direction on a stencil level: p = z + beta p_old (zero at fixed DOFs), q = K p, and the per-RHS
// reduction p.q -> sc[SC_PQ], alpha = (p.r) / (p.q) (the last block of each right-hand side);
// the same contract as the element-matrix k_cg_direction.  p at the neighbours is formed on the fly
// from z and p_old (one FMA each), straight-line as in k_apply_stencil.
template <int DIM>
__global__ void __launch_bounds__(256) k_stencil_cg_direction(Grid g, const double* __restrict__ S,
                                                              const uint8_t* __restrict__ fixed,
                                                              const double* __restrict__ z,
                                                              const double* __restrict__ p_old,
                                                              double* __restrict__ p_new, double* __restrict__ q,
                                                              int64_t stride, double* sc, double* partial,
                                                              unsigned* counters, int64_t pstride) {
  pdl_wait();
  constexpr int NB = StencilDims<DIM>::NB;
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  double* s = sc + (size_t)rhs * kScStride;
  if (s[SC_ACTIVE] == 0.0) return;
  const double beta = s[SC_BETA];
  const int64_t off = (int64_t)rhs * stride;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  double v[1] = {0.0};
  if (node_coords(g, node, i, j, k)) {
    const int64_t nn = g.nnode;
    double acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = 0.0;
#pragma unroll
    for (int nbr = 0; nbr < NB; ++nbr) {
      const int dx = nbr % 3 - 1, dy = (nbr / 3) % 3 - 1, dz = DIM == 3 ? nbr / 9 - 1 : 0;
      const bool in = i + dx >= 0 && i + dx < g.nn[0] && j + dy >= 0 && j + dy < g.nn[1] &&
                      (DIM == 2 || (k + dz >= 0 && k + dz < g.nn[2]));
      const int64_t nb = in ? node + dx + (int64_t)g.nn[0] * (dy + (int64_t)g.nn[1] * dz) : node;
#pragma unroll
      for (int cc = 0; cc < DIM; ++cc) {
        const int64_t id = off + DIM * nb + cc;
        const double pv = in ? __ldg(z + id) + beta * __ldg(p_old + id) : 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] += __ldg(S + (int64_t)((nbr * DIM + c) * DIM + cc) * nn + node) * pv;
      }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t idx = DIM * node + c;
      const bool fx = fixed[idx];
      const double pi = fx ? 0.0 : __ldg(z + off + idx) + beta * __ldg(p_old + off + idx);
      const double qi = fx ? 0.0 : acc[c];
      p_new[off + idx] = pi;
      q[off + idx] = qi;
      v[0] += pi * qi;
    }
  }
  double tot[1];
  if (grid_sum_last<1>(v, partial + rhs * pstride, counters + rhs, tot, smem) && threadIdx.x == 0) {
    const double pq = tot[0];
    s[SC_PQ] = pq;
    if (!(pq > 0.0) || !isfinite(pq)) {
      s[SC_STATUS] = 1.0;  // breakdown: K not positive on the search direction
      s[SC_ACTIVE] = 0.0;
      s[SC_ALPHA] = 0.0;
    } else {
      s[SC_ALPHA] = s[SC_PR] / pq;
    }
  }
}

void launch_stencil_cg_direction(const Grid& g, const double* S, const uint8_t* fixed, const double* z,
                                 const double* p_old, double* p_new, double* q, int nr, int64_t stride, double* sc,
                                 double* partial, unsigned* counters, int64_t pstride, cudaStream_t s) {
  const dim3 grid((unsigned)((g.nnode + 255) / 256), (unsigned)nr);
  if (g.dim == 2)
    launch_pdl(k_stencil_cg_direction<2>, dim3(grid), dim3(256), 0, s, g, S, fixed, z, p_old, p_new, q, stride, sc, partial, counters,
                                                   pstride);
  else
    launch_pdl(k_stencil_cg_direction<3>, dim3(grid), dim3(256), 0, s, g, S, fixed, z, p_old, p_new, q, stride, sc, partial, counters,
                                                   pstride);
}

static int sm_count_cached() {
  static int c = 0;
  if (c == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    if (c <= 0) c = 152;
  }
  return c;
}

template <typename T>
void launch_stencil_jac_prolong_2d(const Grid& g, const Grid& gc, const T* S, const uint8_t* fixed, const T* z,
                                   const T* zc, const T* b, const T* dinv, T* y, SmoothArgs<T> sm, int nr,
                                   int64_t stride, int64_t cstride, cudaStream_t s) {
  const double* act = active_rhs();
  const int nsm = sm_count_cached();
  const int64_t tiles32 = (int64_t)((g.nn[0] + 31) / 32) * ((g.nn[1] + 7) / 8);
  if (tiles32 * ((nr + 1) / 2) >= 2 * nsm) {
    const dim3 grid((g.nn[0] + 31) / 32, (g.nn[1] + 7) / 8, (nr + 1) / 2);
    launch_pdl(k_stencil_jac_prolong<T, 32, 8, 2>, dim3(grid), dim3(256), 0, s, g, gc, S, fixed, z, zc, b, dinv, y, sm, nr, stride,
                                                            cstride, act);
  } else if (tiles32 * nr >= nsm) {
    const dim3 grid((g.nn[0] + 31) / 32, (g.nn[1] + 7) / 8, nr);
    launch_pdl(k_stencil_jac_prolong<T, 32, 8, 1>, dim3(grid), dim3(256), 0, s, g, gc, S, fixed, z, zc, b, dinv, y, sm, nr, stride,
                                                            cstride, act);
  } else {
    const dim3 grid((g.nn[0] + 15) / 16, (g.nn[1] + 7) / 8, nr);
    launch_pdl(k_stencil_jac_prolong<T, 16, 8, 1>, dim3(grid), dim3(128), 0, s, g, gc, S, fixed, z, zc, b, dinv, y, sm, nr, stride,
                                                            cstride, act);
  }
}

template <typename T>
void launch_stencil_res_restrict_2d(const Grid& g, const Grid& gc, const T* S, const uint8_t* fixed, const T* z,
                                    const T* b, int64_t stride, const uint8_t* fixed_c, T* bc, int64_t cstride,
                                    const T* dinv_c, const T* coef_c, T* zc, T* dc, int nr, cudaStream_t s) {
  const double* act = active_rhs();
  const int nsm = sm_count_cached();
  const int64_t big = (int64_t)((gc.nn[0] + 7) / 8) * ((gc.nn[1] + 7) / 8);
  if (big * nr >= 2 * nsm) {  // 17 x 17 fine nodes per tile, two or more blocks resident per SM
    const dim3 grid((gc.nn[0] + 7) / 8, (gc.nn[1] + 7) / 8, nr);
    launch_pdl(k_stencil_res_restrict<T, 8, 8>, dim3(grid), dim3(320), 0, s, g, gc, S, fixed, z, b, stride, fixed_c, bc, cstride,
                                                         dinv_c, coef_c, zc, dc, act);
  } else {
    const dim3 grid((gc.nn[0] + 7) / 8, (gc.nn[1] + 3) / 4, nr);
    launch_pdl(k_stencil_res_restrict<T, 8, 4>, dim3(grid), dim3(160), 0, s, g, gc, S, fixed, z, b, stride, fixed_c, bc, cstride,
                                                         dinv_c, coef_c, zc, dc, act);
  }
}

template void launch_stencil_jac_prolong_2d<double>(const Grid&, const Grid&, const double*, const uint8_t*,
                                                    const double*, const double*, const double*, const double*,
                                                    double*, SmoothArgs<double>, int, int64_t, int64_t, cudaStream_t);
template void launch_stencil_jac_prolong_2d<float>(const Grid&, const Grid&, const float*, const uint8_t*,
                                                   const float*, const float*, const float*, const float*, float*,
                                                   SmoothArgs<float>, int, int64_t, int64_t, cudaStream_t);
template void launch_stencil_res_restrict_2d<double>(const Grid&, const Grid&, const double*, const uint8_t*,
                                                     const double*, const double*, int64_t, const uint8_t*, double*,
                                                     int64_t, const double*, const double*, double*, double*, int,
                                                     cudaStream_t);
template void launch_stencil_res_restrict_2d<float>(const Grid&, const Grid&, const float*, const uint8_t*,
                                                    const float*, const float*, int64_t, const uint8_t*, float*,
                                                    int64_t, const float*, const float*, float*, float*, int,
                                                    cudaStream_t);

}  // namespace tobk
