// CUDA kernels of the multilevel buckling solver (sm_103a).
//
// Paper mapping (Ferrari & Sigmund, arXiv 1909.13585):
//   SIMP moduli E_kappa, E_sigma ........................ Sec. 2, eq. interpolationSIMP2-SIMP
//   K(x) v matrix-free (K_e = E_kappa K_e0) ............. Sec. 2; LA of Algorithm 1 / Algorithm 2
//   G(x,u) from Gauss-point stresses (G_e = E_sigma G_e0) Sec. 2
//   restriction / interpolation, Galerkin K^l, G^l ...... Sec. 2.1 step 1-2, Algorithm 2 'restrict'
//   damped Jacobi smoother, coarsest dense solve ........ the multigrid preconditioner of the
//                                                         mgPCG solves (Appendix A)
//   PCG / flexible CG recurrences ........................ Appendix A (mgPCG / mgBPCG)
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "device_common.cuh"
#include "kernels.h"

namespace tobk {

namespace {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t count, int threads = kThreads) {
  return (unsigned)((count + threads - 1) / threads);
}

template <int DIM, typename T>
FineOp<DIM, T> make_fine(const LevelOpDesc& d, const T* scale) {
  FineOp<DIM, T> op;
  op.g = d.g;
  op.scale_e = scale;
  op.fixed = d.fixed;
  constexpr int ND = Dims<DIM>::ND;
  for (int i = 0; i < ND * ND; ++i) op.M[i] = (T)d.T0[i];
  return op;
}

template <int DIM, typename T>
StoredOp<DIM, T> make_stored(const LevelOpDesc& d, const T* Ke) {
  StoredOp<DIM, T> op;
  op.g = d.g;
  op.Ke = Ke;
  op.fixed = d.fixed;
  return op;
}

}  // namespace

// ================================================================================================
// level operators
// ================================================================================================
template <int DIM, class Op, typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_apply(const __grid_constant__ Op op, const T* __restrict__ v, const T* __restrict__ b,
                                                     const T* __restrict__ dinv, T* __restrict__ y, SmoothArgs<T> sm,
                                                     int64_t stride, const double* __restrict__ act) {
  pdl_wait();
  if (rhs_done(act)) return;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(op.g, node, i, j, k)) return;
  const int64_t off = (int64_t)blockIdx.y * stride;
  v += off;
  y += off;
  if (MODE != APPLY_KV) b += off;
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
  gather_rows<DIM, T>(op, i, j, k, LoadVec<T>{v}, acc);
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t idx = DIM * node + c;
    T out;
    if (op.fixed[idx]) {
      out = T(0);
    } else if (MODE == APPLY_KV) {
      out = acc[c];
    } else if (MODE == APPLY_RES) {
      out = b[idx] - acc[c];
    } else {
      const T r = dinv[idx] * (b[idx] - acc[c]);
      const T dn = (sm.d_in ? sm.coef[0] * sm.d_in[off + idx] : T(0)) + sm.coef[1] * r;
      if (sm.d_out) sm.d_out[off + idx] = dn;
      out = v[idx] + dn;
    }
    y[idx] = out;
  }
}

template <int DIM, class Op, typename T>
void apply_dispatch(const Op& op, int mode, const T* v, const T* b, const T* dinv, T* y, SmoothArgs<T> sm, int nr,
                    int64_t stride, cudaStream_t s) {
  dim3 grid(blocks_for(op.g.nnode), nr);
  if (mode == APPLY_KV)
    launch_pdl(k_apply<DIM, Op, T, APPLY_KV>, dim3(grid), dim3(kThreads), 0, s, op, v, b, dinv, y, sm, stride, active_rhs());
  else if (mode == APPLY_RES)
    launch_pdl(k_apply<DIM, Op, T, APPLY_RES>, dim3(grid), dim3(kThreads), 0, s, op, v, b, dinv, y, sm, stride, active_rhs());
  else
    launch_pdl(k_apply<DIM, Op, T, APPLY_JAC>, dim3(grid), dim3(kThreads), 0, s, op, v, b, dinv, y, sm, stride, active_rhs());
}

template <int DIM>
void apply_dim(const LevelOpDesc& d, int mode, const double* v, const double* b, const double* dinv, double* y,
               SmoothArgs<double> sm, int nr, int64_t stride, cudaStream_t s) {
  if (d.stored)
    apply_dispatch<DIM>(make_stored<DIM, double>(d, d.Ke64), mode, v, b, dinv, y, sm, nr, stride, s);
  else
    apply_dispatch<DIM>(make_fine<DIM, double>(d, d.scale64), mode, v, b, dinv, y, sm, nr, stride, s);
}

template <int DIM>
void apply_dim32(const LevelOpDesc& d, int mode, const float* v, const float* b, const float* dinv, float* y,
                 SmoothArgs<float> sm, int nr, int64_t stride, cudaStream_t s) {
  if (d.stored)
    apply_dispatch<DIM>(make_stored<DIM, float>(d, d.Ke32), mode, v, b, dinv, y, sm, nr, stride, s);
  else
    apply_dispatch<DIM>(make_fine<DIM, float>(d, d.scale32), mode, v, b, dinv, y, sm, nr, stride, s);
}

template <typename T>
void launch_apply_stencil(const Grid& g, const T* S, const uint8_t* fixed, int mode, const T* v, const T* b,
                          const T* dinv, T* y, SmoothArgs<T> sm, int nr, int64_t stride, cudaStream_t s);

template <typename T>
void launch_fine_q4(const Grid& g, const T* Ek, const uint8_t* fixed, const double* Ke0, int mode, const T* v,
                    const T* b, const T* dinv, T* y, SmoothArgs<T> sm, int nr, int64_t stride, cudaStream_t s);

void launch_apply(const LevelOpDesc& op, int mode, const double* v, const double* b, const double* dinv,
                  double* y, SmoothArgs<double> sm, int nr, int64_t stride, cudaStream_t s) {
  if (op.S64) {
    launch_apply_stencil<double>(op.g, op.S64, op.fixed, mode, v, b, dinv, y, sm, nr, stride, s);
    return;
  }
  if (!op.stored && op.g.dim == 2) {
    launch_fine_q4<double>(op.g, op.scale64, op.fixed, op.T0, mode, v, b, dinv, y, sm, nr, stride, s);
    return;
  }
  if (!op.stored && op.g.dim == 3) {
    launch_fine_h8<double>(op.g, op.scale64, op.fixed, op.nu, op.element, mode, v, b, dinv, y, sm, nr, stride, s);
    return;
  }
  if (op.g.dim == 2)
    apply_dim<2>(op, mode, v, b, dinv, y, sm, nr, stride, s);
  else
    apply_dim<3>(op, mode, v, b, dinv, y, sm, nr, stride, s);
}

void launch_apply32(const LevelOpDesc& op, int mode, const float* v, const float* b, const float* dinv,
                    float* y, SmoothArgs<float> sm, int nr, int64_t stride, cudaStream_t s) {
  if (op.S32) {
    launch_apply_stencil<float>(op.g, op.S32, op.fixed, mode, v, b, dinv, y, sm, nr, stride, s);
    return;
  }
  if (!op.stored && op.g.dim == 2) {
    launch_fine_q4<float>(op.g, op.scale32, op.fixed, op.T0, mode, v, b, dinv, y, sm, nr, stride, s);
    return;
  }
  if (!op.stored && op.g.dim == 3) {
    launch_fine_h8<float>(op.g, op.scale32, op.fixed, op.nu, op.element, mode, v, b, dinv, y, sm, nr, stride, s);
    return;
  }
  if (op.g.dim == 2)
    apply_dim32<2>(op, mode, v, b, dinv, y, sm, nr, stride, s);
  else
    apply_dim32<3>(op, mode, v, b, dinv, y, sm, nr, stride, s);
}

// ---- stress stiffness operator (fine level) -----------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_apply_kron(ScalarKronOp<DIM, double> op, const double* __restrict__ v,
                                                         double* __restrict__ y, int64_t stride) {
  pdl_wait();
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(op.g, node, i, j, k)) return;
  const int64_t off = (int64_t)blockIdx.y * stride;
  double acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = 0.0;
  gather_rows_kron<DIM, double>(op, i, j, k, LoadVec<double>{v + off}, acc);
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t idx = DIM * node + c;
    y[off + idx] = op.fixed[idx] ? 0.0 : acc[c];
  }
}

void launch_apply_kron(const Grid& g, const uint8_t* fixed, const double* Gs, const double* v, double* y, int nr,
                       int64_t stride, cudaStream_t s) {
  dim3 grid(blocks_for(g.nnode), nr);
  if (g.dim == 2) {
    ScalarKronOp<2, double> op{g, Gs, fixed};
    launch_pdl(k_apply_kron<2>, dim3(grid), dim3(kThreads), 0, s, op, v, y, stride);
  } else {
    ScalarKronOp<3, double> op{g, Gs, fixed};
    launch_pdl(k_apply_kron<3>, dim3(grid), dim3(kThreads), 0, s, op, v, y, stride);
  }
}

// ---- diagonal -----------------------------------------------------------------------------------
template <int DIM, class Op>
__global__ void k_diag(const __grid_constant__ Op op, double* dinv, float* dinv32) {
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(op.g, node, i, j, k)) return;
  const Grid& g = op.g;
  double d[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) d[c] = 0.0;
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
#pragma unroll
        for (int c = 0; c < DIM; ++c)
          d[c] += (double)op.scale(e) * (double)op.entry(e, ln * DIM + c, ln * DIM + c);
      }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t idx = DIM * node + c;
    const double v = (op.fixed[idx] || !(d[c] > 0.0)) ? 0.0 : 1.0 / d[c];
    dinv[idx] = v;
    if (dinv32) dinv32[idx] = (float)v;
  }
}

void launch_diag(const LevelOpDesc& d, double* dinv, float* dinv32, cudaStream_t s) {
  const unsigned grid = blocks_for(d.g.nnode);
  if (d.g.dim == 2) {
    if (d.stored)
      ::tobk::note_launch(), k_diag<2><<<grid, kThreads, 0, s>>>(make_stored<2, double>(d, d.Ke64), dinv, dinv32);
    else
      ::tobk::note_launch(), k_diag<2><<<grid, kThreads, 0, s>>>(make_fine<2, double>(d, d.scale64), dinv, dinv32);
  } else {
    if (d.stored)
      ::tobk::note_launch(), k_diag<3><<<grid, kThreads, 0, s>>>(make_stored<3, double>(d, d.Ke64), dinv, dinv32);
    else
      ::tobk::note_launch(), k_diag<3><<<grid, kThreads, 0, s>>>(make_fine<3, double>(d, d.scale64), dinv, dinv32);
  }
}

// ---- first Jacobi sweep from zero --------------------------------------------------------------
template <typename T>
__global__ void k_jacobi0(const T* __restrict__ b, const T* __restrict__ dinv, T* __restrict__ z, SmoothArgs<T> sm,
                          int64_t n, int64_t stride, const double* __restrict__ act) {
  pdl_wait();
  if (rhs_done(act)) return;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t off = (int64_t)blockIdx.y * stride;
  const T zi = sm.coef[1] * dinv[i] * b[off + i];
  z[off + i] = zi;
  if (sm.d_out) sm.d_out[off + i] = zi;
}

void launch_jacobi0(const double* b, const double* dinv, double* z, SmoothArgs<double> sm, int64_t n, int nr,
                    int64_t stride, cudaStream_t s) {
  launch_pdl(k_jacobi0<double>, dim3(dim3(blocks_for(n), nr)), dim3(kThreads), 0, s, b, dinv, z, sm, n, stride, active_rhs());
}
void launch_jacobi0_32(const float* b, const float* dinv, float* z, SmoothArgs<float> sm, int64_t n, int nr, int64_t stride,
                       cudaStream_t s) {
  launch_pdl(k_jacobi0<float>, dim3(dim3(blocks_for(n), nr)), dim3(kThreads), 0, s, b, dinv, z, sm, n, stride, active_rhs());
}

// ---- transfers ----------------------------------------------------------------------------------
// Interpolation weights of nested 2:1 grids: fine node f and coarse node C along one axis are
// coupled with weight 1 when f = 2C and 1/2 when |f - 2C| = 1.
template <int DIM, typename T>
__global__ void k_restrict(Grid gf, Grid gc, const uint8_t* __restrict__ fixed_c, const T* __restrict__ rf,
                           T* __restrict__ bc, int64_t sf, int64_t sc, const double* __restrict__ act,
                           const T* __restrict__ dinv_c, const T* __restrict__ coef_c, T* __restrict__ zc,
                           T* __restrict__ dc) {
  pdl_wait();
  if (rhs_done(act)) return;
  const int64_t cn = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int I, J, K;
  if (!node_coords(gc, cn, I, J, K)) return;
  rf += (int64_t)blockIdx.y * sf;
  bc += (int64_t)blockIdx.y * sc;
  if (zc) zc += (int64_t)blockIdx.y * sc;
  if (dc) dc += (int64_t)blockIdx.y * sc;
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
    const int fk = 2 * K + dz;
    if (DIM == 3 && (fk < 0 || fk >= gf.nn[2])) continue;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int fj = 2 * J + dy;
      if (fj < 0 || fj >= gf.nn[1]) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int fi = 2 * I + dx;
        if (fi < 0 || fi >= gf.nn[0]) continue;
        const T w = T((dx == 0 ? 1.0 : 0.5) * (dy == 0 ? 1.0 : 0.5) * (dz == 0 ? 1.0 : 0.5));
        const int64_t fn = fi + (int64_t)gf.nn[0] * (fj + (int64_t)gf.nn[1] * (DIM == 3 ? fk : 0));
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] += w * rf[DIM * fn + c];
      }
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t idx = DIM * cn + c;
    const T bi = fixed_c[idx] ? T(0) : acc[c];
    bc[idx] = bi;
    if (zc) {  // the coarse level's first smoothing step from z = 0 (k_jacobi0), fused
      const T zi = coef_c[1] * dinv_c[idx] * bi;
      zc[idx] = zi;
      if (dc) dc[idx] = zi;
    }
  }
}

template <int DIM, typename T>
__global__ void k_prolong_add(Grid gf, Grid gc, const uint8_t* __restrict__ fixed_f, const T* __restrict__ zc,
                              T* __restrict__ zf, int64_t sf, int64_t sc, const double* __restrict__ act) {
  pdl_wait();
  if (rhs_done(act)) return;
  const int64_t fn = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(gf, fn, i, j, k)) return;
  zc += (int64_t)blockIdx.y * sc;
  zf += (int64_t)blockIdx.y * sf;
  const int ix0 = i >> 1, ix1 = (i + 1) >> 1;
  const int iy0 = j >> 1, iy1 = (j + 1) >> 1;
  const int iz0 = k >> 1, iz1 = (k + 1) >> 1;
  const T wx = (i & 1) ? T(0.5) : T(1), wy = (j & 1) ? T(0.5) : T(1), wz = (k & 1) ? T(0.5) : T(1);
  T acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = T(0);
#pragma unroll
  for (int bz = 0; bz < (DIM == 3 ? 2 : 1); ++bz) {
    if (bz == 1 && !(k & 1)) continue;
    const int K = bz ? iz1 : iz0;
#pragma unroll
    for (int by = 0; by < 2; ++by) {
      if (by == 1 && !(j & 1)) continue;
      const int J = by ? iy1 : iy0;
#pragma unroll
      for (int bx = 0; bx < 2; ++bx) {
        if (bx == 1 && !(i & 1)) continue;
        const int I = bx ? ix1 : ix0;
        const T w = wx * wy * (DIM == 3 ? wz : T(1));
        const int64_t cn = I + (int64_t)gc.nn[0] * (J + (int64_t)gc.nn[1] * (DIM == 3 ? K : 0));
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] += w * zc[DIM * cn + c];
      }
    }
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t idx = DIM * fn + c;
    if (!fixed_f[idx]) zf[idx] += acc[c];
  }
}

template <typename T>
static void restrict_impl(const Grid& gf, const Grid& gc, const uint8_t* fixed_c, const T* rf, T* bc, int nr,
                          int64_t sf, int64_t sc, cudaStream_t s, const T* dinv_c, const T* coef_c, T* zc, T* dc) {
  dim3 grid(blocks_for(gc.nnode), nr);
  if (gf.dim == 2)
    launch_pdl(k_restrict<2, T>, dim3(grid), dim3(kThreads), 0, s, gf, gc, fixed_c, rf, bc, sf, sc, active_rhs(),
                                                                      dinv_c, coef_c, zc, dc);
  else
    launch_pdl(k_restrict<3, T>, dim3(grid), dim3(kThreads), 0, s, gf, gc, fixed_c, rf, bc, sf, sc, active_rhs(),
                                                                      dinv_c, coef_c, zc, dc);
}
template <typename T>
static void prolong_impl(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const T* zc, T* zf, int nr,
                         int64_t sf, int64_t sc, cudaStream_t s) {
  dim3 grid(blocks_for(gf.nnode), nr);
  if (gf.dim == 2)
    launch_pdl(k_prolong_add<2, T>, dim3(grid), dim3(kThreads), 0, s, gf, gc, fixed_f, zc, zf, sf, sc, active_rhs());
  else
    launch_pdl(k_prolong_add<3, T>, dim3(grid), dim3(kThreads), 0, s, gf, gc, fixed_f, zc, zf, sf, sc, active_rhs());
}

void launch_restrict(const Grid& gf, const Grid& gc, const uint8_t* fixed_c, const double* rf, double* bc, int nr,
                     int64_t sf, int64_t sc, cudaStream_t s, const double* dinv_c, const double* coef_c, double* zc,
                     double* dc) {
  restrict_impl<double>(gf, gc, fixed_c, rf, bc, nr, sf, sc, s, dinv_c, coef_c, zc, dc);
}
void launch_restrict32(const Grid& gf, const Grid& gc, const uint8_t* fixed_c, const float* rf, float* bc, int nr,
                       int64_t sf, int64_t sc, cudaStream_t s, const float* dinv_c, const float* coef_c, float* zc,
                       float* dc) {
  restrict_impl<float>(gf, gc, fixed_c, rf, bc, nr, sf, sc, s, dinv_c, coef_c, zc, dc);
}
void launch_prolong_add(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* zc, double* zf,
                        int nr, int64_t sf, int64_t sc, cudaStream_t s) {
  prolong_impl<double>(gf, gc, fixed_f, zc, zf, nr, sf, sc, s);
}
void launch_prolong_add32(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const float* zc, float* zf,
                          int nr, int64_t sf, int64_t sc, cudaStream_t s) {
  prolong_impl<float>(gf, gc, fixed_f, zc, zf, nr, sf, sc, s);
}

// ---- coarsest level: dense inverse --------------------------------------------------------------
template <typename T>
__global__ void k_dense_gemv(const double* __restrict__ A, const T* __restrict__ b, T* __restrict__ z, int64_t n,
                             int64_t stride, const double* __restrict__ act) {
  pdl_wait();
  if (rhs_done(act)) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  b += (int64_t)blockIdx.y * stride;
  z += (int64_t)blockIdx.y * stride;
  const double* a = A + row * n;
  double s = 0.0;
  for (int64_t j = lane; j < n; j += 32) s += a[j] * (double)b[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) z[row] = (T)s;
}

void launch_dense_gemv(const double* Ainv, const double* b, double* z, int64_t n, int nr, int64_t stride,
                       cudaStream_t s) {
  launch_pdl(k_dense_gemv<double>, dim3(dim3(blocks_for(n * 32), nr)), dim3(kThreads), 0, s, Ainv, b, z, n, stride, active_rhs());
}
void launch_dense_gemv32(const double* Ainv, const float* b, float* z, int64_t n, int nr, int64_t stride,
                         cudaStream_t s) {
  launch_pdl(k_dense_gemv<float>, dim3(dim3(blocks_for(n * 32), nr)), dim3(kThreads), 0, s, Ainv, b, z, n, stride, active_rhs());
}

template <int DIM, class Op>
__global__ void k_dense_assemble(Op op, double* A) {
  constexpr int NN = Dims<DIM>::NN;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(op.g, node, i, j, k)) return;
  const Grid& g = op.g;
  const int64_t n = g.n;
  for (int c = 0; c < DIM; ++c) {
    const int64_t row = DIM * node + c;
    double* Ar = A + row * n;
    if (op.fixed[row]) {
      Ar[row] = 1.0;
      continue;
    }
    for (int cz = 0; cz < (DIM == 3 ? 2 : 1); ++cz)
      for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) {
          const int ei = i - cx, ej = j - cy, ek = k - cz;
          if (ei < 0 || ei >= g.nel[0] || ej < 0 || ej >= g.nel[1]) continue;
          if (DIM == 3 && (ek < 0 || ek >= g.nel[2])) continue;
          const int64_t e = ei + (int64_t)g.nel[0] * (ej + (int64_t)g.nel[1] * ek);
          const int64_t n0 = ei + (int64_t)g.nn[0] * (ej + (int64_t)g.nn[1] * ek);
          const int ln = local_node(cx, cy, cz);
          const double sc = (double)op.scale(e);
          for (int lb = 0; lb < NN; ++lb) {
            const int64_t nb = n0 + corner_x(lb) + (int64_t)g.nn[0] * (corner_y(lb) + (int64_t)g.nn[1] * corner_z(lb));
            for (int cc = 0; cc < DIM; ++cc) {
              const int64_t col = DIM * nb + cc;
              if (op.fixed[col]) continue;
              Ar[col] += sc * (double)op.entry(e, ln * DIM + c, lb * DIM + cc);
            }
          }
        }
  }
}

// The fine-level FineOp carries its table in kernel parameters with runtime indices here, so the
// dense assembly of a fine level uses a global-memory copy of the table instead.
template <int DIM>
struct FineOpGlobal {
  Grid g;
  const double* scale_e;
  const uint8_t* fixed;
  const double* M;
  __device__ double scale(int64_t e) const { return scale_e[e]; }
  __device__ double entry(int64_t, int r, int c) const { return M[r * Dims<DIM>::ND + c]; }
};

void launch_dense_assemble(const LevelOpDesc& d, double* A, cudaStream_t s) {
  cudaMemsetAsync(A, 0, sizeof(double) * d.g.n * d.g.n, s);
  const unsigned grid = blocks_for(d.g.nnode, 128);
  if (d.stored) {
    if (d.g.dim == 2)
      ::tobk::note_launch(), k_dense_assemble<2><<<grid, 128, 0, s>>>(make_stored<2, double>(d, d.Ke64), A);
    else
      ::tobk::note_launch(), k_dense_assemble<3><<<grid, 128, 0, s>>>(make_stored<3, double>(d, d.Ke64), A);
  } else {
    if (d.g.dim == 2)
      ::tobk::note_launch(), k_dense_assemble<2><<<grid, 128, 0, s>>>(FineOpGlobal<2>{d.g, d.scale64, d.fixed, d.T0dev}, A);
    else
      ::tobk::note_launch(), k_dense_assemble<3><<<grid, 128, 0, s>>>(FineOpGlobal<3>{d.g, d.scale64, d.fixed, d.T0dev}, A);
  }
}

// One Gauss-Jordan elimination step on an SPD matrix (no pivoting): after steps k = 0..n-1 the
// buffer holds the inverse.
// rcp[k & 1] holds 1 / A[k][k] on entry; the thread that produces the next pivot B[k+1][k+1] stores
// its reciprocal in rcp[(k + 1) & 1], so each step performs a single FP64 division.
__global__ void k_gj_step(const double* __restrict__ A, double* __restrict__ B, int64_t n, int64_t k,
                          double* __restrict__ rcp) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx / n, j = idx % n;
  const double rp = rcp[k & 1];
  double v;
  if (i == k && j == k)
    v = rp;
  else if (i == k)
    v = A[k * n + j] * rp;
  else if (j == k)
    v = -A[i * n + k] * rp;
  else
    v = A[i * n + j] - A[i * n + k] * (A[k * n + j] * rp);
  B[idx] = v;
  if (i == k + 1 && j == k + 1) rcp[(k + 1) & 1] = 1.0 / v;
}

__global__ void k_first_pivot(const double* A, double* rcp) { rcp[0] = 1.0 / A[0]; }

// Blocked in-place Gauss-Jordan (the same elimination as k_gj_step, kGJB pivots at a time): for the
// pivot block K = [k0, k0 + bs),
//   P = A_KK^{-1};  R_K = P A_K,j (j outside K);  A_ij -= A_iK R_Kj (i, j outside K);
//   A_iK <- -A_iK P (i outside K);  A_KK <- P;  A_Kj <- R_Kj.
// After the last block A holds its inverse.  Five launches per block instead of one per pivot.
constexpr int kGJB = 32;

__global__ void __launch_bounds__(kGJB * kGJB) k_bgj_diag(const double* __restrict__ A, int64_t n, int64_t k0, int bs,
                                                          double* __restrict__ P) {
  __shared__ double M[kGJB][kGJB + 1];
  __shared__ double rp_s;
  const int i = threadIdx.y, j = threadIdx.x;
  if (i < bs && j < bs) M[i][j] = A[(k0 + i) * n + k0 + j];
  __syncthreads();
  for (int p = 0; p < bs; ++p) {
    // one reciprocal per pivot (FP64 division is a long instruction sequence at 2 FP64 operations
    // per clock per SM: 1024 threads dividing each would dominate the block)
    if (i == 0 && j == 0) rp_s = 1.0 / M[p][p];
    __syncthreads();
    double v = 0.0;
    if (i < bs && j < bs) {
      const double r = rp_s;
      if (i == p && j == p)
        v = r;
      else if (i == p)
        v = M[p][j] * r;
      else if (j == p)
        v = -M[i][p] * r;
      else
        v = M[i][j] - M[i][p] * (M[p][j] * r);
    }
    __syncthreads();
    if (i < bs && j < bs) M[i][j] = v;
    __syncthreads();
  }
  if (i < bs && j < bs) P[i * kGJB + j] = M[i][j];
}

// R[r][j] = sum_q P[r][q] A[k0 + q][j] for columns j outside the block (R [bs][n])
__global__ void k_bgj_row(const double* __restrict__ A, int64_t n, int64_t k0, int bs, const double* __restrict__ P,
                          double* __restrict__ R) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (j >= n || (j >= k0 && j < k0 + bs)) return;
  double s = 0.0;
  for (int q = 0; q < bs; ++q) s += P[r * kGJB + q] * A[(k0 + q) * n + j];
  R[(int64_t)r * n + j] = s;
}

// A_ij -= sum_q A[i][k0 + q] R[q][j] for i, j outside the block; 32 x 32 tiles, 4 rows per thread
__global__ void __launch_bounds__(256) k_bgj_update(double* __restrict__ A, int64_t n, int64_t k0, int bs,
                                                    const double* __restrict__ R) {
  __shared__ double Ai[32][kGJB + 1];
  __shared__ double Rk[kGJB][33];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int64_t i0 = (int64_t)blockIdx.y * 32, j0 = (int64_t)blockIdx.x * 32;
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t i = i0 + rr;
    Ai[rr][tx] = (i < n && tx < bs) ? A[i * n + k0 + tx] : 0.0;
  }
  for (int q = ty; q < kGJB; q += 8) {
    const int64_t j = j0 + tx;
    Rk[q][tx] = (q < bs && j < n) ? R[(int64_t)q * n + j] : 0.0;
  }
  __syncthreads();
  const int64_t j = j0 + tx;
  if (j >= n || (j >= k0 && j < k0 + bs)) return;
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t i = i0 + rr;
    if (i >= n || (i >= k0 && i < k0 + bs)) continue;
    double acc = 0.0;
#pragma unroll 8
    for (int q = 0; q < kGJB; ++q) acc += Ai[rr][q] * Rk[q][tx];
    A[i * n + j] -= acc;
  }
}

// A_iK <- -A_iK P for i outside the block (one warp per row), then A_KK <- P and A_Kj <- R_Kj
__global__ void k_bgj_col(double* __restrict__ A, int64_t n, int64_t k0, int bs, const double* __restrict__ P) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int c = threadIdx.x & 31;
  if (i >= n || (i >= k0 && i < k0 + bs)) return;
  const double old = c < bs ? A[i * n + k0 + c] : 0.0;
  double s = 0.0;
  for (int q = 0; q < bs; ++q) s += __shfl_sync(0xffffffffu, old, q) * (c < bs ? P[q * kGJB + c] : 0.0);
  if (c < bs) A[i * n + k0 + c] = -s;
}
__global__ void k_bgj_rows_back(double* __restrict__ A, int64_t n, int64_t k0, int bs, const double* __restrict__ P,
                                const double* __restrict__ R) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (j >= n) return;
  A[(k0 + r) * n + j] = (j >= k0 && j < k0 + bs) ? P[r * kGJB + (j - k0)] : R[(int64_t)r * n + j];
}

double* launch_dense_invert(double* A, double* work, int64_t n, double* rcp2, cudaStream_t s) {
  if (n <= 2 * kGJB) {  // small matrices: one launch per pivot
    double* src = A;
    double* dst = work;
    ::tobk::note_launch(), k_first_pivot<<<1, 1, 0, s>>>(A, rcp2);
    for (int64_t k = 0; k < n; ++k) {
      ::tobk::note_launch(), k_gj_step<<<blocks_for(n * n), kThreads, 0, s>>>(src, dst, n, k, rcp2);
      std::swap(src, dst);
    }
    return src;
  }
  // work (n x n, n > 2 kGJB) holds R [kGJB][n] and P [kGJB][kGJB]
  double* R = work;
  double* P = work + (size_t)kGJB * n;
  const unsigned tiles = (unsigned)((n + 31) / 32);
  for (int64_t k0 = 0; k0 < n; k0 += kGJB) {
    const int bs = (int)std::min<int64_t>(kGJB, n - k0);
    ::tobk::note_launch(), k_bgj_diag<<<1, dim3(kGJB, kGJB), 0, s>>>(A, n, k0, bs, P);
    ::tobk::note_launch(), k_bgj_row<<<dim3(blocks_for(n, 128), bs), 128, 0, s>>>(A, n, k0, bs, P, R);
    ::tobk::note_launch(), k_bgj_update<<<dim3(tiles, tiles), dim3(32, 8), 0, s>>>(A, n, k0, bs, R);
    ::tobk::note_launch(), k_bgj_col<<<blocks_for(n * 32, 256), 256, 0, s>>>(A, n, k0, bs, P);
    ::tobk::note_launch(), k_bgj_rows_back<<<dim3(blocks_for(n, 128), bs), 128, 0, s>>>(A, n, k0, bs, P, R);
  }
  return A;
}

// ================================================================================================
// Galerkin coarse element matrices: K_c = sum_children W_k^T (masked child K) W_k
// ================================================================================================
enum { GAL_FINE_K = 0, GAL_FINE_G = 1, GAL_STORED = 2, GAL_SCALED_STORED = 3 };

template <int DIM, int SRC>
__global__ void k_galerkin(Grid gf, Grid gc, const uint8_t* __restrict__ fixed_f, const double* __restrict__ src,
                           const double* __restrict__ T0, const double* __restrict__ W, double* __restrict__ Kc) {
  constexpr int NN = Dims<DIM>::NN;
  constexpr int ND = Dims<DIM>::ND;
  __shared__ double sK[ND * ND];
  __shared__ double sT[ND * ND];
  __shared__ double sW[NN * NN * NN];
  const int t = threadIdx.x;  // blockDim.x == ND*ND
  for (int q = t; q < NN * NN * NN; q += blockDim.x) sW[q] = W[q];
  const int64_t E = blockIdx.x;
  const int EI = (int)(E % gc.nel[0]);
  const int64_t rest = E / gc.nel[0];
  const int EJ = (int)(rest % gc.nel[1]);
  const int EK = (int)(rest / gc.nel[1]);
  const int row = t / ND, col = t % ND;
  const int lr = row / DIM, cr = row % DIM, lc = col / DIM, cc = col % DIM;
  double acc = 0.0;
  __syncthreads();
  for (int kc = 0; kc < NN; ++kc) {
    const int fi = 2 * EI + corner_x(kc), fj = 2 * EJ + corner_y(kc), fk = 2 * EK + corner_z(kc);
    const int64_t ef = fi + (int64_t)gf.nel[0] * (fj + (int64_t)gf.nel[1] * fk);
    const int64_t n0 = fi + (int64_t)gf.nn[0] * (fj + (int64_t)gf.nn[1] * fk);
    const int64_t nr_ = n0 + corner_x(lr) + (int64_t)gf.nn[0] * (corner_y(lr) + (int64_t)gf.nn[1] * corner_z(lr));
    const int64_t nc_ = n0 + corner_x(lc) + (int64_t)gf.nn[0] * (corner_y(lc) + (int64_t)gf.nn[1] * corner_z(lc));
    double val;
    if (SRC == GAL_FINE_K)
      val = src[ef] * T0[row * ND + col];
    else if (SRC == GAL_FINE_G)
      val = (cr == cc) ? src[ef * NN * NN + lr * NN + lc] : 0.0;
    else if (SRC == GAL_SCALED_STORED)
      val = T0[ef] * src[ef * ND * ND + row * ND + col];
    else
      val = src[ef * ND * ND + row * ND + col];
    if (fixed_f[DIM * nr_ + cr] || fixed_f[DIM * nc_ + cc]) val = 0.0;
    sK[t] = val;
    __syncthreads();
    {  // T[r][b*DIM+c'] = sum_l K[r][l*DIM+c'] W[kc][l][b]
      const int b = col / DIM, cp = col % DIM;
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < NN; ++l) s += sK[row * ND + l * DIM + cp] * sW[(kc * NN + l) * NN + b];
      sT[t] = s;
    }
    __syncthreads();
    {  // out[a*DIM+c][col] += sum_i W[kc][i][a] T[i*DIM+c][col]
      const int a = row / DIM, c = row % DIM;
#pragma unroll
      for (int i = 0; i < NN; ++i) acc += sW[(kc * NN + i) * NN + a] * sT[(i * DIM + c) * ND + col];
    }
    __syncthreads();
  }
  Kc[E * ND * ND + t] = acc;
}

template <int SRC>
static void galerkin_impl(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* src,
                          const double* T0, const double* W, double* Kc, cudaStream_t s) {
  if (gf.dim == 2)
    ::tobk::note_launch(), k_galerkin<2, SRC><<<(unsigned)gc.m, 64, 0, s>>>(gf, gc, fixed_f, src, T0, W, Kc);
  else
    ::tobk::note_launch(), k_galerkin<3, SRC><<<(unsigned)gc.m, 576, 0, s>>>(gf, gc, fixed_f, src, T0, W, Kc);
}

void launch_galerkin_fine_K(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* scale,
                            const double* Ke0, const double* W, double* Kc, cudaStream_t s) {
  galerkin_impl<GAL_FINE_K>(gf, gc, fixed_f, scale, Ke0, W, Kc, s);
}
void launch_galerkin_fine_G(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* Gs,
                            const double* W, double* Gc, cudaStream_t s) {
  galerkin_impl<GAL_FINE_G>(gf, gc, fixed_f, Gs, nullptr, W, Gc, s);
}
void launch_galerkin_scaled_stored(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* Kf,
                                   const double* scale, const double* W, double* Kc, cudaStream_t s) {
  galerkin_impl<GAL_SCALED_STORED>(gf, gc, fixed_f, Kf, scale, W, Kc, s);
}
void launch_galerkin_stored(const Grid& gf, const Grid& gc, const uint8_t* fixed_f, const double* Kf,
                            const double* W, double* Kc, cudaStream_t s) {
  galerkin_impl<GAL_STORED>(gf, gc, fixed_f, Kf, nullptr, W, Kc, s);
}

// ================================================================================================
// element stress stiffness from the Gauss-point stresses of u (Sec. 2)
// ================================================================================================
template <int DIM>
__global__ void k_stress_gs(Grid g, const double* __restrict__ u, const double* __restrict__ Es,
                            const double* __restrict__ dN, const double* __restrict__ D, double wdet,
                            double* __restrict__ Gs0, double* __restrict__ Gs) {
  constexpr int NN = Dims<DIM>::NN;
  constexpr int NV = Dims<DIM>::NV;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.m) return;
  const int ei = (int)(e % g.nel[0]);
  const int64_t rest = e / g.nel[0];
  const int ej = (int)(rest % g.nel[1]);
  const int ek = (int)(rest / g.nel[1]);
  const int64_t n0 = ei + (int64_t)g.nn[0] * (ej + (int64_t)g.nn[1] * ek);
  double ue[NN][DIM];
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    const int64_t nb = n0 + corner_x(l) + (int64_t)g.nn[0] * (corner_y(l) + (int64_t)g.nn[1] * corner_z(l));
#pragma unroll
    for (int c = 0; c < DIM; ++c) ue[l][c] = u[DIM * nb + c];
  }
  double G[NN][NN];
#pragma unroll
  for (int a = 0; a < NN; ++a)
#pragma unroll
    for (int b = 0; b < NN; ++b) G[a][b] = 0.0;
  for (int gp = 0; gp < NN; ++gp) {
    const double* dn = dN + gp * DIM * NN;
    double H[DIM][DIM];  // H[a][c] = d u_c / d x_a
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < NN; ++l) s += dn[a * NN + l] * ue[l][c];
        H[a][c] = s;
      }
    double eps[NV];
    if (DIM == 2) {
      eps[0] = H[0][0];
      eps[1] = H[1][1];
      eps[2] = H[0][1] + H[1][0];
    } else {
      eps[0] = H[0][0];
      eps[1] = H[1][1];
      eps[2] = H[DIM - 1][DIM - 1];
      eps[3] = H[0][1] + H[1][0];
      eps[4] = H[1][DIM - 1] + H[DIM - 1][1];
      eps[5] = H[DIM - 1][0] + H[0][DIM - 1];
    }
    double sig[NV];
#pragma unroll
    for (int p = 0; p < NV; ++p) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < NV; ++q) s += D[p * NV + q] * eps[q];
      sig[p] = s;
    }
    double S[DIM][DIM];
    if (DIM == 2) {
      S[0][0] = sig[0];
      S[1][1] = sig[1];
      S[0][1] = S[1][0] = sig[2];
    } else {
      S[0][0] = sig[0];
      S[1][1] = sig[1];
      S[DIM - 1][DIM - 1] = sig[2];
      S[0][1] = S[1][0] = sig[3];
      S[1][DIM - 1] = S[DIM - 1][1] = sig[4];
      S[DIM - 1][0] = S[0][DIM - 1] = sig[5];
    }
    double SdN[DIM][NN];
#pragma unroll
    for (int p = 0; p < DIM; ++p)
#pragma unroll
      for (int b = 0; b < NN; ++b) {
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < DIM; ++q) s += S[p][q] * dn[q * NN + b];
        SdN[p][b] = s;
      }
#pragma unroll
    for (int a = 0; a < NN; ++a)
#pragma unroll
      for (int b = 0; b < NN; ++b) {
        double s = 0.0;
#pragma unroll
        for (int p = 0; p < DIM; ++p) s += dn[p * NN + a] * SdN[p][b];
        G[a][b] += wdet * s;
      }
  }
  const double es = Es[e];
#pragma unroll
  for (int a = 0; a < NN; ++a)
#pragma unroll
    for (int b = 0; b < NN; ++b) {
      Gs0[e * NN * NN + a * NN + b] = G[a][b];
      Gs[e * NN * NN + a * NN + b] = es * G[a][b];
    }
}

void launch_stress_gs_dev(const Grid& g, const double* u, const double* Es, const double* dN, const double* D,
                          double wdet, double* Gs0, double* Gs, cudaStream_t s) {
  if (g.dim == 2)
    ::tobk::note_launch(), k_stress_gs<2><<<blocks_for(g.m, 128), 128, 0, s>>>(g, u, Es, dN, D, wdet, Gs0, Gs);
  else
    ::tobk::note_launch(), k_stress_gs<3><<<blocks_for(g.m, 128), 128, 0, s>>>(g, u, Es, dN, D, wdet, Gs0, Gs);
}

// ================================================================================================
// SIMP and elementwise helpers
// ================================================================================================
__global__ void k_simp(const double* __restrict__ x, int64_t m, double penal, double E0, double Emin, double* Ek,
                       double* Es, double* dEk, double* dEs, float* Ek32) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m) return;
  const double xe = x[e];
  const double xp = pow(xe, penal);
  const double dxp = penal * pow(xe, penal - 1.0);
  const double ek = Emin + xp * (E0 - Emin);
  Ek[e] = ek;
  Es[e] = xp * E0;
  dEk[e] = dxp * (E0 - Emin);
  dEs[e] = dxp * E0;
  if (Ek32) Ek32[e] = (float)ek;
}

void launch_simp(const double* x, int64_t m, double penal, double E0, double Emin, double* Ek, double* Es,
                 double* dEk, double* dEs, float* Ek32, cudaStream_t s) {
  ::tobk::note_launch(), k_simp<<<blocks_for(m), kThreads, 0, s>>>(x, m, penal, E0, Emin, Ek, Es, dEk, dEs, Ek32);
}

__global__ void k_f64_to_f32(const double* a, float* b, int64_t n) {
  pdl_wait();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_f32_to_f64(const float* a, double* b, int64_t n) {
  pdl_wait();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}
void launch_f64_to_f32(const double* a, float* b, int64_t n, cudaStream_t s) {
  launch_pdl(k_f64_to_f32, dim3(blocks_for(n)), dim3(kThreads), 0, s, a, b, n);
}
void launch_f32_to_f64(const float* a, double* b, int64_t n, cudaStream_t s) {
  launch_pdl(k_f32_to_f64, dim3(blocks_for(n)), dim3(kThreads), 0, s, a, b, n);
}

__global__ void k_mask_copy(const double* __restrict__ src, const uint8_t* __restrict__ fixed, double* __restrict__ dst,
                            int64_t n, int64_t stride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t off = (int64_t)blockIdx.y * stride;
  dst[off + i] = fixed[i] ? 0.0 : src[off + i];
}
void launch_mask_copy(const double* src, const uint8_t* fixed, double* dst, int64_t n, int nr, int64_t stride,
                      cudaStream_t s) {
  ::tobk::note_launch(), k_mask_copy<<<dim3(blocks_for(n), nr), kThreads, 0, s>>>(src, fixed, dst, n, stride);
}

// ================================================================================================
// multi-RHS preconditioned CG (Appendix A: mgPCG); one RHS per blockIdx.y, scalars on the device
// ================================================================================================
constexpr int kVecBlocks = 4 * 152;  // vector kernels: grid-stride over DOFs with a fixed grid

// Blocks per right-hand side of the grid-stride vector kernels: about kVecBlocks in total over the
// nr right-hand sides (each block then streams many elements; thousands of short blocks would pay
// their reduction and scheduling cost more often than they move data), at most one per kThreads DOFs.
inline unsigned vec_blocks(int64_t n, int nr) {
  const int64_t per = std::max<int64_t>(8, (kVecBlocks + nr - 1) / std::max(nr, 1));
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(per, (n + kThreads - 1) / kThreads));
}

__device__ __forceinline__ double* rhs_sc(double* sc, int r) { return sc + (size_t)r * kScStride; }

template <int DIM, class Op>
__global__ void __launch_bounds__(kThreads) k_cg_init(const __grid_constant__ Op op, const double* __restrict__ b, double* __restrict__ x,
                                                       double* __restrict__ r, int use_x0, double rtol,
                                                       int64_t stride, double* sc, double* partial,
                                                       unsigned* counters, int64_t pstride, CGZ0 z0) {
  pdl_wait();
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t off = (int64_t)rhs * stride;
  int i, j, k;
  double v[2] = {0.0, 0.0};  // b.b, r.r
  if (node_coords(op.g, node, i, j, k)) {
    double acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = 0.0;
    if (use_x0) gather_rows<DIM, double>(op, i, j, k, LoadVec<double>{x + off}, acc);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t idx = DIM * node + c;
      const double bi = op.fixed[idx] ? 0.0 : b[off + idx];
      const double ri = op.fixed[idx] ? 0.0 : bi - acc[c];
      r[off + idx] = ri;
      if (z0.z) {
        const double zi = z0.coef[1] * z0.dinv[idx] * ri;
        z0.z[off + idx] = zi;
        if (z0.d) z0.d[off + idx] = zi;
      }
      if (!use_x0) x[off + idx] = 0.0;
      v[0] += bi * bi;
      v[1] += ri * ri;
    }
  }
  double tot[2];
  if (grid_sum_last<2>(v, partial + rhs * pstride, counters + rhs, tot, smem) && threadIdx.x == 0) {
    double* s = rhs_sc(sc, rhs);
    for (int q = 0; q < kScStride; ++q) s[q] = 0.0;
    s[SC_BB] = tot[0];
    s[SC_RR] = tot[1];
    s[SC_RTOL] = rtol;
    s[SC_ZR_OLD] = 1.0;
    s[SC_PQ] = 1.0;
    const double rel = tot[0] > 0.0 ? sqrt(tot[1] / tot[0]) : 0.0;
    s[SC_RELRES] = rel;
    s[SC_ACTIVE] = (tot[0] > 0.0 && rel > rtol) ? 1.0 : 0.0;
    if (!isfinite(tot[1])) {
      s[SC_STATUS] = 2.0;
      s[SC_ACTIVE] = 0.0;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_cg_dots(int64_t n, const double* __restrict__ z,
                                                       const double* __restrict__ r, const double* __restrict__ q,
                                                       const double* __restrict__ p, int flexible, int64_t stride,
                                                       double* sc, double* partial, unsigned* counters,
                                                       int64_t pstride) {
  pdl_wait();
  __shared__ double smem[96];
  const int rhs = blockIdx.y;
  double* s = rhs_sc(sc, rhs);
  if (s[SC_ACTIVE] == 0.0) return;
  const int64_t off = (int64_t)rhs * stride;
  double v[3] = {0.0, 0.0, 0.0};  // z.r, z.q_old, p_old.r
  // two grid-stride elements per trip, loads first (twice the loads in flight), summed in the order
  // of the plain grid-stride loop
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + step < n; i += 2 * step) {
    const double z0 = z[off + i], r0 = r[off + i], q0 = q[off + i], p0 = p[off + i];
    const double z1 = z[off + i + step], r1 = r[off + i + step], q1 = q[off + i + step], p1 = p[off + i + step];
    v[0] += z0 * r0;
    v[1] += z0 * q0;
    v[2] += p0 * r0;
    v[0] += z1 * r1;
    v[1] += z1 * q1;
    v[2] += p1 * r1;
  }
  if (i < n) {
    const double zi = z[off + i], ri = r[off + i];
    v[0] += zi * ri;
    v[1] += zi * q[off + i];
    v[2] += p[off + i] * ri;
  }
  double tot[3];
  if (grid_sum_last<3>(v, partial + rhs * pstride, counters + rhs, tot, smem) && threadIdx.x == 0) {
    const double zr = tot[0], zq = tot[1], pr = tot[2];
    double beta = 0.0;
    if (s[SC_ITERS] > 0.0) beta = flexible ? -zq / s[SC_PQ] : zr / s[SC_ZR_OLD];
    s[SC_BETA] = beta;
    s[SC_ZR] = zr;
    s[SC_ZR_OLD] = zr;
    s[SC_PR] = zr + beta * pr;
    if (!isfinite(beta) || !isfinite(zr)) {
      s[SC_STATUS] = 2.0;
      s[SC_ACTIVE] = 0.0;
    }
  }
}

template <int DIM, class Op>
__global__ void __launch_bounds__(kThreads) k_cg_direction(const __grid_constant__ Op op, const double* __restrict__ z,
                                                            const double* __restrict__ p_old,
                                                            double* __restrict__ p_new, double* __restrict__ q,
                                                            int64_t stride, double* sc, double* partial,
                                                            unsigned* counters, int64_t pstride) {
  pdl_wait();
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  double* s = rhs_sc(sc, rhs);
  if (s[SC_ACTIVE] == 0.0) return;
  const int64_t off = (int64_t)rhs * stride;
  const LoadAxpy ld{z + off, p_old + off, s[SC_BETA]};
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  double v[1] = {0.0};
  if (node_coords(op.g, node, i, j, k)) {
    double acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = 0.0;
    gather_rows<DIM, double>(op, i, j, k, ld, acc);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t idx = DIM * node + c;
      const bool fx = op.fixed[idx];
      const double pi = fx ? 0.0 : ld(idx);
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

__global__ void __launch_bounds__(kThreads) k_cg_update(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                                         const double* __restrict__ p, const double* __restrict__ q,
                                                         int64_t stride, double* sc, double* partial,
                                                         unsigned* counters, int64_t pstride, CGZ0 z0) {
  pdl_wait();
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  double* s = rhs_sc(sc, rhs);
  if (s[SC_ACTIVE] == 0.0) return;
  const int64_t off = (int64_t)rhs * stride;
  const double alpha = s[SC_ALPHA];
  double v[1] = {0.0};
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + step < n; i += 2 * step) {  // as in k_cg_dots: two elements per trip, plain order
    const double x0 = x[off + i], p0 = p[off + i], r0 = r[off + i], q0 = q[off + i];
    const double x1 = x[off + i + step], p1 = p[off + i + step], r1 = r[off + i + step], q1 = q[off + i + step];
    x[off + i] = x0 + alpha * p0;
    x[off + i + step] = x1 + alpha * p1;
    const double ra = r0 - alpha * q0, rb = r1 - alpha * q1;
    r[off + i] = ra;
    r[off + i + step] = rb;
    v[0] += ra * ra;
    v[0] += rb * rb;
    if (z0.z) {
      const double za = z0.coef[1] * z0.dinv[i] * ra, zb = z0.coef[1] * z0.dinv[i + step] * rb;
      z0.z[off + i] = za;
      z0.z[off + i + step] = zb;
      if (z0.d) {
        z0.d[off + i] = za;
        z0.d[off + i + step] = zb;
      }
    }
  }
  if (i < n) {
    x[off + i] += alpha * p[off + i];
    const double ri = r[off + i] - alpha * q[off + i];
    r[off + i] = ri;
    v[0] += ri * ri;
    if (z0.z) {
      const double zi = z0.coef[1] * z0.dinv[i] * ri;
      z0.z[off + i] = zi;
      if (z0.d) z0.d[off + i] = zi;
    }
  }
  double tot[1];
  if (grid_sum_last<1>(v, partial + rhs * pstride, counters + rhs, tot, smem) && threadIdx.x == 0) {
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
}

template <int DIM, class Op>
__global__ void __launch_bounds__(kThreads) k_true_residual(const __grid_constant__ Op op, const double* __restrict__ b,
                                                             const double* __restrict__ x, double* __restrict__ r,
                                                             int64_t stride, double* sc, double* partial,
                                                             unsigned* counters, int64_t pstride) {
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  const int64_t off = (int64_t)rhs * stride;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  double v[2] = {0.0, 0.0};
  if (node_coords(op.g, node, i, j, k)) {
    double acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = 0.0;
    gather_rows<DIM, double>(op, i, j, k, LoadVec<double>{x + off}, acc);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t idx = DIM * node + c;
      const double bi = op.fixed[idx] ? 0.0 : b[off + idx];
      const double ri = op.fixed[idx] ? 0.0 : bi - acc[c];
      r[off + idx] = ri;
      v[0] += ri * ri;
      v[1] += bi * bi;
    }
  }
  double tot[2];
  if (grid_sum_last<2>(v, partial + rhs * pstride, counters + rhs, tot, smem) && threadIdx.x == 0) {
    double* s = rhs_sc(sc, rhs);
    s[SC_RR] = tot[0];
    s[SC_BB] = tot[1];
    s[SC_RELRES] = tot[1] > 0.0 ? sqrt(tot[0] / tot[1]) : sqrt(tot[0]);
  }
}

int64_t cg_partial_stride(const Grid& g) {
  const int64_t a = (g.nnode + kThreads - 1) / kThreads;
  return 4 * std::max<int64_t>(std::max<int64_t>(a, kVecBlocks), g.dim == 2 ? fine_q4_tiles(g) : fine_h8_blocks(g));
}

template <int DIM, class Op>
static void cg_init_impl(const Op& op, const double* b, double* x, double* r, bool use_x0, double rtol, int nr,
                         int64_t stride, double* sc, double* partial, unsigned* counters, cudaStream_t s, CGZ0 z0) {
  const int64_t ps = cg_partial_stride(op.g);
  launch_pdl(k_cg_init<DIM, Op>, dim3(dim3(blocks_for(op.g.nnode), nr)), dim3(kThreads), 0, s, op, b, x, r, use_x0 ? 1 : 0, rtol,
                                                                            stride, sc, partial, counters, ps, z0);
}

void launch_cg_init(const LevelOpDesc& d, const double* b, double* x, double* r, bool use_x0, double rtol, int nr,
                    int64_t stride, double* sc, double* partial, unsigned* counters, cudaStream_t s, CGZ0 z0) {
  if (d.g.dim == 2) {
    if (d.stored)
      cg_init_impl<2>(make_stored<2, double>(d, d.Ke64), b, x, r, use_x0, rtol, nr, stride, sc, partial, counters, s,
                      z0);
    else
      cg_init_impl<2>(make_fine<2, double>(d, d.scale64), b, x, r, use_x0, rtol, nr, stride, sc, partial, counters,
                      s, z0);
  } else {
    if (d.stored)
      cg_init_impl<3>(make_stored<3, double>(d, d.Ke64), b, x, r, use_x0, rtol, nr, stride, sc, partial, counters, s,
                      z0);
    else
      cg_init_impl<3>(make_fine<3, double>(d, d.scale64), b, x, r, use_x0, rtol, nr, stride, sc, partial, counters,
                      s, z0);
  }
}

void launch_cg_dots(int64_t n, const double* z, const double* r, const double* q, const double* p, bool flexible,
                    int nr, int64_t stride, double* sc, double* partial, unsigned* counters, cudaStream_t s) {
  const int64_t ps = 4 * kVecBlocks;
  const unsigned g = vec_blocks(n, nr);
  launch_pdl(k_cg_dots, dim3(dim3(g, nr)), dim3(kThreads), 0, s, n, z, r, q, p, flexible ? 1 : 0, stride, sc, partial, counters + kMaxRhs, ps);
}

template <int DIM, class Op>
static void cg_dir_impl(const Op& op, const double* z, const double* p_old, double* p_new, double* q, int nr,
                        int64_t stride, double* sc, double* partial, unsigned* counters, cudaStream_t s) {
  const int64_t ps = cg_partial_stride(op.g);
  launch_pdl(k_cg_direction<DIM, Op>, dim3(dim3(blocks_for(op.g.nnode), nr)), dim3(kThreads), 0, s, op, z, p_old, p_new, q, stride, sc,
                                                                                 partial, counters + 2 * kMaxRhs, ps);
}

void launch_cg_direction(const LevelOpDesc& d, const double* z, const double* p_old, double* p_new, double* q,
                         int nr, int64_t stride, double* sc, double* partial, unsigned* counters, cudaStream_t s) {
  if (d.S64) {  // stencil level: 3^d d^2 multiply-adds per row instead of the element matrices
    launch_stencil_cg_direction(d.g, d.S64, d.fixed, z, p_old, p_new, q, nr, stride, sc, partial,
                                counters + 2 * kMaxRhs, cg_partial_stride(d.g), s);
    return;
  }
  if (d.g.dim == 2 && !d.stored) {
    launch_fine_q4_cg_direction(d.g, d.scale64, d.fixed, d.T0, z, p_old, p_new, q, nr, stride, sc, partial,
                                counters + 2 * kMaxRhs, cg_partial_stride(d.g), s);
    return;
  }
  if (d.g.dim == 3 && !d.stored) {
    launch_fine_h8_cg_direction(d.g, d.scale64, d.fixed, d.nu, d.element, z, p_old, p_new, q, nr, stride, sc, partial,
                                counters + 2 * kMaxRhs, cg_partial_stride(d.g), s);
    return;
  }
  if (d.g.dim == 2) {
    if (d.stored)
      cg_dir_impl<2>(make_stored<2, double>(d, d.Ke64), z, p_old, p_new, q, nr, stride, sc, partial, counters, s);
    else
      cg_dir_impl<2>(make_fine<2, double>(d, d.scale64), z, p_old, p_new, q, nr, stride, sc, partial, counters, s);
  } else {
    if (d.stored)
      cg_dir_impl<3>(make_stored<3, double>(d, d.Ke64), z, p_old, p_new, q, nr, stride, sc, partial, counters, s);
    else
      cg_dir_impl<3>(make_fine<3, double>(d, d.scale64), z, p_old, p_new, q, nr, stride, sc, partial, counters, s);
  }
}

void launch_cg_update(int64_t n, double* x, double* r, const double* p, const double* q, int nr, int64_t stride,
                      double* sc, double* partial, unsigned* counters, cudaStream_t s, CGZ0 z0) {
  const int64_t ps = 4 * kVecBlocks;
  const unsigned g = vec_blocks(n, nr);
  launch_pdl(k_cg_update, dim3(dim3(g, nr)), dim3(kThreads), 0, s, n, x, r, p, q, stride, sc, partial,
                                                                      counters + 3 * kMaxRhs, ps, z0);
}

template <int DIM, class Op>
static void true_res_impl(const Op& op, const double* b, const double* x, double* r, int nr, int64_t stride,
                          double* sc, double* partial, unsigned* counters, cudaStream_t s) {
  const int64_t ps = cg_partial_stride(op.g);
  ::tobk::note_launch(), k_true_residual<DIM, Op><<<dim3(blocks_for(op.g.nnode), nr), kThreads, 0, s>>>(op, b, x, r, stride, sc, partial,
                                                                                  counters + 4 * kMaxRhs, ps);
}

void launch_true_residual(const LevelOpDesc& d, const double* b, const double* x, double* r, int nr, int64_t stride,
                          double* sc, double* partial, unsigned* counters, cudaStream_t s) {
  if (d.g.dim == 2) {
    if (d.stored)
      true_res_impl<2>(make_stored<2, double>(d, d.Ke64), b, x, r, nr, stride, sc, partial, counters, s);
    else
      true_res_impl<2>(make_fine<2, double>(d, d.scale64), b, x, r, nr, stride, sc, partial, counters, s);
  } else {
    if (d.stored)
      true_res_impl<3>(make_stored<3, double>(d, d.Ke64), b, x, r, nr, stride, sc, partial, counters, s);
    else
      true_res_impl<3>(make_fine<3, double>(d, d.scale64), b, x, r, nr, stride, sc, partial, counters, s);
  }
}

// ================================================================================================
// tall-skinny block products for the block eigensolver
// ================================================================================================
constexpr int kGramChunk = 32;  // smallest chunk of rows per block

// SMs of the current device (queried once per device).
static int device_sm_count() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 152;
  if (cached[dev] == 0) {
    int c = 0;
    cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = c > 0 ? c : 152;
  }
  return cached[dev];
}

// Rows per block of the Gram product: the n rows are split into two chunks per SM (the product runs
// at GB300's FP64 rate of 2 FMA per clock per SM, so an SM with one chunk more than the others sets
// the time of the launch; two resident blocks per SM overlap one block's loads with the other's
// multiply-adds), at least kGramChunk rows and no more than the shared memory holds.
static int gram_chunk_rows(int na, int nb, int64_t n) {
  const int64_t per_sm = (n + 2 * device_sm_count() - 1) / (2 * device_sm_count());
  const int chunk = (int)std::min<int64_t>(std::max<int64_t>(per_sm, kGramChunk), 1 << 20);
  const int cap = std::max(kGramChunk, (int)((200 * 1024) / (sizeof(double) * (size_t)(na + nb))) - 1);
  return std::min(chunk, cap);
}

// partial[chunk][i][j] = sum_{k in chunk} A[i][k] B[j][k]; shared rows of odd stride len + 1.
__global__ void k_gram_partial(const double* __restrict__ A, int na, const double* __restrict__ B, int nb, int64_t n,
                               int64_t stride, int chunk, double* __restrict__ partial) {
  pdl_wait();
  extern __shared__ double sm[];
  const int ldc = chunk + 1;
  double* sA = sm;              // [na][ldc]
  double* sB = sm + na * ldc;   // [nb][ldc]
  const int64_t k0 = (int64_t)blockIdx.x * chunk;
  const int len = (n - k0) < chunk ? (int)(n - k0) : chunk;
  for (int t = threadIdx.x; t < na * chunk; t += blockDim.x) {
    const int i = t / chunk, kk = t % chunk;
    sA[i * ldc + kk] = kk < len ? A[(int64_t)i * stride + k0 + kk] : 0.0;
  }
  for (int t = threadIdx.x; t < nb * chunk; t += blockDim.x) {
    const int j = t / chunk, kk = t % chunk;
    sB[j * ldc + kk] = kk < len ? B[(int64_t)j * stride + k0 + kk] : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < na * nb; t += blockDim.x) {
    const int i = t / nb, j = t % nb;
    const double* a = sA + i * ldc;
    const double* b = sB + j * ldc;
    double s = 0.0;
#pragma unroll 8
    for (int kk = 0; kk < len; ++kk) s += a[kk] * b[kk];
    partial[(size_t)blockIdx.x * na * nb + t] = s;
  }
}

// C[o] = sum over chunks of partial[c][o]: a block sums 32 consecutive outputs, its 8 warps take every
// 8th chunk (coalesced over the outputs) and the 8 partial sums are added in a fixed order.
__global__ void __launch_bounds__(256) k_gram_final(const double* __restrict__ partial, int nchunks, int nout,
                                                    double* __restrict__ C) {
  pdl_wait();
  __shared__ double red[8][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  double s = 0.0;
  if (o < nout)
    for (int c = w; c < nchunks; c += 8) s += partial[(size_t)c * nout + o];
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && o < nout) {
    double a = red[0][lane];
#pragma unroll
    for (int k = 1; k < 8; ++k) a += red[k][lane];
    C[o] = a;
  }
}

// Upper bound of the chunks of any Gram product over n rows with na, nb <= 64 (sizes the partial
// buffer): a chunk holds at least min(max(n / (2 SMs), kGramChunk), 199) rows, since the shared-memory
// cap of gram_chunk_rows is at least 199 rows for na + nb <= 128.
int gram_partial_blocks(int64_t n) {
  const int64_t per_sm = (n + 2 * device_sm_count() - 1) / (2 * device_sm_count());
  const int64_t cmin = std::min<int64_t>(std::max<int64_t>(per_sm, kGramChunk), 199);
  return (int)((n + cmin - 1) / cmin);
}

void launch_gram_final(const double* partial, int nchunks, int nout, double* C, cudaStream_t s) {
  launch_pdl(k_gram_final, dim3((nout + 31) / 32), dim3(256), 0, s, partial, nchunks, nout, C);
}

void launch_gram(const double* A, int na, const double* B, int nb, int64_t n, int64_t stride, double* C,
                 double* partial, cudaStream_t s) {
  const int chunk = gram_chunk_rows(na, nb, n);
  const int chunks = (int)((n + chunk - 1) / chunk);
  const size_t smem = sizeof(double) * (size_t)(na + nb) * (chunk + 1);
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_gram_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024 + 1024);
    configured = true;
  }
  launch_pdl(k_gram_partial, dim3(chunks), dim3(kThreads), smem, s, A, na, B, nb, n, stride, chunk, partial);
  launch_pdl(k_gram_final, dim3((na * nb + 31) / 32), dim3(256), 0, s, partial, chunks, na * nb, C);
}

// Y[j] = beta * Y[j] + alpha * sum_i X[i] C[i][j].  A work item is one row index k and kCombineJ
// consecutive output columns (items ordered row-fastest, so loads of X and stores of Y coalesce).
// The items are cut into equal contiguous ranges, one per block, and the grid is a fixed number of
// blocks per SM, so that every SM gets the same share of the FP64 multiply-adds even when the
// vectors are short (GB300 runs FP64 at 2 FMA per clock per SM: an SM with one extra block sets the
// time of the launch).
constexpr int kCombineJ = 2;
constexpr int kCombineThreads = 128;
__global__ void __launch_bounds__(kCombineThreads) k_combine(const double* __restrict__ X, int nx,
                                                             const double* __restrict__ C, int ldc, int ny,
                                                             double alpha, double beta, double* __restrict__ Y,
                                                             int64_t n, int64_t stride, int64_t per_block) {
  pdl_wait();
  const int groups = (ny + kCombineJ - 1) / kCombineJ;
  const int64_t items = n * groups;
  const int64_t end = min(items, ((int64_t)blockIdx.x + 1) * per_block);
  for (int64_t it = (int64_t)blockIdx.x * per_block + threadIdx.x; it < end; it += blockDim.x) {
    const int64_t k = it % n;
    const int j0 = (int)(it / n) * kCombineJ;
    const int nj = min(kCombineJ, ny - j0);
    double acc[kCombineJ];
#pragma unroll
    for (int j = 0; j < kCombineJ; ++j) acc[j] = 0.0;
    for (int i = 0; i < nx; ++i) {
      const double xi = __ldg(X + (int64_t)i * stride + k);
      const double* ci = C + (size_t)i * ldc + j0;
#pragma unroll
      for (int j = 0; j < kCombineJ; ++j)
        if (j < nj) acc[j] += xi * __ldg(ci + j);
    }
#pragma unroll
    for (int j = 0; j < kCombineJ; ++j) {
      if (j < nj) {
        double* y = Y + (int64_t)(j0 + j) * stride + k;
        *y = (beta == 0.0 ? 0.0 : beta * *y) + alpha * acc[j];
      }
    }
  }
}

// Y_s[j] = sum_i X_s[i] C[i][j] for nsrc <= 3 pairs (X_s, Y_s) sharing the coefficients C: a block
// of basis vectors and its K and G images in one launch.  Items as in k_combine, source slowest.
struct CombineSet {
  const double* X[3];
  double* Y[3];
};
__global__ void __launch_bounds__(kCombineThreads) k_combine_set(CombineSet cs, int nsrc, int nx,
                                                                 const double* __restrict__ C, int ldc, int ny,
                                                                 int64_t n, int64_t stride, int64_t per_block) {
  pdl_wait();
  const int groups = (ny + kCombineJ - 1) / kCombineJ;
  const int64_t per_src = n * groups;
  const int64_t items = per_src * nsrc;
  const int64_t end = min(items, ((int64_t)blockIdx.x + 1) * per_block);
  for (int64_t it = (int64_t)blockIdx.x * per_block + threadIdx.x; it < end; it += blockDim.x) {
    const int src = (int)(it / per_src);
    const int64_t rem = it - (int64_t)src * per_src;
    const int64_t k = rem % n;
    const int j0 = (int)(rem / n) * kCombineJ;
    const int nj = min(kCombineJ, ny - j0);
    const double* X = src == 0 ? cs.X[0] : (src == 1 ? cs.X[1] : cs.X[2]);
    double* Y = src == 0 ? cs.Y[0] : (src == 1 ? cs.Y[1] : cs.Y[2]);
    double acc[kCombineJ];
#pragma unroll
    for (int j = 0; j < kCombineJ; ++j) acc[j] = 0.0;
    for (int i = 0; i < nx; ++i) {
      const double xi = __ldg(X + (int64_t)i * stride + k);
      const double* ci = C + (size_t)i * ldc + j0;
#pragma unroll
      for (int j = 0; j < kCombineJ; ++j)
        if (j < nj) acc[j] += xi * __ldg(ci + j);
    }
#pragma unroll
    for (int j = 0; j < kCombineJ; ++j)
      if (j < nj) Y[(int64_t)(j0 + j) * stride + k] = acc[j];
  }
}

void launch_combine3(const double* X0, const double* X1, const double* X2, int nx, const double* C, int ldc, int ny,
                     double* Y0, double* Y1, double* Y2, int64_t n, int64_t stride, cudaStream_t s) {
  CombineSet cs{{X0, X1, X2}, {Y0, Y1, Y2}};
  const int64_t items = 3 * n * ((ny + kCombineJ - 1) / kCombineJ);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((items + 31) / 32, 4 * (int64_t)device_sm_count()));
  const int64_t per_block = (items + grid - 1) / grid;
  launch_pdl(k_combine_set, dim3((unsigned)grid), dim3(kCombineThreads), 0, s, cs, 3, nx, C, ldc, ny, n, stride,
                                                                                 per_block);
}

void launch_combine(const double* X, int nx, const double* C, int ldc, int ny, double alpha, double beta, double* Y,
                    int64_t n, int64_t stride, cudaStream_t s) {
  const int64_t items = n * ((ny + kCombineJ - 1) / kCombineJ);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((items + 31) / 32, 4 * (int64_t)device_sm_count()));
  const int64_t per_block = (items + grid - 1) / grid;
  launch_pdl(k_combine, dim3((unsigned)grid), dim3(kCombineThreads), 0, s, X, nx, C, ldc, ny, alpha, beta, Y, n,
                                                                             stride, per_block);
}

}  // namespace tobk
