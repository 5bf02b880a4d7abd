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
#pragma unroll
  for (int nbr = 0; nbr < NB; ++nbr) {
    const int dx = nbr % 3 - 1, dy = (nbr / 3) % 3 - 1, dz = DIM == 3 ? nbr / 9 - 1 : 0;
    if (i + dx < 0 || i + dx >= g.nn[0] || j + dy < 0 || j + dy >= g.nn[1]) continue;
    if (DIM == 3 && (k + dz < 0 || k + dz >= g.nn[2])) continue;
    const int64_t nb = node + dx + (int64_t)g.nn[0] * (dy + (int64_t)g.nn[1] * dz);
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
        const T vv = __ldg(vr + cc);
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
  dim3 grid((unsigned)((g.nnode + 255) / 256), (unsigned)((nr + R - 1) / R));
  const double* act = active_rhs();
  note_launch();
  if (mode == APPLY_KV)
    k_apply_stencil<DIM, T, APPLY_KV, R><<<grid, 256, 0, s>>>(g, S, fixed, v, b, dinv, y, sm, nr, stride, act);
  else if (mode == APPLY_RES)
    k_apply_stencil<DIM, T, APPLY_RES, R><<<grid, 256, 0, s>>>(g, S, fixed, v, b, dinv, y, sm, nr, stride, act);
  else
    k_apply_stencil<DIM, T, APPLY_JAC, R><<<grid, 256, 0, s>>>(g, S, fixed, v, b, dinv, y, sm, nr, stride, act);
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

}  // namespace tobk
