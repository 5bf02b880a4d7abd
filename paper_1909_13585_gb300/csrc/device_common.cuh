// Device-side building blocks shared by the kernels of the library: element-local numbering,
// the matrix-free and stored-matrix element operators, node-gather products and deterministic
// block reductions.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "tobk_internal.cuh"

namespace tobk {

template <int DIM>
struct Dims {
  static constexpr int NN = 1 << DIM;        // nodes per element
  static constexpr int ND = DIM * NN;        // DOFs per element
  static constexpr int NV = DIM == 2 ? 3 : 6;  // Voigt components
  static constexpr int NGP = NN;             // 2-point Gauss rule per axis
};

// Corner offsets of the local nodes: Q4 order (0,0) (1,0) (1,1) (0,1), H8 = Q4 on z=0 then z=1.
__host__ __device__ constexpr int corner_x(int ln) { return ((ln & 3) == 1 || (ln & 3) == 2) ? 1 : 0; }
__host__ __device__ constexpr int corner_y(int ln) { return ((ln & 3) >= 2) ? 1 : 0; }
__host__ __device__ constexpr int corner_z(int ln) { return ln >> 2; }
__host__ __device__ constexpr int local_node(int cx, int cy, int cz) {
  return (cy ? (cx ? 2 : 3) : (cx ? 1 : 0)) + 4 * cz;
}

// True in blocks whose right-hand side (blockIdx.y) has stopped iterating: multi-RHS kernels of the
// V-cycle skip converged columns when the CG driver passes its per-RHS scalar state.
__device__ __forceinline__ bool rhs_done(const double* act) {
  return act != nullptr && act[(size_t)blockIdx.y * kScStride + SC_ACTIVE] == 0.0;
}

// ------------------------------------------------------------------------------------------------
// element operators
// ------------------------------------------------------------------------------------------------
// Fine level: K_e = s_e * T0, with T0 a constant (unit-modulus) element matrix held in the kernel's
// parameter space and s_e a per-element scale (E_kappa(x_e), or E_sigma for the G operator built
// from K-shaped tables).
template <int DIM, typename T>
struct FineOp {
  Grid g;
  const T* scale_e;          // [m]
  const uint8_t* fixed;      // [n]
  T M[Dims<DIM>::ND * Dims<DIM>::ND];
  __device__ __forceinline__ T scale(int64_t e) const { return scale_e[e]; }
  __device__ __forceinline__ T entry(int64_t, int r, int c) const { return M[r * Dims<DIM>::ND + c]; }
};

// Stored element matrices, one dense (ND x ND) row-major block per element.
template <int DIM, typename T>
struct StoredOp {
  Grid g;
  const T* Ke;               // [m][ND*ND]
  const uint8_t* fixed;      // [n]
  __device__ __forceinline__ T scale(int64_t) const { return T(1); }
  __device__ __forceinline__ T entry(int64_t e, int r, int c) const {
    return __ldg(Ke + e * (Dims<DIM>::ND * Dims<DIM>::ND) + r * Dims<DIM>::ND + c);
  }
};

// Per-element scalar-field operator (the stress stiffness): K_e = Gs_e (x) I_d, Gs_e a stored
// symmetric (NN x NN) matrix that already includes E_sigma(x_e).
template <int DIM, typename T>
struct ScalarKronOp {
  Grid g;
  const T* Gs;               // [m][NN*NN]
  const uint8_t* fixed;
};

template <typename T>
struct LoadVec {
  const T* v;
  __device__ __forceinline__ T operator()(int64_t i) const { return __ldg(v + i); }
};

// v_i = z_i + beta * p_i  (the CG direction, formed on the fly by the matvec)
struct LoadAxpy {
  const double* z;
  const double* p;
  double beta;
  __device__ __forceinline__ double operator()(int64_t i) const { return __ldg(z + i) + beta * __ldg(p + i); }
};

__device__ __forceinline__ bool node_coords(const Grid& g, int64_t node, int& i, int& j, int& k) {
  if (node >= g.nnode) return false;
  i = (int)(node % g.nn[0]);
  int64_t t = node / g.nn[0];
  j = (int)(t % g.nn[1]);
  k = (int)(t / g.nn[1]);
  return true;
}

// acc[c] += sum over the elements adjacent to node (i,j,k) of (K_e v_e) at the node's rows.
template <int DIM, typename Acc, class Op, class Loader>
__device__ __forceinline__ void gather_rows(const Op& op, int i, int j, int k, const Loader& ld, Acc acc[DIM]) {
  constexpr int NN = Dims<DIM>::NN;
  const Grid& g = op.g;
#pragma unroll
  for (int cz = 0; cz < (DIM == 3 ? 2 : 1); ++cz) {
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) {
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const int ei = i - cx, ej = j - cy, ek = k - cz;
        if (ei < 0 || ei >= g.nel[0] || ej < 0 || ej >= g.nel[1]) continue;
        if (DIM == 3 && (ek < 0 || ek >= g.nel[2])) continue;
        const int64_t e = ei + (int64_t)g.nel[0] * (ej + (int64_t)g.nel[1] * ek);
        const int64_t n0 = ei + (int64_t)g.nn[0] * (ej + (int64_t)g.nn[1] * ek);
        const int ln = local_node(cx, cy, cz);
        Acc part[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) part[c] = Acc(0);
#pragma unroll
        for (int lb = 0; lb < NN; ++lb) {
          const int64_t nb = n0 + corner_x(lb) + (int64_t)g.nn[0] * (corner_y(lb) + (int64_t)g.nn[1] * corner_z(lb));
#pragma unroll
          for (int cc = 0; cc < DIM; ++cc) {
            const Acc vb = (Acc)ld(DIM * nb + cc);
#pragma unroll
            for (int c = 0; c < DIM; ++c) part[c] += (Acc)op.entry(e, ln * DIM + c, lb * DIM + cc) * vb;
          }
        }
        const Acc s = (Acc)op.scale(e);
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] += s * part[c];
      }
    }
  }
}

// Same for the scalar-Kronecker operator (stress stiffness): rows of Gs_e (x) I_d.
template <int DIM, typename Acc, typename T, class Loader>
__device__ __forceinline__ void gather_rows_kron(const ScalarKronOp<DIM, T>& op, int i, int j, int k,
                                                 const Loader& ld, Acc acc[DIM]) {
  constexpr int NN = Dims<DIM>::NN;
  const Grid& g = op.g;
#pragma unroll
  for (int cz = 0; cz < (DIM == 3 ? 2 : 1); ++cz) {
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) {
#pragma unroll
      for (int cx = 0; cx < 2; ++cx) {
        const int ei = i - cx, ej = j - cy, ek = k - cz;
        if (ei < 0 || ei >= g.nel[0] || ej < 0 || ej >= g.nel[1]) continue;
        if (DIM == 3 && (ek < 0 || ek >= g.nel[2])) continue;
        const int64_t e = ei + (int64_t)g.nel[0] * (ej + (int64_t)g.nel[1] * ek);
        const int64_t n0 = ei + (int64_t)g.nn[0] * (ej + (int64_t)g.nn[1] * ek);
        const int ln = local_node(cx, cy, cz);
        const T* row = op.Gs + e * (NN * NN) + ln * NN;
#pragma unroll
        for (int lb = 0; lb < NN; ++lb) {
          const int64_t nb = n0 + corner_x(lb) + (int64_t)g.nn[0] * (corner_y(lb) + (int64_t)g.nn[1] * corner_z(lb));
          const Acc w = (Acc)__ldg(row + lb);
#pragma unroll
          for (int c = 0; c < DIM; ++c) acc[c] += w * (Acc)ld(DIM * nb + c);
        }
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// deterministic reductions: warp shuffles, then a fixed-order block tree, then a last-block pass
// over the per-block partials in index order (no floating-point atomics).
// ------------------------------------------------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* smem /* >= 32*NV */) {
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) smem[wid * NV + q] = v[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double t = (lane < nw) ? smem[lane * NV + q] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      v[q] = t;
    }
  }
}

// Writes this block's partials, and returns true in the block that arrives last; that block then
// holds the grid totals in tot[] (valid in thread 0).  partial: [nblocks][NV] for this slot; bid is
// this block's index among the nblocks blocks that reduce into the slot.
template <int NV>
__device__ __forceinline__ bool grid_sum_last_idx(double (&v)[NV], double* partial, unsigned* counter,
                                                  double (&tot)[NV], double* smem, unsigned bid, unsigned nblocks) {
  block_sum<NV>(v, smem);
  __shared__ bool s_last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) partial[(size_t)bid * NV + q] = v[q];
    __threadfence();
    const unsigned ticket = atomicAdd(counter, 1u);
    s_last = (ticket == nblocks - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  double w[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) w[q] = 0.0;
  for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x) {
#pragma unroll
    for (int q = 0; q < NV; ++q) w[q] += __ldcg(partial + (size_t)b * NV + q);
  }
  block_sum<NV>(w, smem);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] = w[q];
    *counter = 0u;
  }
  return true;
}

template <int NV>
__device__ __forceinline__ bool grid_sum_last(double (&v)[NV], double* partial, unsigned* counter,
                                              double (&tot)[NV], double* smem) {
  return grid_sum_last_idx<NV>(v, partial, counter, tot, smem, blockIdx.x, gridDim.x);
}

}  // namespace tobk
