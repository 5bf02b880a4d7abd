// Fine-level (matrix-free) K(x) v = sum_e E_kappa(x_e) K_e0 v_e of Sec. 2 (applied inside the mgPCG of
// Algorithm 1 step 3 and Appendix A) for Q4 elements.
//
// Q4 operator in factored form (q4_element.cuh), element by element on
// shared-memory tiles: a block computes the (TX + 1) x (TY + 1) elements around a TX x TY tile of
// nodes once (one element per thread, so the FP64-bound force phase is a single full round), stores
// their nodal forces in shared memory and gathers the four contributions of each node.  On GB300,
// where FP64 runs at 2 FMA/clk/SM, the FP64 fine-level smoother is bound by the element's
// arithmetic, so the ~41 operations of the factored form (against 64 multiply-adds for the dense
// 8 x 8 product) set its speed -- and so does every element a tile computes beyond the grid's own:
// the ring of elements around a tile is computed by each of its neighbours too, and a last tile row
// or column that the grid only partly covers computes its whole element tile.  The tile shape is
// therefore chosen per grid (q4_tile_choice) among a few with a multiple of 32 threads, to minimise
// the elements computed: on the 161 x 481-node column, 24 x 12 elements over 23 x 11 nodes compute
// 88,704 element forces per RHS against 105,984 for 32 x 8 over 31 x 7.
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"
#include "q4_element.cuh"

namespace tobk {

// Node tile TX x TY, element tile (TX + 1) x (TY + 1) = one element per thread.
template <int TX_, int TY_>
struct Q4Tile {
  static constexpr int TX = TX_, TY = TY_;
  static constexpr int EX = TX + 1, EY = TY + 1;  // element tile
  static constexpr int NX = TX + 2, NY = TY + 2;  // node tile with its halo
  static constexpr int kThreads = EX * EY;
  static_assert(kThreads % 32 == 0 && kThreads <= 512, "whole warps, one element per thread");
};

// Element forces of the (EX x EY) element tile into fe, zero outside the grid.
template <typename T, class Tl>
__device__ __forceinline__ void q4_tile_forces(const Grid& g, const T* __restrict__ Ek, const Q4Consts<T>& cst, int x0,
                                               int y0, const T (&su)[Tl::NY][Tl::NX], const T (&sv)[Tl::NY][Tl::NX],
                                               T (&fe)[Tl::EY][Tl::EX][8]) {
  constexpr int EX = Tl::EX, EY = Tl::EY;
  for (int q = threadIdx.x; q < EX * EY; q += Tl::kThreads) {
    const int lx = q % EX, ly = q / EX;
    const int ex = x0 - 1 + lx, ey = y0 - 1 + ly;
    T f[8];
    if (ex >= 0 && ex < g.nel[0] && ey >= 0 && ey < g.nel[1]) {
      q4_forces<T>(su[ly][lx], su[ly][lx + 1], su[ly + 1][lx + 1], su[ly + 1][lx], sv[ly][lx], sv[ly][lx + 1],
                   sv[ly + 1][lx + 1], sv[ly + 1][lx], __ldg(Ek + ex + (int64_t)g.nel[0] * ey), cst, f);
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = T(0);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) fe[ly][lx][k] = f[k];
  }
}

template <typename T, int MODE, class Tl>
__global__ void __launch_bounds__(Tl::kThreads) k_fine_q4(Grid g, const T* __restrict__ Ek, const uint8_t* __restrict__ fixed,
                                                      Q4Consts<T> cst, const T* __restrict__ v, const T* __restrict__ b,
                                                      const T* __restrict__ dinv, T* __restrict__ y, SmoothArgs<T> sm,
                                                      int64_t stride, const double* __restrict__ act) {
  pdl_wait();
  constexpr int TX = Tl::TX, TY = Tl::TY, NX = Tl::NX, NY = Tl::NY, EX = Tl::EX, EY = Tl::EY;
  __shared__ T su[NY][NX], sv[NY][NX];
  __shared__ T fe[EY][EX][8];
  const int rhs = blockIdx.z;
  if (act != nullptr && act[(size_t)rhs * kScStride + SC_ACTIVE] == 0.0) return;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int nnx = g.nn[0], nny = g.nn[1];
  const int64_t off = (int64_t)rhs * stride;
  for (int q = tid; q < NX * NY; q += Tl::kThreads) {
    const int lx = q % NX, ly = q / NX;
    const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
    T a = T(0), c = T(0);
    if (gx >= 0 && gx < nnx && gy >= 0 && gy < nny) {
      const int64_t node = gx + (int64_t)nnx * gy;
      a = __ldg(v + off + 2 * node);
      c = __ldg(v + off + 2 * node + 1);
    }
    su[ly][lx] = a;
    sv[ly][lx] = c;
  }
  __syncthreads();
  q4_tile_forces<T, Tl>(g, Ek, cst, x0, y0, su, sv, fe);
  __syncthreads();
  const int tx = tid % TX, ty = tid / TX;  // threads TX * TY .. only computed elements
  const int X = x0 + tx, Y = y0 + ty;
  if (tid >= TX * TY || X >= nnx || Y >= nny) return;
  // elements around node (X, Y): (X-1,Y-1) local node 2, (X,Y-1) node 3, (X-1,Y) node 1, (X,Y) node 0
  const T fx = fe[ty][tx][4] + fe[ty][tx + 1][6] + fe[ty + 1][tx][2] + fe[ty + 1][tx + 1][0];
  const T fy = fe[ty][tx][5] + fe[ty][tx + 1][7] + fe[ty + 1][tx][3] + fe[ty + 1][tx + 1][1];
  const int64_t node = X + (int64_t)nnx * Y;
  const T acc[2] = {fx, fy};
  const T vloc[2] = {su[ty + 1][tx + 1], sv[ty + 1][tx + 1]};
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const int64_t idx = 2 * node + c;
    T out;
    if (fixed[idx])
      out = T(0);
    else if (MODE == APPLY_KV)
      out = acc[c];
    else if (MODE == APPLY_RES)
      out = b[off + idx] - acc[c];
    else
    {
      const T r = dinv[idx] * (b[off + idx] - acc[c]);
      const T dn = (sm.d_in ? sm.coef[0] * sm.d_in[off + idx] : T(0)) + sm.coef[1] * r;
      if (sm.d_out) sm.d_out[off + idx] = dn;
      out = vloc[c] + dn;
    }
    y[off + idx] = out;
  }
}

// The candidate tile shapes (node tiles; element tiles of 256, 288 and 224 threads) and the one used
// on grid g: the shape that computes the fewest elements (ties: the earlier one).  The choice depends
// on the grid only, not on the number of right-hand sides, so that the block partition of the CG
// reductions -- and with it every right-hand side's result, bit for bit -- is the same however a
// solve is batched or split.
using Q4TileA = Q4Tile<31, 7>;
using Q4TileB = Q4Tile<23, 11>;
using Q4TileC = Q4Tile<15, 13>;
static int64_t q4_tiles_of(const Grid& g, int tx, int ty) {
  return (int64_t)((g.nn[0] + tx - 1) / tx) * ((g.nn[1] + ty - 1) / ty);
}
static int q4_tile_choice(const Grid& g) {
  const int64_t w[3] = {q4_tiles_of(g, Q4TileA::TX, Q4TileA::TY) * Q4TileA::kThreads,
                        q4_tiles_of(g, Q4TileB::TX, Q4TileB::TY) * Q4TileB::kThreads,
                        q4_tiles_of(g, Q4TileC::TX, Q4TileC::TY) * Q4TileC::kThreads};
  int best = 0;
  for (int c = 1; c < 3; ++c)
    if (w[c] < w[best]) best = c;
  return best;
}

template <typename T, class Tl>
static void fine_q4_launch(const Grid& g, const T* Ek, const uint8_t* fixed, const Q4Consts<T>& cst, int mode,
                           const T* v, const T* b, const T* dinv, T* y, SmoothArgs<T> sm, int nr, int64_t stride,
                           const double* act, cudaStream_t s) {
  const dim3 grid((unsigned)((g.nn[0] + Tl::TX - 1) / Tl::TX), (unsigned)((g.nn[1] + Tl::TY - 1) / Tl::TY),
                  (unsigned)nr);
  const dim3 block(Tl::kThreads);
  if (mode == APPLY_KV)
    launch_pdl(k_fine_q4<T, APPLY_KV, Tl>, grid, block, 0, s, g, Ek, fixed, cst, v, b, dinv, y, sm, stride, act);
  else if (mode == APPLY_RES)
    launch_pdl(k_fine_q4<T, APPLY_RES, Tl>, grid, block, 0, s, g, Ek, fixed, cst, v, b, dinv, y, sm, stride, act);
  else
    launch_pdl(k_fine_q4<T, APPLY_JAC, Tl>, grid, block, 0, s, g, Ek, fixed, cst, v, b, dinv, y, sm, stride, act);
}

template <typename T>
void launch_fine_q4(const Grid& g, const T* Ek, const uint8_t* fixed, const double* Ke0, int mode, const T* v,
                    const T* b, const T* dinv, T* y, SmoothArgs<T> sm, int nr, int64_t stride, cudaStream_t s) {
  const Q4Consts<T> cst = q4_consts<T>(Ke0);
  const double* act = active_rhs();
  switch (q4_tile_choice(g)) {
    case 0: fine_q4_launch<T, Q4TileA>(g, Ek, fixed, cst, mode, v, b, dinv, y, sm, nr, stride, act, s); break;
    case 1: fine_q4_launch<T, Q4TileB>(g, Ek, fixed, cst, mode, v, b, dinv, y, sm, nr, stride, act, s); break;
    default: fine_q4_launch<T, Q4TileC>(g, Ek, fixed, cst, mode, v, b, dinv, y, sm, nr, stride, act, s); break;
  }
}

template void launch_fine_q4<double>(const Grid&, const double*, const uint8_t*, const double*, int, const double*,
                                     const double*, const double*, double*, SmoothArgs<double>, int, int64_t,
                                     cudaStream_t);
template void launch_fine_q4<float>(const Grid&, const float*, const uint8_t*, const double*, int, const float*,
                                    const float*, const float*, float*, SmoothArgs<float>, int, int64_t, cudaStream_t);

// Blocks per RHS of the fine Q4 kernels on grid g (the most any candidate tile shape uses, so that
// reduction buffers sized with it hold every choice).
int64_t fine_q4_tiles(const Grid& g) {
  return std::max({q4_tiles_of(g, Q4TileA::TX, Q4TileA::TY), q4_tiles_of(g, Q4TileB::TX, Q4TileB::TY),
                   q4_tiles_of(g, Q4TileC::TX, Q4TileC::TY)});
}

// CG direction on the fine level (FP64): p = z + beta p_old (zero at fixed DOFs), q = K p, and the
// per-RHS reduction p.q -> sc[SC_PQ], alpha = (p.r) / (p.q) (last block of the RHS).
template <class Tl>
__global__ void __launch_bounds__(Tl::kThreads) k_fine_q4_cg_direction(Grid g, const double* __restrict__ Ek,
                                                                 const uint8_t* __restrict__ fixed, Q4Consts<double> cst,
                                                                 const double* __restrict__ z,
                                                                 const double* __restrict__ p_old,
                                                                 double* __restrict__ p_new, double* __restrict__ q,
                                                                 int64_t stride, double* sc, double* partial,
                                                                 unsigned* counters, int64_t pstride) {
  pdl_wait();
  constexpr int TX = Tl::TX, TY = Tl::TY, NX = Tl::NX, NY = Tl::NY, EX = Tl::EX, EY = Tl::EY;
  __shared__ double su[NY][NX], sv[NY][NX];
  __shared__ double fe[EY][EX][8];
  __shared__ double red[64];
  const int rhs = blockIdx.z;
  double* s = sc + (size_t)rhs * kScStride;
  if (s[SC_ACTIVE] == 0.0) return;
  const double beta = s[SC_BETA];
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int nnx = g.nn[0], nny = g.nn[1];
  const int64_t off = (int64_t)rhs * stride;
  for (int t = tid; t < NX * NY; t += Tl::kThreads) {
    const int lx = t % NX, ly = t / NX;
    const int gx = x0 - 1 + lx, gy = y0 - 1 + ly;
    double a = 0.0, c = 0.0;
    if (gx >= 0 && gx < nnx && gy >= 0 && gy < nny) {
      const int64_t i0 = off + 2 * (gx + (int64_t)nnx * gy);
      const int64_t f0 = i0 - off;
      a = fixed[f0] ? 0.0 : __ldg(z + i0) + beta * __ldg(p_old + i0);
      c = fixed[f0 + 1] ? 0.0 : __ldg(z + i0 + 1) + beta * __ldg(p_old + i0 + 1);
    }
    su[ly][lx] = a;
    sv[ly][lx] = c;
  }
  __syncthreads();
  q4_tile_forces<double, Tl>(g, Ek, cst, x0, y0, su, sv, fe);
  __syncthreads();
  const int tx = tid % TX, ty = tid / TX;
  const int X = x0 + tx, Y = y0 + ty;
  double v[1] = {0.0};
  if (tid < TX * TY && X < nnx && Y < nny) {
    const double fx = fe[ty][tx][4] + fe[ty][tx + 1][6] + fe[ty + 1][tx][2] + fe[ty + 1][tx + 1][0];
    const double fy = fe[ty][tx][5] + fe[ty][tx + 1][7] + fe[ty + 1][tx][3] + fe[ty + 1][tx + 1][1];
    const int64_t idx = 2 * (X + (int64_t)nnx * Y);
    const double px = su[ty + 1][tx + 1], py = sv[ty + 1][tx + 1];
    const double qx = fixed[idx] ? 0.0 : fx, qy = fixed[idx + 1] ? 0.0 : fy;
    p_new[off + idx] = px;
    p_new[off + idx + 1] = py;
    q[off + idx] = qx;
    q[off + idx + 1] = qy;
    v[0] = px * qx + py * qy;
  }
  double tot[1];
  const unsigned bid = blockIdx.x + gridDim.x * blockIdx.y, nblk = gridDim.x * gridDim.y;
  if (grid_sum_last_idx<1>(v, partial + rhs * pstride, counters + rhs, tot, red, bid, nblk) && tid == 0) {
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

template <class Tl>
static void fine_q4_cg_direction_launch(const Grid& g, const double* Ek, const uint8_t* fixed,
                                        const Q4Consts<double>& cst, const double* z, const double* p_old,
                                        double* p_new, double* q, int nr, int64_t stride, double* sc, double* partial,
                                        unsigned* counters, int64_t pstride, cudaStream_t s) {
  const dim3 grid((unsigned)((g.nn[0] + Tl::TX - 1) / Tl::TX), (unsigned)((g.nn[1] + Tl::TY - 1) / Tl::TY),
                  (unsigned)nr);
  launch_pdl(k_fine_q4_cg_direction<Tl>, grid, dim3(Tl::kThreads), 0, s, g, Ek, fixed, cst, z, p_old, p_new, q,
             stride, sc, partial, counters, pstride);
}

void launch_fine_q4_cg_direction(const Grid& g, const double* Ek, const uint8_t* fixed, const double* Ke0,
                                 const double* z, const double* p_old, double* p_new, double* q, int nr,
                                 int64_t stride, double* sc, double* partial, unsigned* counters, int64_t pstride,
                                 cudaStream_t s) {
  const Q4Consts<double> cst = q4_consts<double>(Ke0);
  switch (q4_tile_choice(g)) {
    case 0:
      fine_q4_cg_direction_launch<Q4TileA>(g, Ek, fixed, cst, z, p_old, p_new, q, nr, stride, sc, partial, counters,
                                           pstride, s);
      break;
    case 1:
      fine_q4_cg_direction_launch<Q4TileB>(g, Ek, fixed, cst, z, p_old, p_new, q, nr, stride, sc, partial, counters,
                                           pstride, s);
      break;
    default:
      fine_q4_cg_direction_launch<Q4TileC>(g, Ek, fixed, cst, z, p_old, p_new, q, nr, stride, sc, partial, counters,
                                           pstride, s);
      break;
  }
}

}  // namespace tobk
