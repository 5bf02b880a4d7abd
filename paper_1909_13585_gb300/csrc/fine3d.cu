// Fine-level (matrix-free) K(x) v = sum_e E_kappa(x_e) K_e0 v_e of Sec. 2 (applied inside the mgPCG of
// Algorithm 1 step 3 and Appendix A) for H8 elements: the operator in factored form
// (h8_element.cuh), element by element.
//
// A block owns a (EX - 1) x 7 column of nodes in the (x, y) plane and a range of zc node planes, and
// marches up in z one element layer at a time: it keeps two node planes of the input (with a
// one-node halo) in shared memory, computes the forces of the EX x 8 elements of the layer (one
// element per thread), stores them structure-of-arrays in shared memory, and each node thread adds
// the four contributions from below (finishing its node plane, which is then written out with the
// smoother / residual / CG update) and keeps the four from above for the next plane.  The factored
// element needs about 200 FP64 operations instead of the 576 multiply-adds of the dense 24 x 24
// product, which on GB300 (2 FP64 instructions per clock per SM) sets the speed of the FP64 path.
// The tile width EX (32, 36 or 44) is chosen per grid to minimise the element slots of the launch:
// a tile column the grid only partly covers holds its SM slot for the whole march with most of its
// threads idle (97 nodes across: 31-node tiles leave 4 of the last tile's 31 columns in use, 35-node
// tiles cover them with 3 tiles; 129 nodes: 43-node tiles exactly).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "h8_element.cuh"
#include "kernels.h"

namespace tobk {

namespace {
constexpr int EY = 8;                     // element tile rows per layer (one element per thread)
constexpr int TY = EY - 1;                // node tile rows
constexpr int PY = EY + 1;                // node-plane tile rows with halo
constexpr int APPLY_CGDIR = 3;

template <typename T, int EX>
struct H8Smem {
  static constexpr int PX = EX + 1;  // node-plane tile columns with halo
  T pv[2][3][PY][PX];     // ring of two node planes (components separate)
  T fe[24][EY][EX];       // element forces of the current layer, [c*8 + cz*4 + cy*2 + cx]
  double red[64];
};

template <typename T>
struct H8Args {
  const T* v;          // input vector (KV/RES/JAC) or z (CGDIR)
  const T* b;          // right-hand side (RES/JAC) or p_old (CGDIR)
  const T* dinv;
  T* y;                // output (KV/RES/JAC) or p_new (CGDIR)
  T* q;                // CGDIR: K p
  SmoothArgs<T> sm;
  double* sc;          // CGDIR: per-RHS scalars
  double* partial;
  unsigned* counters;
  int64_t pstride;
  const double* act;   // active-RHS flags of the V-cycle (or null)
};
}  // namespace

template <typename T, int MODE, int EX>
__global__ void __launch_bounds__(EX * EY) k_fine_h8(Grid g, const T* __restrict__ Ek,
                                                     const uint8_t* __restrict__ fixed, H8Consts<T> cst, H8Args<T> a,
                                                     int zc, int nzc, int64_t stride) {
  constexpr int TX = EX - 1, PX = EX + 1, kThreads3 = EX * EY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  H8Smem<T, EX>& S = *reinterpret_cast<H8Smem<T, EX>*>(smem_raw);
  const int rhs = blockIdx.z / nzc, chunk = blockIdx.z % nzc;
  double beta = 0.0;
  if (MODE == APPLY_CGDIR) {
    if (a.sc[(size_t)rhs * kScStride + SC_ACTIVE] == 0.0) return;
    beta = a.sc[(size_t)rhs * kScStride + SC_BETA];
  } else if (a.act != nullptr && a.act[(size_t)rhs * kScStride + SC_ACTIVE] == 0.0) {
    return;
  }
  const int t = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = chunk * zc, z1 = min(z0 + zc, g.nn[2]);
  const int nnx = g.nn[0], nny = g.nn[1], nnz = g.nn[2];
  const int64_t off = (int64_t)rhs * stride;
  // node plane p (global z) into ring slot p & 1, with halo; zero outside the grid
  auto load_plane = [&](int p) {
    T(*dst)[PY][PX] = S.pv[p & 1];
    for (int q = t; q < PX * PY; q += kThreads3) {
      const int px = q % PX, py = q / PX;
      const int gx = x0 - 1 + px, gy = y0 - 1 + py;
      T c0 = T(0), c1 = T(0), c2 = T(0);
      if (p >= 0 && p < nnz && gx >= 0 && gx < nnx && gy >= 0 && gy < nny) {
        const int64_t i0 = 3 * (gx + (int64_t)nnx * (gy + (int64_t)nny * p));
        if (MODE == APPLY_CGDIR) {
          c0 = fixed[i0] ? T(0) : (T)(a.v[off + i0] + beta * a.b[off + i0]);
          c1 = fixed[i0 + 1] ? T(0) : (T)(a.v[off + i0 + 1] + beta * a.b[off + i0 + 1]);
          c2 = fixed[i0 + 2] ? T(0) : (T)(a.v[off + i0 + 2] + beta * a.b[off + i0 + 2]);
        } else {
          c0 = a.v[off + i0];
          c1 = a.v[off + i0 + 1];
          c2 = a.v[off + i0 + 2];
        }
      }
      dst[0][py][px] = c0;
      dst[1][py][px] = c1;
      dst[2][py][px] = c2;
    }
  };
  const int ex = t % EX, ey = t / EX;  // element of the layer owned by this thread
  const bool node_thread = t < TX * TY;
  const int tx = t % TX, ty = t / TX;  // node of the column owned by this thread
  const int gx = x0 + tx, gy = y0 + ty;
  T acc[3] = {T(0), T(0), T(0)};
  double dot = 0.0;
  load_plane(z0 - 1);
  for (int l = z0 - 1; l < z1; ++l) {
    load_plane(l + 1);
    __syncthreads();
    // forces of element (x0 - 1 + ex, y0 - 1 + ey, l)
    {
      const int gex = x0 - 1 + ex, gey = y0 - 1 + ey;
      T f[3][2][2][2];
      if (l >= 0 && l < g.nel[2] && gex >= 0 && gex < g.nel[0] && gey >= 0 && gey < g.nel[1]) {
        T v[3][2][2][2];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int cz = 0; cz < 2; ++cz)
#pragma unroll
            for (int cy = 0; cy < 2; ++cy)
#pragma unroll
              for (int cx = 0; cx < 2; ++cx) v[c][cz][cy][cx] = S.pv[(l + cz) & 1][c][ey + cy][ex + cx];
        const T E = Ek[gex + (int64_t)g.nel[0] * (gey + (int64_t)g.nel[1] * l)];
        h8_forces<T>(v, E, cst, f);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int k = 0; k < 8; ++k) (&f[c][0][0][0])[k] = T(0);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int k = 0; k < 8; ++k) S.fe[c * 8 + k][ey][ex] = (&f[c][0][0][0])[k];
    }
    __syncthreads();
    if (node_thread) {
      T below[3], above[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        // element (ex', ey') = (tx + 1 - cx, ty + 1 - cy) touches this node at its corner (cx, cy)
        below[c] = S.fe[c * 8 + 0][ty + 1][tx + 1] + S.fe[c * 8 + 1][ty + 1][tx] + S.fe[c * 8 + 2][ty][tx + 1] +
                   S.fe[c * 8 + 3][ty][tx];
        above[c] = S.fe[c * 8 + 4][ty + 1][tx + 1] + S.fe[c * 8 + 5][ty + 1][tx] + S.fe[c * 8 + 6][ty][tx + 1] +
                   S.fe[c * 8 + 7][ty][tx];
        acc[c] += below[c];
      }
      if (l >= z0 && gx < nnx && gy < nny) {
        const int64_t node = gx + (int64_t)nnx * (gy + (int64_t)nny * l);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int64_t idx = 3 * node + c;
          const T vloc = S.pv[l & 1][c][ty + 1][tx + 1];
          if (MODE == APPLY_CGDIR) {
            const T qv = fixed[idx] ? T(0) : acc[c];
            a.y[off + idx] = vloc;
            a.q[off + idx] = qv;
            dot += (double)vloc * (double)qv;
          } else if (fixed[idx]) {
            a.y[off + idx] = T(0);
          } else if (MODE == APPLY_KV) {
            a.y[off + idx] = acc[c];
          } else if (MODE == APPLY_RES) {
            a.y[off + idx] = a.b[off + idx] - acc[c];
          } else {
            const T r = a.dinv[idx] * (a.b[off + idx] - acc[c]);
            const T dn = (a.sm.d_in ? a.sm.coef[0] * a.sm.d_in[off + idx] : T(0)) + a.sm.coef[1] * r;
            if (a.sm.d_out) a.sm.d_out[off + idx] = dn;
            a.y[off + idx] = vloc + dn;
          }
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] = above[c];
    }
    __syncthreads();
  }
  if (MODE == APPLY_CGDIR) {
    double v[1] = {dot};
    double tot[1];
    const unsigned bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * chunk);
    const unsigned nblk = gridDim.x * gridDim.y * nzc;
    if (grid_sum_last_idx<1>(v, a.partial + rhs * a.pstride, a.counters + rhs, tot, S.red, bid, nblk) && t == 0) {
      double* s = a.sc + (size_t)rhs * kScStride;
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
}

namespace {

// tile width of the grid: the fewest element slots (tiles x EX x EY per layer; ties: the earlier)
constexpr int kH8Widths[3] = {32, 36, 44};
int64_t h8_cols(const Grid& g, int ex) {
  return (int64_t)((g.nn[0] + ex - 2) / (ex - 1)) * ((g.nn[1] + TY - 1) / TY);
}
int h8_width(const Grid& g) {
  int best = kH8Widths[0];
  for (int w : kH8Widths)
    if (h8_cols(g, w) * w < h8_cols(g, best) * best) best = w;
  return best;
}

// node planes per block: as many as keep at least two blocks per SM busy for one RHS
int h8_zc(const Grid& g, int nr, int ex) {
  const int64_t cols = h8_cols(g, ex);
  int zc = 16;
  while (zc > 4 && cols * ((g.nn[2] + zc - 1) / zc) * nr < 2 * 152) zc /= 2;
  return zc;
}

template <typename T, int MODE, int EX>
void h8_launch_w(const Grid& g, const T* Ek, const uint8_t* fixed, double nu, int element, const H8Args<T>& a, int nr,
                 int64_t stride, cudaStream_t s) {
  static bool configured = false;
  const size_t smem = sizeof(H8Smem<T, EX>);
  if (!configured) {
    cudaFuncSetAttribute(k_fine_h8<T, MODE, EX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  const int zc = h8_zc(g, nr, EX), nzc = (g.nn[2] + zc - 1) / zc;
  dim3 grid((unsigned)((g.nn[0] + EX - 2) / (EX - 1)), (unsigned)((g.nn[1] + TY - 1) / TY), (unsigned)(nzc * nr));
  note_launch();
  k_fine_h8<T, MODE, EX><<<grid, EX * EY, smem, s>>>(g, Ek, fixed, h8_consts<T>(nu, element), a, zc, nzc, stride);
}

template <typename T, int MODE>
void h8_launch(const Grid& g, const T* Ek, const uint8_t* fixed, double nu, int element, const H8Args<T>& a, int nr,
               int64_t stride, cudaStream_t s) {
  switch (h8_width(g)) {
    case 32: h8_launch_w<T, MODE, 32>(g, Ek, fixed, nu, element, a, nr, stride, s); break;
    case 36: h8_launch_w<T, MODE, 36>(g, Ek, fixed, nu, element, a, nr, stride, s); break;
    default: h8_launch_w<T, MODE, 44>(g, Ek, fixed, nu, element, a, nr, stride, s); break;
  }
}

}  // namespace

int64_t fine_h8_blocks(const Grid& g) {
  // the CG-direction launch reduces over this many blocks per RHS (at most: one RHS, the smallest
  // z range, the widest column count of the candidate tiles)
  const int zc = 4;
  int64_t cols = 0;
  for (int w : kH8Widths) cols = std::max(cols, h8_cols(g, w));
  return cols * ((g.nn[2] + zc - 1) / zc);
}

template <typename T>
void launch_fine_h8(const Grid& g, const T* Ek, const uint8_t* fixed, double nu, int element, int mode, const T* v, const T* b,
                    const T* dinv, T* y, SmoothArgs<T> sm, int nr, int64_t stride, cudaStream_t s) {
  H8Args<T> a{};
  a.v = v;
  a.b = b;
  a.dinv = dinv;
  a.y = y;
  a.sm = sm;
  a.act = active_rhs();
  if (mode == APPLY_KV)
    h8_launch<T, APPLY_KV>(g, Ek, fixed, nu, element, a, nr, stride, s);
  else if (mode == APPLY_RES)
    h8_launch<T, APPLY_RES>(g, Ek, fixed, nu, element, a, nr, stride, s);
  else
    h8_launch<T, APPLY_JAC>(g, Ek, fixed, nu, element, a, nr, stride, s);
}

template void launch_fine_h8<double>(const Grid&, const double*, const uint8_t*, double, int, int, const double*,
                                     const double*, const double*, double*, SmoothArgs<double>, int, int64_t,
                                     cudaStream_t);
template void launch_fine_h8<float>(const Grid&, const float*, const uint8_t*, double, int, int, const float*, const float*,
                                    const float*, float*, SmoothArgs<float>, int, int64_t, cudaStream_t);

void launch_fine_h8_cg_direction(const Grid& g, const double* Ek, const uint8_t* fixed, double nu, int element, const double* z,
                                 const double* p_old, double* p_new, double* q, int nr, int64_t stride, double* sc,
                                 double* partial, unsigned* counters, int64_t pstride, cudaStream_t s) {
  H8Args<double> a{};
  a.v = z;
  a.b = p_old;
  a.y = p_new;
  a.q = q;
  a.sc = sc;
  a.partial = partial;
  a.counters = counters;
  a.pstride = pstride;
  h8_launch<double, APPLY_CGDIR>(g, Ek, fixed, nu, element, a, nr, stride, s);
}

}  // namespace tobk
