// Kaczmarz smoothing of prolongated buckling modes (Algorithm 2, the smoother S[.] on every grid
// Omega_j between the eigen level and the fine grid; Appendix A): for the shifted pencil
// A^j = K^j + sigma G^j (not positive definite, since sigma exceeds the level's lowest load factor)
// and each mode psi, the rows a_i of A^j are taken in turn and
//     psi <- psi - (a_i . psi / |a_i|^2) a_i,
// the orthogonal projection onto the hyperplane a_i . psi = 0 (Gauss-Seidel on A^T A).
//
// Row order.  The paper gives none.  Here the rows are grouped by a 3^d node colouring: node
// (i, j, k) has colour (i mod 3) + 3 (j mod 3) + 9 (k mod 3).  A row of node a touches only the
// 3^d nodes around a, so rows of two different nodes of one colour (three or more nodes apart along
// some axis) share no unknown: their projections commute exactly and run in parallel, one thread per
// node.  The d rows of one node share their support and run in turn (component 0, 1, ...).  A sweep
// is the colours in increasing order.  The oracle takes the rows in exactly this order.
//
// A^j is assembled once per level and shift into a 3^d-point nodal stencil of d x d blocks (the
// layout of stencil.cu) with rows and columns of fixed DOFs left out, together with the squared row
// norms |a_i|^2.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace tobk {

template <int DIM>
struct PencilDims {
  static constexpr int NB = DIM == 2 ? 9 : 27;
  static constexpr int NE = NB * DIM * DIM;
};

// S[((nbr * d + c) * d + c') * nnode + node] = A[d node + c][d nb + c'], nbr = (dx+1) + 3 (dy+1) [+ 9
// (dz+1)], for A = K + sigma G.  K: fine level from E_kappa [m] and the unit matrix Ke0 [nd*nd]
// (Ek != nullptr), else stored element matrices Ke [m][nd*nd].  G: fine level from the stored
// scalar matrices Gs [m][nn*nn] (the operator Gs (x) I_d; Gs != nullptr), else stored Ge [m][nd*nd],
// times Gscale[e] when Gscale != nullptr (the condensed stress stiffness of incompatible modes).
// rn2 [n] = squared norms of the rows (0 at fixed DOFs).
template <int DIM>
__global__ void k_pencil_stencil(Grid g, const uint8_t* __restrict__ fixed, const double* __restrict__ Ek,
                                 const double* __restrict__ Ke0, const double* __restrict__ Ke,
                                 const double* __restrict__ Gs, const double* __restrict__ Ge,
                                 const double* __restrict__ Gscale, double sigma, double* __restrict__ S,
                                 double* __restrict__ rn2) {
  constexpr int NN = Dims<DIM>::NN, ND = Dims<DIM>::ND, NE = PencilDims<DIM>::NE;
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
        const double sk = Ek ? Ek[e] : 1.0;
        const double sg = Gscale ? Gscale[e] : 1.0;
        for (int lb = 0; lb < NN; ++lb) {
          const int dx = corner_x(lb) - cx, dy = corner_y(lb) - cy, dz = corner_z(lb) - cz;
          const int nbr = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
          const int64_t nb = node + dx + (int64_t)g.nn[0] * (dy + (int64_t)g.nn[1] * dz);
          for (int c = 0; c < DIM; ++c)
            for (int cc = 0; cc < DIM; ++cc) {
              if (fixed[DIM * node + c] || fixed[DIM * nb + cc]) continue;
              const int r = ln * DIM + c, col = lb * DIM + cc;
              const double kv = Ek ? sk * Ke0[r * ND + col] : Ke[e * ND * ND + r * ND + col];
              const double gv = Gs ? (c == cc ? Gs[e * NN * NN + ln * NN + lb] : 0.0) : sg * Ge[e * ND * ND + r * ND + col];
              S[(int64_t)((nbr * DIM + c) * DIM + cc) * nn + node] += kv + sigma * gv;
            }
        }
      }
  for (int c = 0; c < DIM; ++c) {
    double s = 0.0;
    for (int nbr = 0; nbr < PencilDims<DIM>::NB; ++nbr)
      for (int cc = 0; cc < DIM; ++cc) {
        const double a = S[(int64_t)((nbr * DIM + c) * DIM + cc) * nn + node];
        s += a * a;
      }
    rn2[DIM * node + c] = fixed[DIM * node + c] ? 0.0 : s;
  }
}

// One colour of a sweep: every node of the colour (one thread each) projects its d rows in turn, for
// mode blockIdx.y (modes [q][stride]).
template <int DIM>
__global__ void __launch_bounds__(128) k_kaczmarz_colour(Grid g, const uint8_t* __restrict__ fixed,
                                                         const double* __restrict__ S, const double* __restrict__ rn2,
                                                         int ci, int cj, int ck, int ni, int nj, int nk,
                                                         double* __restrict__ Psi, int64_t stride) {
  constexpr int NB = PencilDims<DIM>::NB;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ni * nj * nk) return;
  const int i = ci + 3 * (int)(t % ni);
  const int j = cj + 3 * (int)((t / ni) % nj);
  const int k = ck + 3 * (int)(t / ((int64_t)ni * nj));
  const int64_t node = i + (int64_t)g.nn[0] * (j + (int64_t)g.nn[1] * k);
  const int64_t nn = g.nnode;
  double* psi = Psi + (int64_t)blockIdx.y * stride;
  for (int c = 0; c < DIM; ++c) {
    const int64_t row = DIM * node + c;
    const double r2 = rn2[row];
    if (fixed[row] || !(r2 > 0.0)) continue;
    double dot = 0.0;
    for (int nbr = 0; nbr < NB; ++nbr) {
      const int dx = nbr % 3 - 1, dy = (nbr / 3) % 3 - 1, dz = DIM == 3 ? nbr / 9 - 1 : 0;
      if (i + dx < 0 || i + dx >= g.nn[0] || j + dy < 0 || j + dy >= g.nn[1]) continue;
      if (DIM == 3 && (k + dz < 0 || k + dz >= g.nn[2])) continue;
      const int64_t nb = node + dx + (int64_t)g.nn[0] * (dy + (int64_t)g.nn[1] * dz);
      for (int cc = 0; cc < DIM; ++cc) dot += S[(int64_t)((nbr * DIM + c) * DIM + cc) * nn + node] * psi[DIM * nb + cc];
    }
    const double coef = dot / r2;
    for (int nbr = 0; nbr < NB; ++nbr) {
      const int dx = nbr % 3 - 1, dy = (nbr / 3) % 3 - 1, dz = DIM == 3 ? nbr / 9 - 1 : 0;
      if (i + dx < 0 || i + dx >= g.nn[0] || j + dy < 0 || j + dy >= g.nn[1]) continue;
      if (DIM == 3 && (k + dz < 0 || k + dz >= g.nn[2])) continue;
      const int64_t nb = node + dx + (int64_t)g.nn[0] * (dy + (int64_t)g.nn[1] * dz);
      for (int cc = 0; cc < DIM; ++cc)
        psi[DIM * nb + cc] -= coef * S[(int64_t)((nbr * DIM + c) * DIM + cc) * nn + node];
    }
  }
}

void launch_pencil_stencil(const Grid& g, const uint8_t* fixed, const double* Ek, const double* Ke0,
                           const double* Ke, const double* Gs, const double* Ge, const double* Gscale, double sigma,
                           double* S, double* rn2, cudaStream_t s) {
  const unsigned grid = (unsigned)((g.nnode + 127) / 128);
  note_launch();
  if (g.dim == 2)
    k_pencil_stencil<2><<<grid, 128, 0, s>>>(g, fixed, Ek, Ke0, Ke, Gs, Ge, Gscale, sigma, S, rn2);
  else
    k_pencil_stencil<3><<<grid, 128, 0, s>>>(g, fixed, Ek, Ke0, Ke, Gs, Ge, Gscale, sigma, S, rn2);
}

void launch_kaczmarz_sweeps(const Grid& g, const uint8_t* fixed, const double* S, const double* rn2, double* Psi,
                            int q, int64_t stride, int sweeps, cudaStream_t s) {
  const int nz = g.dim == 3 ? 3 : 1;
  for (int sw = 0; sw < sweeps; ++sw)
    for (int ck = 0; ck < nz; ++ck)
      for (int cj = 0; cj < 3; ++cj)
        for (int ci = 0; ci < 3; ++ci) {
          const int ni = (g.nn[0] - ci + 2) / 3, nj = (g.nn[1] - cj + 2) / 3;
          const int nk = g.dim == 3 ? (g.nn[2] - ck + 2) / 3 : 1;
          const int64_t cnt = (int64_t)ni * nj * nk;
          if (cnt <= 0) continue;
          const dim3 grid((unsigned)((cnt + 127) / 128), (unsigned)q);
          note_launch();
          if (g.dim == 2)
            k_kaczmarz_colour<2><<<grid, 128, 0, s>>>(g, fixed, S, rn2, ci, cj, ck, ni, nj, nk, Psi, stride);
          else
            k_kaczmarz_colour<3><<<grid, 128, 0, s>>>(g, fixed, S, rn2, ci, cj, ck, ni, nj, nk, Psi, stride);
        }
}

}  // namespace tobk
