// Fine-grid kernels of the incompatible-mode elements (Sec. 2: Wilson's quadrilateral in 2D, the
// hexahedron with 11 interpolation functions per component in 3D) that differ from the plain Q4 / H8
// path: the stress stiffness and the adjoint right-hand side.
//
// Every displacement component is interpolated by the 2^d nodal functions and the d internal modes
// P_k = 1 - xi_k^2; the internal amplitudes are condensed out, alpha = A u_e with the constant map
// A = -K_aa^{-1} K_au (unit_element.h), so an element acts on its nodal DOFs through
// T = [I ; A].  Reading of the paper (which does not say how the stress stiffness treats the internal
// modes): the same condensation, with Gauss-point stresses from the enhanced strain of u_e,
//     G_c0[u_e] = T^T (G_full (x) I_d) T,  G_full(f, f') = sum_gp w |J| grad F_f . S(sigma_gp) grad F_f',
// over the 2^d + d functions F (unit modulus; the operator is E_sigma(x_e) G_c0).  The adjoint element
// vector d(phi_e^T G_c0[u_e] phi_e)/du_e = sum_gp w |J| (B~ T)^T D h(T phi_e), h the Voigt form (doubled
// shear) of H_ab = sum_c d_a phi~_c d_b phi~_c.
//
// Gradients of the functions at the Gauss points: nodal ones from the handle's table dN
// [ngp][d][nn]; internal ones d P_k / d x_a = delta_ak 2 (-2 xi_k) (d/dx = 2 d/dxi on a unit element).
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace tobk {

template <int DIM>
struct IncDims {
  static constexpr int NN = Dims<DIM>::NN, ND = Dims<DIM>::ND, NV = Dims<DIM>::NV;
  static constexpr int NF = NN + DIM;       // interpolation functions per component
  static constexpr int NI = DIM * DIM;      // internal DOFs
};

// gradient of function f along axis a at Gauss point gp
template <int DIM>
__device__ __forceinline__ double inc_grad(const double* __restrict__ dN, int gp, int a, int f) {
  constexpr int NN = Dims<DIM>::NN;
  if (f < NN) return dN[(gp * DIM + a) * NN + f];
  const int k = f - NN;
  if (k != a) return 0.0;
  const double xk = ((gp >> k) & 1) ? 0.57735026918962576451 : -0.57735026918962576451;
  return -4.0 * xk;
}

template <int DIM>
__device__ __forceinline__ void element_dofs(const Grid& g, int64_t e, int64_t (&dof)[Dims<DIM>::ND]) {
  constexpr int NN = Dims<DIM>::NN;
  const int ei = (int)(e % g.nel[0]);
  const int64_t rest = e / g.nel[0];
  const int ej = (int)(rest % g.nel[1]);
  const int ek = (int)(rest / g.nel[1]);
  const int64_t n0 = ei + (int64_t)g.nn[0] * (ej + (int64_t)g.nn[1] * ek);
#pragma unroll
  for (int l = 0; l < NN; ++l) {
    const int64_t nb = n0 + corner_x(l) + (int64_t)g.nn[0] * (corner_y(l) + (int64_t)g.nn[1] * corner_z(l));
#pragma unroll
    for (int c = 0; c < DIM; ++c) dof[l * DIM + c] = DIM * nb + c;
  }
}

// Voigt strain (engineering shear) from a displacement gradient grad[a][c] = d u_c / d x_a
template <int DIM>
__device__ __forceinline__ void voigt_strain(const double (&grad)[DIM][DIM], double (&eps)[Dims<DIM>::NV]) {
  if constexpr (DIM == 2) {
    eps[0] = grad[0][0];
    eps[1] = grad[1][1];
    eps[2] = grad[0][1] + grad[1][0];
  } else {
    eps[0] = grad[0][0];
    eps[1] = grad[1][1];
    eps[2] = grad[DIM - 1][DIM - 1];
    eps[3] = grad[0][1] + grad[1][0];
    eps[4] = grad[1][DIM - 1] + grad[DIM - 1][1];
    eps[5] = grad[DIM - 1][0] + grad[0][DIM - 1];
  }
}

// Per element: the enhanced Gauss-point stresses of u_e (unit modulus) and
// G_full [m][NF][NF] = sum_gp w |J| dF^T S dF.
template <int DIM>
__global__ void __launch_bounds__(128) k_inc_gfull(Grid g, const double* __restrict__ u, const double* __restrict__ A,
                                                   const double* __restrict__ dN, const double* __restrict__ D,
                                                   double wdet, double* __restrict__ Gfull) {
  using I = IncDims<DIM>;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.m) return;
  int64_t dof[I::ND];
  element_dofs<DIM>(g, e, dof);
  double w[I::NF][DIM];  // nodal displacements, then the condensed internal amplitudes
#pragma unroll
  for (int l = 0; l < I::NN; ++l)
#pragma unroll
    for (int c = 0; c < DIM; ++c) w[l][c] = u[dof[l * DIM + c]];
  for (int i = 0; i < I::NI; ++i) {
    double s = 0.0;
    for (int j = 0; j < I::ND; ++j) s += A[i * I::ND + j] * w[j / DIM][j % DIM];
    w[I::NN + i / DIM][i % DIM] = s;
  }
  double S[I::NN][DIM][DIM];  // Gauss-point stress tensors
  for (int gp = 0; gp < I::NN; ++gp) {
    double grad[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double s = 0.0;
        for (int f = 0; f < I::NF; ++f) s += inc_grad<DIM>(dN, gp, a, f) * w[f][c];
        grad[a][c] = s;
      }
    double eps[I::NV], sig[I::NV];
    voigt_strain<DIM>(grad, eps);
#pragma unroll
    for (int p = 0; p < I::NV; ++p) {
      double s = 0.0;
#pragma unroll
      for (int q = 0; q < I::NV; ++q) s += D[p * I::NV + q] * eps[q];
      sig[p] = s;
    }
    if constexpr (DIM == 2) {
      S[gp][0][0] = sig[0];
      S[gp][DIM - 1][DIM - 1] = sig[1];
      S[gp][0][DIM - 1] = S[gp][DIM - 1][0] = sig[2];
    } else {
      S[gp][0][0] = sig[0];
      S[gp][1][1] = sig[1];
      S[gp][DIM - 1][DIM - 1] = sig[2];
      S[gp][0][1] = S[gp][1][0] = sig[3];
      S[gp][1][DIM - 1] = S[gp][DIM - 1][1] = sig[4];
      S[gp][DIM - 1][0] = S[gp][0][DIM - 1] = sig[I::NV - 1];
    }
  }
  double* out = Gfull + e * I::NF * I::NF;
  for (int f1 = 0; f1 < I::NF; ++f1)
    for (int f2 = f1; f2 < I::NF; ++f2) {
      double acc = 0.0;
      for (int gp = 0; gp < I::NN; ++gp) {
        double g1[DIM], g2[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          g1[a] = inc_grad<DIM>(dN, gp, a, f1);
          g2[a] = inc_grad<DIM>(dN, gp, a, f2);
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a)
#pragma unroll
          for (int b = 0; b < DIM; ++b) acc += g1[a] * S[gp][a][b] * g2[b];
      }
      out[f1 * I::NF + f2] = wdet * acc;
      out[f2 * I::NF + f1] = wdet * acc;
    }
}

// Row r of the condensed element matrix G_c0 = T^T (G_full (x) I) T, one thread per (element, row).
template <int DIM>
__global__ void __launch_bounds__(128) k_inc_gc0(Grid g, const double* __restrict__ Gfull,
                                                 const double* __restrict__ A, double* __restrict__ Gc0) {
  using I = IncDims<DIM>;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= g.m * I::ND) return;
  const int64_t e = t / I::ND;
  const int r = (int)(t % I::ND);
  const int ra = r / DIM, rc = r % DIM;
  const double* Gf = Gfull + e * I::NF * I::NF;
  // v[f][c] = sum_f1 T[(f1, c)][r] G_full[f1][f]
  double v[I::NF][DIM];
  for (int f = 0; f < I::NF; ++f)
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      double s = (c == rc) ? Gf[ra * I::NF + f] : 0.0;
      for (int k = 0; k < DIM; ++k) s += A[(k * DIM + c) * I::ND + r] * Gf[(I::NN + k) * I::NF + f];
      v[f][c] = s;
    }
  double* out = Gc0 + e * I::ND * I::ND + (int64_t)r * I::ND;
  for (int col = 0; col < I::ND; ++col) {
    double s = v[col / DIM][col % DIM];
    for (int i = 0; i < I::NI; ++i) s += v[I::NN + i / DIM][i % DIM] * A[i * I::ND + col];
    out[col] = s;
  }
}

// y = sum_e E_sigma(x_e) A_e^T G_c0[e] A_e v (rows of fixed DOFs 0)
template <int DIM>
struct ScaledStoredOp {
  Grid g;
  const double* Gc0;
  const double* scale_e;
  __device__ __forceinline__ double scale(int64_t e) const { return scale_e[e]; }
  __device__ __forceinline__ double entry(int64_t e, int r, int c) const {
    return __ldg(Gc0 + e * (Dims<DIM>::ND * Dims<DIM>::ND) + r * Dims<DIM>::ND + c);
  }
};

template <int DIM>
__global__ void __launch_bounds__(256) k_inc_apply_g(ScaledStoredOp<DIM> op, const uint8_t* __restrict__ fixed,
                                                     const double* __restrict__ v, double* __restrict__ y,
                                                     int64_t stride) {
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(op.g, node, i, j, k)) return;
  const int64_t off = (int64_t)blockIdx.y * stride;
  double acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = 0.0;
  gather_rows<DIM, double>(op, i, j, k, LoadVec<double>{v + off}, acc);
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t idx = DIM * node + c;
    y[off + idx] = fixed[idx] ? 0.0 : acc[c];
  }
}

// Adjoint element vectors out [m][ND] = E_sigma sum_gp w |J| (B~ T)^T D h(T phi_e)
template <int DIM>
__global__ void __launch_bounds__(128) k_inc_adjoint(Grid g, const double* __restrict__ phi,
                                                     const double* __restrict__ Es, const double* __restrict__ A,
                                                     const double* __restrict__ dN, const double* __restrict__ D,
                                                     double wdet, double* __restrict__ out) {
  using I = IncDims<DIM>;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= g.m) return;
  int64_t dof[I::ND];
  element_dofs<DIM>(g, e, dof);
  double w[I::NF][DIM];
#pragma unroll
  for (int l = 0; l < I::NN; ++l)
#pragma unroll
    for (int c = 0; c < DIM; ++c) w[l][c] = phi[dof[l * DIM + c]];
  for (int i = 0; i < I::NI; ++i) {
    double s = 0.0;
    for (int j = 0; j < I::ND; ++j) s += A[i * I::ND + j] * w[j / DIM][j % DIM];
    w[I::NN + i / DIM][i % DIM] = s;
  }
  double vf[I::NF][DIM];  // (B~)^T s accumulated over the Gauss points, per function and component
  for (int f = 0; f < I::NF; ++f)
#pragma unroll
    for (int c = 0; c < DIM; ++c) vf[f][c] = 0.0;
  const double es = Es[e] * wdet;
  for (int gp = 0; gp < I::NN; ++gp) {
    double grad[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        double s = 0.0;
        for (int f = 0; f < I::NF; ++f) s += inc_grad<DIM>(dN, gp, a, f) * w[f][c];
        grad[a][c] = s;
      }
    double Hm[DIM][DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
      for (int b = 0; b < DIM; ++b) {
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) s += grad[a][c] * grad[b][c];
        Hm[a][b] = s;
      }
    double hv[I::NV];
    if constexpr (DIM == 2) {
      hv[0] = Hm[0][0];
      hv[1] = Hm[DIM - 1][DIM - 1];
      hv[2] = 2.0 * Hm[0][DIM - 1];
    } else {
      hv[0] = Hm[0][0];
      hv[1] = Hm[1][1];
      hv[2] = Hm[DIM - 1][DIM - 1];
      hv[3] = 2.0 * Hm[0][1];
      hv[4] = 2.0 * Hm[1][DIM - 1];
      hv[I::NV - 1] = 2.0 * Hm[DIM - 1][0];
    }
    double s[I::NV];
#pragma unroll
    for (int p = 0; p < I::NV; ++p) {
      double a = 0.0;
#pragma unroll
      for (int q = 0; q < I::NV; ++q) a += D[p * I::NV + q] * hv[q];
      s[p] = es * a;
    }
    for (int f = 0; f < I::NF; ++f) {
      const double dx = inc_grad<DIM>(dN, gp, 0, f), dy = inc_grad<DIM>(dN, gp, 1, f);
      if constexpr (DIM == 2) {
        vf[f][0] += dx * s[0] + dy * s[2];
        vf[f][DIM - 1] += dy * s[1] + dx * s[2];
      } else {
        const double dz = inc_grad<DIM>(dN, gp, DIM - 1, f);
        vf[f][0] += dx * s[0] + dy * s[3] + dz * s[I::NV - 1];
        vf[f][1] += dy * s[1] + dx * s[3] + dz * s[4];
        vf[f][DIM - 1] += dz * s[2] + dy * s[4] + dx * s[I::NV - 1];
      }
    }
  }
  double* o = out + e * I::ND;
  for (int j = 0; j < I::ND; ++j) {
    double s = vf[j / DIM][j % DIM];
    for (int i = 0; i < I::NI; ++i) s += A[i * I::ND + j] * vf[I::NN + i / DIM][i % DIM];
    o[j] = s;
  }
}

// b[a, c] = sum over the elements around node a of their element vectors at the node (masked)
template <int DIM>
__global__ void k_gather_element_vectors(Grid g, const uint8_t* __restrict__ fixed, const double* __restrict__ ev,
                                         double* __restrict__ b) {
  constexpr int ND = Dims<DIM>::ND;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int i, j, k;
  if (!node_coords(g, node, i, j, k)) return;
  double acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c] = 0.0;
  for (int cz = 0; cz < (DIM == 3 ? 2 : 1); ++cz)
    for (int cy = 0; cy < 2; ++cy)
      for (int cx = 0; cx < 2; ++cx) {
        const int ei = i - cx, ej = j - cy, ek = k - cz;
        if (ei < 0 || ei >= g.nel[0] || ej < 0 || ej >= g.nel[1]) continue;
        if (DIM == 3 && (ek < 0 || ek >= g.nel[2])) continue;
        const int64_t e = ei + (int64_t)g.nel[0] * (ej + (int64_t)g.nel[1] * ek);
        const int ln = local_node(cx, cy, cz);
#pragma unroll
        for (int c = 0; c < DIM; ++c) acc[c] += ev[e * ND + ln * DIM + c];
      }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t idx = DIM * node + c;
    b[idx] = fixed[idx] ? 0.0 : acc[c];
  }
}

void launch_inc_stress(const Grid& g, const double* u, const double* A, const double* dN, const double* D,
                       double wdet, double* Gfull, double* Gc0, cudaStream_t s) {
  const unsigned b1 = (unsigned)((g.m + 127) / 128);
  const unsigned b2 = (unsigned)((g.m * (g.dim << g.dim) + 127) / 128);
  note_launch();
  if (g.dim == 2)
    k_inc_gfull<2><<<b1, 128, 0, s>>>(g, u, A, dN, D, wdet, Gfull);
  else
    k_inc_gfull<3><<<b1, 128, 0, s>>>(g, u, A, dN, D, wdet, Gfull);
  note_launch();
  if (g.dim == 2)
    k_inc_gc0<2><<<b2, 128, 0, s>>>(g, Gfull, A, Gc0);
  else
    k_inc_gc0<3><<<b2, 128, 0, s>>>(g, Gfull, A, Gc0);
}

void launch_inc_apply_g(const Grid& g, const uint8_t* fixed, const double* Gc0, const double* Es, const double* v,
                        double* y, int nr, int64_t stride, cudaStream_t s) {
  const dim3 grid((unsigned)((g.nnode + 255) / 256), (unsigned)nr);
  note_launch();
  if (g.dim == 2)
    k_inc_apply_g<2><<<grid, 256, 0, s>>>(ScaledStoredOp<2>{g, Gc0, Es}, fixed, v, y, stride);
  else
    k_inc_apply_g<3><<<grid, 256, 0, s>>>(ScaledStoredOp<3>{g, Gc0, Es}, fixed, v, y, stride);
}

void launch_inc_adjoint(const Grid& g, const uint8_t* fixed, const double* phi, const double* Es, const double* A,
                        const double* dN, const double* D, double wdet, double* ev, double* b, cudaStream_t s) {
  const unsigned b1 = (unsigned)((g.m + 127) / 128);
  const unsigned b2 = (unsigned)((g.nnode + 255) / 256);
  note_launch();
  if (g.dim == 2)
    k_inc_adjoint<2><<<b1, 128, 0, s>>>(g, phi, Es, A, dN, D, wdet, ev);
  else
    k_inc_adjoint<3><<<b1, 128, 0, s>>>(g, phi, Es, A, dN, D, wdet, ev);
  note_launch();
  if (g.dim == 2)
    k_gather_element_vectors<2><<<b2, 256, 0, s>>>(g, fixed, ev, b);
  else
    k_gather_element_vectors<3><<<b2, 256, 0, s>>>(g, fixed, ev, b);
}

}  // namespace tobk
