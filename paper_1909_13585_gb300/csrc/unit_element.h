// Unit-element tables of the plain bilinear Q4 (plane stress, unit thickness) and trilinear H8
// elements on the unit square / cube (Sec. 2: K_e = E_kappa(x_e) K_e0): the unit-modulus
// constitutive matrix D, the shape-function gradients at the 2-point Gauss points per axis and
// K_e0 = sum_gp w |J| B^T D B (exact for these elements).
//
// Host code on caller-provided arrays only (no heap use), shared by the handle set-up and the
// allocation-free residual check, so that both evaluate the same K_e0.
//
// Local node l has corner bits x = ((l & 3) == 1 || (l & 3) == 2), y = ((l & 3) >= 2), z = l >> 2
// (the Q4 nodes counter-clockwise, then the same on the upper face).  Voigt order: 2D [xx yy xy],
// 3D [xx yy zz xy yz zx], engineering shear strains.
#pragma once
#include <cmath>

namespace tobk {
namespace unit_element {

constexpr int kMaxNodes = 8, kMaxDofs = 24, kMaxVoigt = 6;

inline int nodes(int dim) { return 1 << dim; }
inline int dofs(int dim) { return dim << dim; }
inline int voigt(int dim) { return dim == 2 ? 3 : 6; }

// natural coordinate (+-1) of local node l along axis a
inline double xi_node(int l, int a) {
  const int cx = ((l & 3) == 1 || (l & 3) == 2) ? 1 : 0;
  const int cy = ((l & 3) >= 2) ? 1 : 0;
  const int cz = l >> 2;
  const int c = a == 0 ? cx : (a == 1 ? cy : cz);
  return c ? 1.0 : -1.0;
}

// Gauss weight x |J|: weight 1 per point, |J| = (1/2)^dim on the unit element
inline double weight_det(int dim) { return std::pow(0.5, dim); }

// D [nv][nv] for unit Young's modulus and Poisson ratio nu
inline void constitutive(int dim, double nu, double* D) {
  const int nv = voigt(dim);
  for (int q = 0; q < nv * nv; ++q) D[q] = 0.0;
  if (dim == 2) {
    const double c = 1.0 / (1.0 - nu * nu);
    D[0] = c;
    D[1] = c * nu;
    D[3] = c * nu;
    D[4] = c;
    D[8] = c * (1.0 - nu) / 2.0;
  } else {
    const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    const double mu = 1.0 / (2.0 * (1.0 + nu));
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) D[a * 6 + b] = lam + (a == b ? 2.0 * mu : 0.0);
    for (int a = 3; a < 6; ++a) D[a * 6 + a] = mu;
  }
}

// dN [dim][nn]: physical gradients of the shape functions at Gauss point q (bit a of q set: the
// point's a-th natural coordinate is +1/sqrt(3), else -1/sqrt(3))
inline void shape_gradients(int dim, int q, double* dN) {
  const int nn = nodes(dim);
  const double g = 1.0 / std::sqrt(3.0);
  double gp[3];
  for (int a = 0; a < dim; ++a) gp[a] = ((q >> a) & 1) ? g : -g;
  for (int a = 0; a < dim; ++a)
    for (int l = 0; l < nn; ++l) {
      double v = xi_node(l, a) / std::pow(2.0, dim);
      for (int b = 0; b < dim; ++b)
        if (b != a) v *= 1.0 + xi_node(l, b) * gp[b];
      dN[a * nn + l] = 2.0 * v;  // d/dx = 2 d/dxi on the unit element
    }
}

// strain-displacement matrix B [nv][nd] from dN [dim][nn]
inline void strain_matrix(int dim, const double* dN, double* B) {
  const int nn = nodes(dim), nd = dofs(dim), nv = voigt(dim);
  for (int q = 0; q < nv * nd; ++q) B[q] = 0.0;
  for (int l = 0; l < nn; ++l) {
    const double dx = dN[0 * nn + l], dy = dN[1 * nn + l];
    if (dim == 2) {
      B[0 * nd + 2 * l] = dx;
      B[1 * nd + 2 * l + 1] = dy;
      B[2 * nd + 2 * l] = dy;
      B[2 * nd + 2 * l + 1] = dx;
    } else {
      const double dz = dN[2 * nn + l];
      B[0 * nd + 3 * l] = dx;
      B[1 * nd + 3 * l + 1] = dy;
      B[2 * nd + 3 * l + 2] = dz;
      B[3 * nd + 3 * l] = dy;
      B[3 * nd + 3 * l + 1] = dx;
      B[4 * nd + 3 * l + 1] = dz;
      B[4 * nd + 3 * l + 2] = dy;
      B[5 * nd + 3 * l] = dz;
      B[5 * nd + 3 * l + 2] = dx;
    }
  }
}

// K_e0 [nd][nd] = sum_gp w |J| B^T D B (unit modulus)
inline void stiffness(int dim, double nu, double* Ke) {
  const int nd = dofs(dim), nv = voigt(dim), ngp = nodes(dim);
  double D[kMaxVoigt * kMaxVoigt], dN[3 * kMaxNodes], B[kMaxVoigt * kMaxDofs];
  constitutive(dim, nu, D);
  const double wdet = weight_det(dim);
  for (int q = 0; q < nd * nd; ++q) Ke[q] = 0.0;
  for (int q = 0; q < ngp; ++q) {
    shape_gradients(dim, q, dN);
    strain_matrix(dim, dN, B);
    for (int r = 0; r < nd; ++r)
      for (int c = 0; c < nd; ++c) {
        double s = 0.0;
        for (int a = 0; a < nv; ++a)
          for (int b = 0; b < nv; ++b) s += B[a * nd + r] * D[a * nv + b] * B[b * nd + c];
        Ke[r * nd + c] += wdet * s;
      }
  }
}

// ---- incompatible-mode elements (Sec. 2: Wilson's quadrilateral, the hexahedron with 11
// interpolation functions per component) --------------------------------------------------------
// Each component is interpolated by the 2^d nodal functions plus d internal modes P_k = 1 - xi_k^2
// (natural coordinates xi in [-1, 1]^d), whose amplitudes alpha (d per component, ordered
// [mode][component] after the nodal DOFs) are condensed out element by element:
//   alpha = A u_e,  A = -K_aa^{-1} K_au,  K_c = K_uu + K_ua A.
// A does not depend on the modulus, so one table serves every element of a unit-square / unit-cube
// grid.

constexpr int kMaxInternal = 9;  // d * d internal DOFs
constexpr int kMaxFunctions = 11;  // 2^d + d interpolation functions per component

inline int functions(int dim) { return nodes(dim) + dim; }
inline int internal_dofs(int dim) { return dim * dim; }

// dF [dim][nf]: gradients of the 2^d nodal functions then of the d internal modes at Gauss point q
inline void full_gradients(int dim, int q, double* dF) {
  const int nn = nodes(dim), nf = functions(dim);
  double dN[3 * kMaxNodes];
  shape_gradients(dim, q, dN);
  const double g = 1.0 / std::sqrt(3.0);
  for (int a = 0; a < dim; ++a) {
    for (int l = 0; l < nn; ++l) dF[a * nf + l] = dN[a * nn + l];
    for (int k = 0; k < dim; ++k) {
      const double xk = ((q >> k) & 1) ? g : -g;
      dF[a * nf + nn + k] = a == k ? 2.0 * (-2.0 * xk) : 0.0;  // d/dx = 2 d/dxi
    }
  }
}

// Kc [nd][nd] (condensed unit-modulus stiffness) and A [dd][nd] (condensation map)
inline void incompatible_tables(int dim, double nu, double* Kc, double* A) {
  const int nd = dofs(dim), dd = internal_dofs(dim), nf = functions(dim), nt = nd + dd, nv = voigt(dim);
  constexpr int kT = kMaxDofs + kMaxInternal;
  double D[kMaxVoigt * kMaxVoigt], dF[3 * kMaxFunctions], B[kMaxVoigt * kT], K[kT * kT];
  constitutive(dim, nu, D);
  const double wdet = weight_det(dim);
  for (int q = 0; q < nt * nt; ++q) K[q] = 0.0;
  for (int q = 0; q < nodes(dim); ++q) {
    full_gradients(dim, q, dF);
    for (int r = 0; r < nv * nt; ++r) B[r] = 0.0;
    for (int f = 0; f < nf; ++f) {  // the strain matrix over all functions, DOF f * dim + c
      const double dx = dF[0 * nf + f], dy = dF[1 * nf + f];
      if (dim == 2) {
        B[0 * nt + 2 * f] = dx;
        B[1 * nt + 2 * f + 1] = dy;
        B[2 * nt + 2 * f] = dy;
        B[2 * nt + 2 * f + 1] = dx;
      } else {
        const double dz = dF[2 * nf + f];
        B[0 * nt + 3 * f] = dx;
        B[1 * nt + 3 * f + 1] = dy;
        B[2 * nt + 3 * f + 2] = dz;
        B[3 * nt + 3 * f] = dy;
        B[3 * nt + 3 * f + 1] = dx;
        B[4 * nt + 3 * f + 1] = dz;
        B[4 * nt + 3 * f + 2] = dy;
        B[5 * nt + 3 * f] = dz;
        B[5 * nt + 3 * f + 2] = dx;
      }
    }
    for (int r = 0; r < nt; ++r)
      for (int c = 0; c < nt; ++c) {
        double s = 0.0;
        for (int a = 0; a < nv; ++a)
          for (int b = 0; b < nv; ++b) s += B[a * nt + r] * D[a * nv + b] * B[b * nt + c];
        K[r * nt + c] += wdet * s;
      }
  }
  // A = -K_aa^{-1} K_au by Gauss-Jordan on [K_aa | -K_au] (K_aa is symmetric positive definite)
  double M[kMaxInternal * (kMaxInternal + kMaxDofs)];
  const int w = dd + nd;
  for (int i = 0; i < dd; ++i) {
    for (int j = 0; j < dd; ++j) M[i * w + j] = K[(nd + i) * nt + nd + j];
    for (int j = 0; j < nd; ++j) M[i * w + dd + j] = -K[(nd + i) * nt + j];
  }
  for (int p = 0; p < dd; ++p) {
    const double piv = M[p * w + p];
    for (int j = 0; j < w; ++j) M[p * w + j] /= piv;
    for (int i = 0; i < dd; ++i) {
      if (i == p) continue;
      const double f = M[i * w + p];
      for (int j = 0; j < w; ++j) M[i * w + j] -= f * M[p * w + j];
    }
  }
  for (int i = 0; i < dd; ++i)
    for (int j = 0; j < nd; ++j) A[i * nd + j] = M[i * w + dd + j];
  // K_c = K_uu + K_ua A, symmetrised
  for (int r = 0; r < nd; ++r)
    for (int c = 0; c < nd; ++c) {
      double s = K[r * nt + c];
      for (int i = 0; i < dd; ++i) s += K[r * nt + nd + i] * A[i * nd + c];
      Kc[r * nd + c] = s;
    }
  for (int r = 0; r < nd; ++r)
    for (int c = r + 1; c < nd; ++c) {
      const double v = 0.5 * (Kc[r * nd + c] + Kc[c * nd + r]);
      Kc[r * nd + c] = Kc[c * nd + r] = v;
    }
}

}  // namespace unit_element
}  // namespace tobk
