// The unit-modulus element stiffness K_e0 of Sec. 2 for the unit-square Q4 element, in factored
// form.
//
// Factored unit-square Q4 element operator (plane stress, 2 x 2 Gauss), shared by the fine-level
// kernels of one design (fine2d.cu) and of a batch of designs (batch.cu).
//
// For the unit square element with 2x2 Gauss integration, the bilinear displacement gradient is
// fully described by six numbers per element: the mean gradients A_u = du/dx, B_u = du/dy,
// A_v = dv/dx, B_v = dv/dy and the two hourglass amplitudes h_u, h_v (u0 - u1 + u2 - u3).  The element
// strain energy is exactly
//   E/2 [D11 (A_u^2 + h_u^2/12) + 2 D12 A_u B_v + D22 (B_v^2 + h_v^2/12) + D33 ((B_u + A_v)^2 + (h_u^2 + h_v^2)/12)],
// so K_e v_e costs about 41 arithmetic operations instead of the 64 multiply-adds (plus scaling)
// of the dense 8 x 8 product.
#pragma once
#include <cuda_runtime.h>

namespace tobk {

template <typename T>
struct Q4Consts {
  T d11, d12, d22, d33;  // plane-stress unit-modulus constitutive entries
  T hu, hv;              // (D11 + D33)/12, (D22 + D33)/12
};

// Recovers the constants from the unit element matrix K_e0 (row-major 8 x 8).  The hourglass
// coefficients from the hourglass vectors g = (+1, -1, +1, -1) on the x (resp. y) DOFs:
// g^T K g = 16 hu.  The mean-gradient part from entries with the hourglass part removed:
// K[0][0] - hu = (D11 + D33)/4, K[0][2] + hu = (D33 - D11)/4, K[0][1] = (D12 + D33)/4.  For the plain
// Q4 element hu = hv = (D11 + D33)/12; Wilson's incompatible-mode element (Sec. 2) condenses to the
// same matrix with hu = hv = (D11 - D12^2/D22)/12, the bending modulus, so both come out of K_e0.
template <typename T>
inline Q4Consts<T> q4_consts(const double* Ke0) {
  const double g[4] = {1.0, -1.0, 1.0, -1.0};
  double gKg = 0.0, hKh = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      gKg += g[a] * Ke0[(2 * a) * 8 + 2 * b] * g[b];
      hKh += g[a] * Ke0[(2 * a + 1) * 8 + 2 * b + 1] * g[b];
    }
  const double hu = gKg / 16.0, hv = hKh / 16.0;
  const double mean_xx = Ke0[0] - hu, mean_x01 = Ke0[2] + hu;
  const double d11 = 2.0 * (mean_xx - mean_x01);
  const double d33 = 2.0 * (mean_xx + mean_x01);
  const double d12 = 4.0 * Ke0[1] - d33;
  Q4Consts<T> c;
  c.d11 = (T)d11;
  c.d22 = (T)d11;
  c.d12 = (T)d12;
  c.d33 = (T)d33;
  c.hu = (T)hu;
  c.hv = (T)hv;
  return c;
}

// Nodal forces f[8] = E K_e0 v_e of one element from its nodal displacements (local nodes 0..3 at
// (0,0), (1,0), (1,1), (0,1); u = x components, w = y components).
template <typename T>
__device__ __forceinline__ void q4_forces(T u0, T u1, T u2, T u3, T w0, T w1, T w2, T w3, T E, const Q4Consts<T>& cst,
                                          T (&f)[8]) {
  const T du10 = u1 - u0, du23 = u2 - u3, du30 = u3 - u0, du21 = u2 - u1;
  const T dw10 = w1 - w0, dw23 = w2 - w3, dw30 = w3 - w0, dw21 = w2 - w1;
  const T Au = du10 + du23, Bu = du30 + du21, hu = du23 - du10;  // 2 A_u, 2 B_u, h_u
  const T Av = dw10 + dw23, Bv = dw30 + dw21, hv = dw23 - dw10;  // 2 A_v, 2 B_v, h_v
  const T e4 = T(0.25) * E;
  const T a = cst.d11 * Au + cst.d12 * Bv;
  const T c = cst.d12 * Au + cst.d22 * Bv;
  const T t = cst.d33 * (Bu + Av);
  const T Pu = e4 * (a + t), Qu = e4 * (a - t);
  const T Pv = e4 * (c + t), Rv = e4 * (t - c);
  const T Hu = E * cst.hu * hu, Hv = E * cst.hv * hv;
  f[0] = -Pu + Hu;  // node 0 (0,0), x
  f[1] = -Pv + Hv;  //              y
  f[2] = Qu - Hu;   // node 1 (1,0)
  f[3] = Rv - Hv;
  f[4] = Pu + Hu;   // node 2 (1,1)
  f[5] = Pv + Hv;
  f[6] = -Qu - Hu;  // node 3 (0,1)
  f[7] = -Rv - Hv;
}

}  // namespace tobk
