// The unit-modulus element stiffness K_e0 of Sec. 2 for the unit-cube H8 element, in factored form.
//
// Factored unit-cube H8 element operator (trilinear, isotropic, exact integration = 2x2x2 Gauss).
//
// With centred coordinates (xi, eta, zeta) in [-1/2, 1/2]^3, a trilinear field is
//   u = W_1/8 + (W_x xi + W_y eta + W_z zeta)/4 + (W_xy xi eta + W_yz eta zeta + W_zx zeta xi)/2
//       + W_xyz xi eta zeta,
// W_S = sum over the 8 nodes of s_S(node) u_node (s_S the product of the node's +-1 corner signs
// over the axes in S): a Walsh-Hadamard transform of the nodal values.  The displacement gradient
// then splits over the L2-orthogonal monomials 1, xi, eta, zeta, eta zeta, zeta xi, xi eta (norms 1,
// 1/12, 1/144), so the element strain energy E sum_phi |phi|^2 e(g_phi), e(g) = lambda/2 tr(g)^2 +
// mu |sym g|^2, needs only the 21 transformed values per element, and K_e v_e = dU/dv_e is the
// transposed transform of dU/dW.  About 200 arithmetic operations per element instead of the 576
// multiply-adds of the dense 24 x 24 product; exact (not an approximation) for unit cubes.
#pragma once
#include <cuda_runtime.h>

#include "unit_element.h"

namespace tobk {

template <typename T>
struct H8Consts {
  T l1, m1;   // mean gradient: lambda/16, mu/16
  T l2, m2;   // linear monomials: lambda/48, mu/48
  T hx;       // xi eta zeta mode: (lambda + 4 mu)/144
  T icd, ico; // incompatible-mode correction (0 for the plain element), see h8_forces
};

// Walsh sign s_S(l) of local node l for the mode S given as a bit set over the axes (1 x, 2 y, 4 z)
inline double h8_walsh_sign(int l, int S) {
  const int bx = ((l & 3) == 1 || (l & 3) == 2) ? 1 : 0, by = ((l & 3) >= 2) ? 1 : 0, bz = l >> 2;
  double s = 1.0;
  if (S & 1) s *= bx ? 1.0 : -1.0;
  if (S & 2) s *= by ? 1.0 : -1.0;
  if (S & 4) s *= bz ? 1.0 : -1.0;
  return s;
}

// Constants of the factored operator.  For the incompatible-mode hexahedron (Sec. 2) the condensed
// stiffness K_c differs from the trilinear one only in six bilinear Walsh modes, coupled in three
// pairs (u.xy, w.yz), (u.zx, v.yz), (v.xy, w.zx): per 64 of the Walsh sums, a diagonal entry icd and a
// pair coupling ico, here projected out of K_c - K_e0 on the host (their closed forms are
// -(4/3)(mu + lambda^2 / (lambda + 2 mu)) / 64 and -(4/3) lambda^2 / (lambda + 2 mu) / 64).
template <typename T>
inline H8Consts<T> h8_consts(double nu, int element = 0) {
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  H8Consts<T> c;
  c.l1 = (T)(lam / 16.0);
  c.m1 = (T)(mu / 16.0);
  c.l2 = (T)(lam / 48.0);
  c.m2 = (T)(mu / 48.0);
  c.hx = (T)((lam + 4.0 * mu) / 144.0);
  c.icd = c.ico = (T)0;
  if (element == 1) {
    double K0[24 * 24], Kc[24 * 24], A[9 * 24];
    unit_element::stiffness(3, nu, K0);
    unit_element::incompatible_tables(3, nu, Kc, A);
    double gux[24] = {0.0}, gwy[24] = {0.0};  // Walsh vectors of (u, xy) and (w, yz)
    for (int l = 0; l < 8; ++l) {
      gux[3 * l + 0] = h8_walsh_sign(l, 1 | 2);
      gwy[3 * l + 2] = h8_walsh_sign(l, 2 | 4);
    }
    double d = 0.0, o = 0.0;
    for (int a = 0; a < 24; ++a)
      for (int b = 0; b < 24; ++b) {
        const double cab = Kc[a * 24 + b] - K0[a * 24 + b];
        d += gux[a] * cab * gux[b];
        o += gux[a] * cab * gwy[b];
      }
    c.icd = (T)(d / 64.0);  // W^T W = 8 I for the 24 x 24 Walsh matrix W: C = W^T (W C W^T / 64) W
    c.ico = (T)(o / 64.0);
  }
  return c;
}

// Walsh sums of one component from v[cz][cy][cx]: out = {W_x, W_y, W_z, W_xy, W_yz, W_zx, W_xyz}
template <typename T>
__device__ __forceinline__ void h8_walsh(const T (&v)[2][2][2], T (&W)[7]) {
  T a[2][2], d[2][2];  // [cz][cy]
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int y = 0; y < 2; ++y) {
      a[z][y] = v[z][y][1] + v[z][y][0];
      d[z][y] = v[z][y][1] - v[z][y][0];
    }
  T aa[2], ad[2], da[2], dd[2];
#pragma unroll
  for (int z = 0; z < 2; ++z) {
    aa[z] = a[z][1] + a[z][0];
    ad[z] = a[z][1] - a[z][0];
    da[z] = d[z][1] + d[z][0];
    dd[z] = d[z][1] - d[z][0];
  }
  W[0] = da[1] + da[0];  // x
  W[1] = ad[1] + ad[0];  // y
  W[2] = aa[1] - aa[0];  // z
  W[3] = dd[1] + dd[0];  // xy
  W[4] = ad[1] - ad[0];  // yz
  W[5] = da[1] - da[0];  // zx
  W[6] = dd[1] - dd[0];  // xyz
}

// Transposed transform: f[cz][cy][cx] = sum_S D_S s_S(node), D_1 = 0.
template <typename T>
__device__ __forceinline__ void h8_walsh_t(const T (&D)[7], T (&f)[2][2][2]) {
  T aa[2], ad[2], da[2], dd[2];
  aa[1] = D[2];
  aa[0] = -D[2];
  ad[1] = D[1] + D[4];
  ad[0] = D[1] - D[4];
  da[1] = D[0] + D[5];
  da[0] = D[0] - D[5];
  dd[1] = D[3] + D[6];
  dd[0] = D[3] - D[6];
#pragma unroll
  for (int z = 0; z < 2; ++z) {
    const T a1 = aa[z] + ad[z], a0 = aa[z] - ad[z];
    const T d1 = da[z] + dd[z], d0 = da[z] - dd[z];
    f[z][1][1] = a1 + d1;
    f[z][1][0] = a1 - d1;
    f[z][0][1] = a0 + d0;
    f[z][0][0] = a0 - d0;
  }
}

// Element forces f[c][cz][cy][cx] = E (K_e0 v_e) for nodal displacements v[c][cz][cy][cx].
template <typename T>
__device__ __forceinline__ void h8_forces(const T (&v)[3][2][2][2], T E, const H8Consts<T>& k, T (&f)[3][2][2][2]) {
  T W[3][7];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h8_walsh<T>(v[c], W[c]);
#pragma unroll
    for (int s = 0; s < 7; ++s) W[c][s] *= E;
  }
  // indices into W[c]: 0 x, 1 y, 2 z, 3 xy, 4 yz, 5 zx, 6 xyz; components c: 0 u, 1 v, 2 w
  T D[3][7];
  // mean gradient g_ij = W[i][j] (x 1/4 folded into l1, m1)
  {
    const T tr = W[0][0] + W[1][1] + W[2][2];
    const T lt = k.l1 * tr;
    D[0][0] = lt + T(2) * k.m1 * W[0][0];
    D[1][1] = lt + T(2) * k.m1 * W[1][1];
    D[2][2] = lt + T(2) * k.m1 * W[2][2];
    const T sxy = k.m1 * (W[0][1] + W[1][0]);
    const T syz = k.m1 * (W[1][2] + W[2][1]);
    const T szx = k.m1 * (W[2][0] + W[0][2]);
    D[0][1] = sxy;
    D[1][0] = sxy;
    D[1][2] = syz;
    D[2][1] = syz;
    D[2][0] = szx;
    D[0][2] = szx;
  }
  // xi monomial: g_{i,y} = W[i][xy], g_{i,z} = W[i][zx]  (x 1/2 and the norm 1/12 folded into l2, m2)
  T Dxy[3], Dzx[3], Dyz[3];
  {
    const T ay = W[1][3], bz = W[2][5];
    const T lt = k.l2 * (ay + bz);
    const T syz = k.m2 * (W[1][5] + W[2][3]);
    Dxy[0] = k.m2 * W[0][3];
    Dxy[1] = lt + T(2) * k.m2 * ay;
    Dxy[2] = syz;
    Dzx[0] = k.m2 * W[0][5];
    Dzx[1] = syz;
    Dzx[2] = lt + T(2) * k.m2 * bz;
  }
  // eta monomial: g_{i,x} = W[i][xy], g_{i,z} = W[i][yz]
  {
    const T cx = W[0][3], dz = W[2][4];
    const T lt = k.l2 * (cx + dz);
    const T sxz = k.m2 * (W[0][4] + W[2][3]);
    Dxy[0] += lt + T(2) * k.m2 * cx;
    Dxy[1] += k.m2 * W[1][3];
    Dxy[2] += sxz;
    Dyz[0] = sxz;
    Dyz[1] = k.m2 * W[1][4];
    Dyz[2] = lt + T(2) * k.m2 * dz;
  }
  // zeta monomial: g_{i,x} = W[i][zx], g_{i,y} = W[i][yz]
  {
    const T ex = W[0][5], hy = W[1][4];
    const T lt = k.l2 * (ex + hy);
    const T sxy = k.m2 * (W[0][4] + W[1][5]);
    Dzx[0] += lt + T(2) * k.m2 * ex;
    Dzx[1] += sxy;
    Dzx[2] += k.m2 * W[2][5];
    Dyz[0] += sxy;
    Dyz[1] += lt + T(2) * k.m2 * hy;
    Dyz[2] += k.m2 * W[2][4];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    D[c][3] = Dxy[c];
    D[c][4] = Dyz[c];
    D[c][5] = Dzx[c];
  }
  if (k.icd != T(0)) {  // incompatible modes: the three coupled pairs of bilinear Walsh modes
    const T a03 = W[0][3], a24 = W[2][4], a05 = W[0][5], a14 = W[1][4], a13 = W[1][3], a25 = W[2][5];
    D[0][3] += k.icd * a03 + k.ico * a24;
    D[2][4] += k.icd * a24 + k.ico * a03;
    D[0][5] += k.icd * a05 + k.ico * a14;
    D[1][4] += k.icd * a14 + k.ico * a05;
    D[1][3] += k.icd * a13 + k.ico * a25;
    D[2][5] += k.icd * a25 + k.ico * a13;
  }
  // the three bilinear monomials act only on W_xyz: D_xyz = (lambda + 4 mu)/144 W_xyz per component
  D[0][6] = k.hx * W[0][6];
  D[1][6] = k.hx * W[1][6];
  D[2][6] = k.hx * W[2][6];
#pragma unroll
  for (int c = 0; c < 3; ++c) h8_walsh_t<T>(D[c], f[c]);
}

}  // namespace tobk
