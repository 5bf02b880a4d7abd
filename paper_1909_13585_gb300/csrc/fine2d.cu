// Fine-level (matrix-free) Q4 operator in factored form, element by element on shared-memory tiles.
//
// For the unit square element with 2x2 Gauss integration, the bilinear displacement gradient is
// fully described by six numbers per element: the mean gradients A_u = du/dx, B_u = du/dy,
// A_v = dv/dx, B_v = dv/dy and the two hourglass amplitudes h_u, h_v (u0 - u1 + u2 - u3).  The element
// strain energy is exactly
//   E/2 [D11 (A_u^2 + h_u^2/12) + 2 D12 A_u B_v + D22 (B_v^2 + h_v^2/12) + D33 ((B_u + A_v)^2 + (h_u^2 + h_v^2)/12)],
// so K_e v_e costs about 41 arithmetic operations instead of the 64 multiply-adds (plus scaling)
// of the dense 8 x 8 product; on GB300, where FP64 runs at 2 FMA/clk/SM, the fine-level smoother
// is bound by exactly this count.  A block computes the elements around a 32 x 8 tile of nodes once,
// stores their nodal forces in shared memory and gathers the four contributions of each node.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace tobk {

namespace {
constexpr int TX = 32, TY = 8;
constexpr int EX = TX + 1, EY = TY + 1;  // element tile
constexpr int NX = TX + 2, NY = TY + 2;  // node tile
}  // namespace

template <typename T>
struct Q4Consts {
  T d11, d12, d22, d33;  // plane-stress unit-modulus constitutive entries
  T hu, hv;              // (D11 + D33)/12, (D22 + D33)/12
};

template <typename T, int MODE>
__global__ void __launch_bounds__(TX* TY) k_fine_q4(Grid g, const T* __restrict__ Ek, const uint8_t* __restrict__ fixed,
                                                    Q4Consts<T> cst, const T* __restrict__ v, const T* __restrict__ b,
                                                    const T* __restrict__ dinv, T* __restrict__ y, SmoothArgs<T> sm,
                                                    int64_t stride, const double* __restrict__ act) {
  __shared__ T su[NY][NX], sv[NY][NX];
  __shared__ T fe[EY][EX][8];
  const int rhs = blockIdx.z;
  if (act != nullptr && act[(size_t)rhs * kScStride + SC_ACTIVE] == 0.0) return;
  const int tid = threadIdx.x;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int nnx = g.nn[0], nny = g.nn[1];
  const int64_t off = (int64_t)rhs * stride;
  for (int q = tid; q < NX * NY; q += TX * TY) {
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
  for (int q = tid; q < EX * EY; q += TX * TY) {
    const int lx = q % EX, ly = q / EX;
    const int ex = x0 - 1 + lx, ey = y0 - 1 + ly;
    T f[8];
    if (ex >= 0 && ex < g.nel[0] && ey >= 0 && ey < g.nel[1]) {
      const T E = __ldg(Ek + ex + (int64_t)g.nel[0] * ey);
      const T u0 = su[ly][lx], u1 = su[ly][lx + 1], u2 = su[ly + 1][lx + 1], u3 = su[ly + 1][lx];
      const T w0 = sv[ly][lx], w1 = sv[ly][lx + 1], w2 = sv[ly + 1][lx + 1], w3 = sv[ly + 1][lx];
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
    } else {
#pragma unroll
      for (int k = 0; k < 8; ++k) f[k] = T(0);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) fe[ly][lx][k] = f[k];
  }
  __syncthreads();
  const int tx = tid % TX, ty = tid / TX;
  const int X = x0 + tx, Y = y0 + ty;
  if (X >= nnx || Y >= nny) return;
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

template <typename T>
static Q4Consts<T> q4_consts(const double* Ke0) {
  // recover the constitutive entries from the unit element matrix (row-major 8 x 8):
  // K[0][0] = (D11 + D33)/3, K[0][1] = (D12 + D33)/4, K[0][2] = (-D11 + D33/2)/3 ... solved below
  // from three independent entries of K_e0 = sum_gp w|J| B^T D B:
  //   K[0][0] = D11/3 + D33/3,  K[0][2] = -D11/3 + D33/6,  K[0][1] = D12/4 + D33/4
  const double k00 = Ke0[0], k02 = Ke0[2], k01 = Ke0[1];
  const double d33 = 2.0 * (k00 + k02);              // (k00 + k02) = D33/2
  const double d11 = 3.0 * k00 - d33;
  const double d12 = 4.0 * k01 - d33;
  Q4Consts<T> c;
  c.d11 = (T)d11;
  c.d22 = (T)d11;
  c.d12 = (T)d12;
  c.d33 = (T)d33;
  c.hu = (T)((d11 + d33) / 12.0);
  c.hv = (T)((d11 + d33) / 12.0);
  return c;
}

template <typename T>
void launch_fine_q4(const Grid& g, const T* Ek, const uint8_t* fixed, const double* Ke0, int mode, const T* v,
                    const T* b, const T* dinv, T* y, SmoothArgs<T> sm, int nr, int64_t stride, cudaStream_t s) {
  const Q4Consts<T> cst = q4_consts<T>(Ke0);
  dim3 grid((unsigned)((g.nn[0] + TX - 1) / TX), (unsigned)((g.nn[1] + TY - 1) / TY), (unsigned)nr);
  const double* act = active_rhs();
  note_launch();
  if (mode == APPLY_KV)
    k_fine_q4<T, APPLY_KV><<<grid, TX * TY, 0, s>>>(g, Ek, fixed, cst, v, b, dinv, y, sm, stride, act);
  else if (mode == APPLY_RES)
    k_fine_q4<T, APPLY_RES><<<grid, TX * TY, 0, s>>>(g, Ek, fixed, cst, v, b, dinv, y, sm, stride, act);
  else
    k_fine_q4<T, APPLY_JAC><<<grid, TX * TY, 0, s>>>(g, Ek, fixed, cst, v, b, dinv, y, sm, stride, act);
}

template void launch_fine_q4<double>(const Grid&, const double*, const uint8_t*, const double*, int, const double*,
                                     const double*, const double*, double*, SmoothArgs<double>, int, int64_t,
                                     cudaStream_t);
template void launch_fine_q4<float>(const Grid&, const float*, const uint8_t*, const double*, int, const float*,
                                    const float*, const float*, float*, SmoothArgs<float>, int, int64_t, cudaStream_t);

}  // namespace tobk
