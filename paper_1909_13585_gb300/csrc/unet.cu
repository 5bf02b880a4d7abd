// Learned warm start for the 3D MGCG solve: a small 3D U-Net (density field + load -> displacement
// guess u0) with hand-written forward, backward and Adam kernels.  Not part of the paper's method:
// plain mgPCG (Appendix A) still runs from u0 to the same tolerance and remains the fallback.
//
// Architecture (levels L, channels c_l; element grid nz x ny x nx, x fastest; tensors [C][D][H][W]):
//   features  ch0 = 2x - 1, ch1..3 = nodal load summed over each element's nodes / its largest value
//   encoder   e_0 = R(C(R(C(feat)))), e_l = R(C(R(C(avgpool(e_{l-1})))))
//   decoder   d_{L-1} = e_{L-1}, d_l = R(C(R(C([up(d_{l+1}), e_l]))))
//   output    y = H(d_0) + up^{L-1}(Hc(e_{L-1}))  (fine head + coarse-correction head, 3 channels)
//   guess     u0 = c (mean of y over the elements around each node) / s at free DOFs,
//             s = mean(E_kappa) / (largest element load sum), c a fixed output scale (set from the
//             training data, so that the network's outputs are of order one)
//   C = 3x3x3 convolution (zero padding, bias), R = ReLU, H, Hc = 1x1x1 convolutions.
// Loss of a sample with solution u (t = c x node averages, t* = s u, K the sample's stiffness):
//   energy (default): (t - t*)^T K (t - t*) / t*^T K t* over the free DOFs (K t* = s f), the
//                     relative energy-norm error of the guess, which is what CG convergence sees;
//                     K t comes from the library's factored H8 operator;
//   mse:              sum_free (t - t*)^2 / sum_free t*^2.
// Parameters: one flat FP32 vector (master copy for Adam) in the order enc_l a, enc_l b (l = 0..L-1),
// dec_l a, dec_l b (l = L-2..0), head, coarse head; each layer W [Cout][Cin][taps] then b [Cout];
// the kernels read a bfloat16 copy and accumulate in FP32.
//
// Kernels: the 3x3x3 convolution is a direct convolution on 4 x 4 x 16 voxel tiles, 16 output
// channels per block, input channels staged through shared memory 8 at a time (the backward data
// pass is the same kernel with the weights read transposed and flipped); the weight gradient
// reduces over voxel tiles per (16 x 16) channel block with one FP32 atomic add per weight and block.
// Inference (predict) runs the 3x3x3 convolutions on the tensor cores by default (conv3_tc.cuh:
// tcgen05 implicit GEMM, activations rounded to bfloat16 when staged, FP32 accumulation); training
// keeps FP32 activations (the gradients are those of the FP32-activation network).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tobk.h"
#include "conv3_tc.cuh"
#include "kernels.h"
#include "tobk_internal.cuh"

namespace tobk {
namespace {

constexpr int kTZ = 4, kTY = 4, kTX = 16;  // voxel tile of the convolution kernels (256 threads)
constexpr int kCOT = 16;                  // output channels per block
constexpr int kCIT = 8;                   // input channels per shared-memory stage
constexpr int kHZ = kTZ + 2, kHY = kTY + 2, kHX = kTX + 2;

struct Dim3 {
  int D, H, W;
  __host__ __device__ int64_t vox() const { return (int64_t)D * H * W; }
};

// ---- 3x3x3 convolution (forward, and backward-data with wmode = 1) ------------------------------
// out[co][v] = bias[co] + sum_ci sum_tap w(co, ci, tap) * inp(ci, v + tap), inp(ci) = in1 (channels
// < C1; read at half resolution when up1) or in2 (channels >= C1), each optionally multiplied by
// (mask > 0).  wmode 0: w(co, ci, tap) = W[(co * Cin + ci) * 27 + tap]; wmode 1 (transposed and
// flipped, for the gradient with respect to the input of a layer with wcout outputs and Cin inputs
// here playing the roles swapped): w(co, ci, tap) = W[(ci * wcin + co) * 27 + 26 - tap].
__global__ void __launch_bounds__(256) k_conv3(const float* __restrict__ in1, const float* __restrict__ mask1, int C1,
                                               int up1, const float* __restrict__ in2, int C2,
                                               const __nv_bfloat16* __restrict__ W, int wmode, int wcin,
                                               const __nv_bfloat16* __restrict__ bias, float* __restrict__ out,
                                               int Cout, Dim3 d, int relu) {
  __shared__ float s_in[kCIT][kHZ][kHY][kHX];
  __shared__ float4 s_w[kCIT][27][kCOT / 4];
  const int Cin = C1 + C2;
  const int tx = threadIdx.x % kTX, ty = (threadIdx.x / kTX) % kTY, tz = threadIdx.x / (kTX * kTY);
  const int tilesX = (d.W + kTX - 1) / kTX, tilesY = (d.H + kTY - 1) / kTY;
  const int bx = blockIdx.x % tilesX, by = (blockIdx.x / tilesX) % tilesY, bz = blockIdx.x / (tilesX * tilesY);
  const int x0 = bx * kTX, y0 = by * kTY, z0 = bz * kTZ;
  const int co0 = blockIdx.y * kCOT;
  const int64_t V = d.vox();
  const Dim3 dc{d.D / 2, d.H / 2, d.W / 2};
  float acc[kCOT];
#pragma unroll
  for (int k = 0; k < kCOT; ++k) acc[k] = 0.f;
  for (int c0 = 0; c0 < Cin; c0 += kCIT) {
    for (int q = threadIdx.x; q < kCIT * kHZ * kHY * kHX; q += 256) {
      const int lx = q % kHX, ly = (q / kHX) % kHY, lz = (q / (kHX * kHY)) % kHZ, lc = q / (kHX * kHY * kHZ);
      const int x = x0 + lx - 1, y = y0 + ly - 1, z = z0 + lz - 1, c = c0 + lc;
      float v = 0.f;
      if (c < Cin && x >= 0 && x < d.W && y >= 0 && y < d.H && z >= 0 && z < d.D) {
        if (c < C1) {
          int64_t idx;
          if (up1)
            idx = (int64_t)c * dc.vox() + ((int64_t)(z >> 1) * dc.H + (y >> 1)) * dc.W + (x >> 1);
          else
            idx = (int64_t)c * V + ((int64_t)z * d.H + y) * d.W + x;
          v = in1[idx];
          if (mask1 && !(mask1[idx] > 0.f)) v = 0.f;
        } else {
          v = in2[(int64_t)(c - C1) * V + ((int64_t)z * d.H + y) * d.W + x];
        }
      }
      s_in[lc][lz][ly][lx] = v;
    }
    for (int q = threadIdx.x; q < kCIT * 27 * kCOT; q += 256) {
      const int co = q % kCOT, tap = (q / kCOT) % 27, lc = q / (kCOT * 27);
      const int ci = c0 + lc, o = co0 + co;
      float w = 0.f;
      if (ci < Cin && o < Cout) {
        const int64_t wi = wmode == 0 ? ((int64_t)o * Cin + ci) * 27 + tap : ((int64_t)ci * wcin + o) * 27 + 26 - tap;
        w = __bfloat162float(W[wi]);
      }
      reinterpret_cast<float*>(&s_w[lc][tap][0])[co] = w;
    }
    __syncthreads();
#pragma unroll 1
    for (int lc = 0; lc < kCIT; ++lc) {
#pragma unroll
      for (int tap = 0; tap < 27; ++tap) {
        const float v = s_in[lc][tz + tap / 9][ty + (tap / 3) % 3][tx + tap % 3];
#pragma unroll
        for (int k = 0; k < kCOT / 4; ++k) {
          const float4 w = s_w[lc][tap][k];
          acc[4 * k] += w.x * v;
          acc[4 * k + 1] += w.y * v;
          acc[4 * k + 2] += w.z * v;
          acc[4 * k + 3] += w.w * v;
        }
      }
    }
    __syncthreads();
  }
  const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
  if (x >= d.W || y >= d.H || z >= d.D) return;
  const int64_t vi = ((int64_t)z * d.H + y) * d.W + x;
#pragma unroll
  for (int k = 0; k < kCOT; ++k) {
    const int o = co0 + k;
    if (o >= Cout) break;
    float r = acc[k] + (bias ? __bfloat162float(bias[o]) : 0.f);
    if (relu) r = fmaxf(r, 0.f);
    out[(int64_t)o * V + vi] = r;
  }
}

// ---- weight / bias gradient of a 3x3x3 convolution ----------------------------------------------
// gW[co][ci][tap] += sum_v gm(co, v) inp(ci, v + tap), gb[co] += sum_v gm(co, v), gm = g * (out > 0).
// Block: 16 output x 16 input channels (thread = one (co, ci) pair, 27 accumulators), a strided set
// of 4 x 4 x 8 voxel tiles.
constexpr int kWX = 8;
__global__ void __launch_bounds__(256) k_conv3_wgrad(const float* __restrict__ g, const float* __restrict__ omask,
                                                     const float* __restrict__ in1, int C1, int up1,
                                                     const float* __restrict__ in2, int C2, float* __restrict__ gW,
                                                     float* __restrict__ gb, int Cout, Dim3 d) {
  __shared__ float s_g[16][kTZ * kTY * kWX];
  __shared__ float s_in[16][kHZ][kHY][kWX + 2];
  const int Cin = C1 + C2;
  const int co = blockIdx.y * 16 + threadIdx.x / 16, ci = blockIdx.z * 16 + threadIdx.x % 16;
  const int lco = threadIdx.x / 16, lci = threadIdx.x % 16;
  const int tilesX = (d.W + kWX - 1) / kWX, tilesY = (d.H + kTY - 1) / kTY, tilesZ = (d.D + kTZ - 1) / kTZ;
  const int ntiles = tilesX * tilesY * tilesZ;
  const int64_t V = d.vox();
  const Dim3 dc{d.D / 2, d.H / 2, d.W / 2};
  float acc[27];
#pragma unroll
  for (int t = 0; t < 27; ++t) acc[t] = 0.f;
  float bacc = 0.f;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int bx = tile % tilesX, by = (tile / tilesX) % tilesY, bz = tile / (tilesX * tilesY);
    const int x0 = bx * kWX, y0 = by * kTY, z0 = bz * kTZ;
    for (int q = threadIdx.x; q < 16 * kTZ * kTY * kWX; q += 256) {
      const int lv = q % (kTZ * kTY * kWX), lc = q / (kTZ * kTY * kWX);
      const int x = x0 + lv % kWX, y = y0 + (lv / kWX) % kTY, z = z0 + lv / (kWX * kTY);
      const int o = blockIdx.y * 16 + lc;
      float v = 0.f;
      if (o < Cout && x < d.W && y < d.H && z < d.D) {
        const int64_t idx = (int64_t)o * V + ((int64_t)z * d.H + y) * d.W + x;
        v = g[idx];
        if (omask && !(omask[idx] > 0.f)) v = 0.f;
      }
      s_g[lc][lv] = v;
    }
    for (int q = threadIdx.x; q < 16 * kHZ * kHY * (kWX + 2); q += 256) {
      const int lx = q % (kWX + 2), ly = (q / (kWX + 2)) % kHY, lz = (q / ((kWX + 2) * kHY)) % kHZ,
                lc = q / ((kWX + 2) * kHY * kHZ);
      const int x = x0 + lx - 1, y = y0 + ly - 1, z = z0 + lz - 1, c = blockIdx.z * 16 + lc;
      float v = 0.f;
      if (c < Cin && x >= 0 && x < d.W && y >= 0 && y < d.H && z >= 0 && z < d.D) {
        if (c < C1) {
          const int64_t idx = up1 ? (int64_t)c * dc.vox() + ((int64_t)(z >> 1) * dc.H + (y >> 1)) * dc.W + (x >> 1)
                                  : (int64_t)c * V + ((int64_t)z * d.H + y) * d.W + x;
          v = in1[idx];
        } else {
          v = in2[(int64_t)(c - C1) * V + ((int64_t)z * d.H + y) * d.W + x];
        }
      }
      s_in[lc][lz][ly][lx] = v;
    }
    __syncthreads();
    for (int lv = 0; lv < kTZ * kTY * kWX; ++lv) {
      const int vx = lv % kWX, vy = (lv / kWX) % kTY, vz = lv / (kWX * kTY);
      const float gv = s_g[lco][lv];
      bacc += gv;
#pragma unroll
      for (int t = 0; t < 27; ++t) acc[t] += gv * s_in[lci][vz + t / 9][vy + (t / 3) % 3][vx + t % 3];
    }
    __syncthreads();
  }
  if (co < Cout && ci < Cin) {
#pragma unroll
    for (int t = 0; t < 27; ++t) atomicAdd(gW + ((int64_t)co * Cin + ci) * 27 + t, acc[t]);
    if (blockIdx.z == 0 && lci == 0) atomicAdd(gb + co, bacc);
  }
}

// ---- 1x1x1 convolutions (the heads) -------------------------------------------------------------
// out[o][v] (+)= b[o] + sum_i W[o][i] in[i][v], o < 3
__global__ void k_conv1(const float* __restrict__ in, int Cin, const __nv_bfloat16* __restrict__ W,
                        const __nv_bfloat16* __restrict__ b, float* __restrict__ out, int64_t V) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float a0 = __bfloat162float(b[0]), a1 = __bfloat162float(b[1]), a2 = __bfloat162float(b[2]);
  for (int i = 0; i < Cin; ++i) {
    const float x = in[(int64_t)i * V + v];
    a0 += __bfloat162float(W[i]) * x;
    a1 += __bfloat162float(W[Cin + i]) * x;
    a2 += __bfloat162float(W[2 * Cin + i]) * x;
  }
  out[v] = a0;
  out[V + v] = a1;
  out[2 * V + v] = a2;
}

// gin[i][v] (+)= sum_o W[o][i] g[o][v]  (accumulate when acc != 0)
__global__ void k_conv1_bwd_data(const float* __restrict__ g, int Cin, const __nv_bfloat16* __restrict__ W,
                                 float* __restrict__ gin, int64_t V, int acc) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const float g0 = g[v], g1 = g[V + v], g2 = g[2 * V + v];
  for (int i = 0; i < Cin; ++i) {
    const float r = __bfloat162float(W[i]) * g0 + __bfloat162float(W[Cin + i]) * g1 + __bfloat162float(W[2 * Cin + i]) * g2;
    gin[(int64_t)i * V + v] = acc ? gin[(int64_t)i * V + v] + r : r;
  }
}

// gW[o][i] += sum_v g[o][v] in[i][v], gb[o] += sum_v g[o][v]; one block per input channel i (and
// one extra block, i = Cin, for the bias)
__global__ void __launch_bounds__(256) k_conv1_wgrad(const float* __restrict__ g, const float* __restrict__ in, int Cin,
                                                     float* __restrict__ gW, float* __restrict__ gb, int64_t V) {
  __shared__ float red[3][8];
  const int i = blockIdx.x;
  float a[3] = {0.f, 0.f, 0.f};
  for (int64_t v = threadIdx.x; v < V; v += blockDim.x) {
    const float x = i < Cin ? in[(int64_t)i * V + v] : 1.f;
#pragma unroll
    for (int o = 0; o < 3; ++o) a[o] += g[(int64_t)o * V + v] * x;
  }
#pragma unroll
  for (int o = 0; o < 3; ++o) {
    for (int s = 16; s > 0; s >>= 1) a[o] += __shfl_xor_sync(0xffffffffu, a[o], s);
    if ((threadIdx.x & 31) == 0) red[o][threadIdx.x >> 5] = a[o];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float s = 0.f;
    for (int w = 0; w < 8; ++w) s += red[threadIdx.x][w];
    if (i < Cin)
      gW[threadIdx.x * Cin + i] += s;
    else
      gb[threadIdx.x] += s;
  }
}

// ---- pooling / upsampling -----------------------------------------------------------------------
__global__ void k_avgpool(const float* __restrict__ a, float* __restrict__ out, int C, Dim3 dc) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)C * dc.vox()) return;
  const int64_t c = q / dc.vox(), r = q % dc.vox();
  const int x = (int)(r % dc.W), y = (int)((r / dc.W) % dc.H), z = (int)(r / ((int64_t)dc.W * dc.H));
  const Dim3 df{2 * dc.D, 2 * dc.H, 2 * dc.W};
  float s = 0.f;
  for (int k = 0; k < 8; ++k)
    s += a[c * df.vox() + ((int64_t)(2 * z + (k >> 2)) * df.H + 2 * y + ((k >> 1) & 1)) * df.W + 2 * x + (k & 1)];
  out[q] = 0.125f * s;
}

// gf[c][v] += gc[c][v/2] / 8 (avgpool backward, accumulated into the fine gradient)
__global__ void k_avgpool_bwd(const float* __restrict__ gc, float* __restrict__ gf, int C, Dim3 df) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)C * df.vox()) return;
  const int64_t c = q / df.vox(), r = q % df.vox();
  const int x = (int)(r % df.W), y = (int)((r / df.W) % df.H), z = (int)(r / ((int64_t)df.W * df.H));
  const Dim3 dc{df.D / 2, df.H / 2, df.W / 2};
  gf[q] += 0.125f * gc[c * dc.vox() + ((int64_t)(z >> 1) * dc.H + (y >> 1)) * dc.W + (x >> 1)];
}

// gc[c][V] (+)= sum of the 8 children of V in gf[c0 + c]  (nearest-upsampling backward)
__global__ void k_sumpool(const float* __restrict__ gf, int c0, float* __restrict__ gc, int C, Dim3 dc, int acc) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)C * dc.vox()) return;
  const int64_t c = q / dc.vox(), r = q % dc.vox();
  const int x = (int)(r % dc.W), y = (int)((r / dc.W) % dc.H), z = (int)(r / ((int64_t)dc.W * dc.H));
  const Dim3 df{2 * dc.D, 2 * dc.H, 2 * dc.W};
  float s = 0.f;
  for (int k = 0; k < 8; ++k)
    s += gf[(c0 + c) * df.vox() + ((int64_t)(2 * z + (k >> 2)) * df.H + 2 * y + ((k >> 1) & 1)) * df.W + 2 * x + (k & 1)];
  gc[q] = acc ? gc[q] + s : s;
}

// dst[c][v] += src[c0 + c][v]
__global__ void k_add_channels(const float* __restrict__ src, int c0, float* __restrict__ dst, int64_t count, int64_t V) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < count) dst[q] += src[c0 * V + q];
}

// ---- features, output and loss -------------------------------------------------------------------
// feat[0] = 2x - 1; feat[1..3] = sum of the element's nodal loads (scaled later); Ek per element.
__global__ void k_unet_features(const float* __restrict__ xf, const double* __restrict__ xd, const double* __restrict__ f,
                                Dim3 d, double penal, double E0, double Emin, float* __restrict__ feat,
                                float* __restrict__ Ek) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.vox()) return;
  const int x = (int)(e % d.W), y = (int)((e / d.W) % d.H), z = (int)(e / ((int64_t)d.W * d.H));
  const double xe = xf ? (double)xf[e] : xd[e];
  float s[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < 8; ++k) {
    const int64_t a = ((int64_t)(z + (k >> 2)) * (d.H + 1) + y + ((k >> 1) & 1)) * (d.W + 1) + x + (k & 1);
#pragma unroll
    for (int c = 0; c < 3; ++c) s[c] += (float)f[3 * a + c];
  }
  const int64_t V = d.vox();
  feat[e] = (float)(2.0 * xe - 1.0);
  for (int c = 0; c < 3; ++c) feat[(1 + c) * V + e] = s[c];
  Ek[e] = (float)(Emin + pow(xe, penal) * (E0 - Emin));
}

// one block: sc[0] = 1 / max|feat[1..3]|, sc[1] = s = mean(Ek) * sc[0]; then the load channels are
// scaled by sc[0] (second kernel)
__global__ void __launch_bounds__(1024) k_unet_scale(const float* __restrict__ feat, const float* __restrict__ Ek,
                                                     int64_t V, float* __restrict__ sc) {
  __shared__ double rm[32], rs[32];
  double mx = 0.0, sum = 0.0;
  for (int64_t q = threadIdx.x; q < V; q += blockDim.x) {
    for (int c = 1; c < 4; ++c) mx = fmax(mx, fabs((double)feat[c * V + q]));
    sum += Ek[q];
  }
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rm[threadIdx.x >> 5] = mx;
    rs[threadIdx.x >> 5] = sum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      m = fmax(m, rm[w]);
      s += rs[w];
    }
    const double inv = m > 0.0 ? 1.0 / m : 1.0;
    sc[0] = (float)inv;
    sc[1] = (float)(s / (double)V * inv);
  }
}

__global__ void k_unet_scale_load(float* __restrict__ feat, int64_t V, const float* __restrict__ sc) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 3 * V) feat[V + q] *= sc[0];
}

// node value t[a][c] = mean over the elements around node a of (yh[c] + yc[c] at the element's
// coarse ancestor), coarse level cl (yc at resolution / 2^cl)
__device__ __forceinline__ float y_elem(const float* yh, const float* yc, int c, int x, int y, int z, Dim3 d, int cl) {
  const Dim3 dc{d.D >> cl, d.H >> cl, d.W >> cl};
  return yh[(int64_t)c * d.vox() + ((int64_t)z * d.H + y) * d.W + x] +
         yc[(int64_t)c * dc.vox() + ((int64_t)(z >> cl) * dc.H + (y >> cl)) * dc.W + (x >> cl)];
}

// mode 0: predict: u0[3a + c] = t / s (0 at fixed DOFs), FP64 output
// mode 1: node values t (FP32, 0 at fixed DOFs) into tn, for the loss
__global__ void __launch_bounds__(256) k_unet_nodes(const float* __restrict__ yh, const float* __restrict__ yc, Dim3 d,
                                                    int cl, const uint8_t* __restrict__ fixed, const float* __restrict__ sc,
                                                    float out_scale, int mode, double* __restrict__ u0,
                                                    float* __restrict__ tn) {
  const int64_t nnode = (int64_t)(d.D + 1) * (d.H + 1) * (d.W + 1);
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nnode) return;
  const int x = (int)(a % (d.W + 1)), y = (int)((a / (d.W + 1)) % (d.H + 1)), z = (int)(a / ((int64_t)(d.W + 1) * (d.H + 1)));
  float t[3] = {0.f, 0.f, 0.f};
  int cnt = 0;
  for (int k = 0; k < 8; ++k) {
    const int ex = x - (k & 1), ey = y - ((k >> 1) & 1), ez = z - (k >> 2);
    if (ex < 0 || ex >= d.W || ey < 0 || ey >= d.H || ez < 0 || ez >= d.D) continue;
    ++cnt;
    for (int c = 0; c < 3; ++c) t[c] += y_elem(yh, yc, c, ex, ey, ez, d, cl);
  }
  const float s = sc[1];
  for (int c = 0; c < 3; ++c) {
    const int64_t i = 3 * a + c;
    const float tv = out_scale * t[c] / (float)cnt;
    if (mode == 0)
      u0[i] = fixed[i] ? 0.0 : (double)tv / (double)s;
    else
      tn[i] = fixed[i] ? 0.f : tv;
  }
}

// Loss partials over the free DOFs (one pair of sums per block, 3 sums each):
//   mse:    (t - s u)^2, (s u)^2;                     dt = t - s u
//   energy: t.Kt, t.f, u.f;                           dt = K t - s f
__global__ void __launch_bounds__(256) k_unet_loss_partial(const float* __restrict__ tn, const float* __restrict__ Kt,
                                                           const float* __restrict__ u, const double* __restrict__ f,
                                                           const uint8_t* __restrict__ fixed,
                                                           const float* __restrict__ sc, int64_t n, int energy,
                                                           float* __restrict__ dt, double* __restrict__ partial) {
  __shared__ double red[3][8];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double v[3] = {0.0, 0.0, 0.0};
  if (i < n) {
    const float s = sc[1];
    const bool fr = !fixed[i];
    if (energy) {
      const double fi = f[i];
      dt[i] = fr ? (float)((double)Kt[i] - s * fi) : 0.f;
      if (fr) {
        v[0] = (double)tn[i] * Kt[i];
        v[1] = (double)tn[i] * fi;
        v[2] = (double)u[i] * fi;
      }
    } else {
      const float tgt = s * u[i];
      const float df = fr ? tn[i] - tgt : 0.f;
      dt[i] = df;
      v[0] = (double)df * df;
      v[1] = fr ? (double)tgt * tgt : 0.0;
    }
  }
  for (int q = 0; q < 3; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 3; ++q) red[q][threadIdx.x >> 5] = v[q];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) {
      double a = 0.0;
      for (int w = 0; w < 8; ++w) a += red[q][w];
      partial[3 * blockIdx.x + q] = a;
    }
}

// loss[0] += the sample's loss; gscale[0] = d loss / d(dt) factor (one block)
//   mse:    sum0 / sum1,                               2 / sum1
//   energy: (t.Kt - 2 s t.f + s^2 u.f) / (s^2 u.f),    2 / (s^2 u.f)
__global__ void __launch_bounds__(256) k_unet_loss_final(const double* __restrict__ partial, int nb,
                                                         const float* __restrict__ sc, int energy,
                                                         float* __restrict__ loss, float* __restrict__ gscale) {
  __shared__ double red[3][8];
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    for (int q = 0; q < 3; ++q) v[q] += partial[3 * b + q];
  for (int q = 0; q < 3; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  if ((threadIdx.x & 31) == 0)
    for (int q = 0; q < 3; ++q) red[q][threadIdx.x >> 5] = v[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    double a[3] = {0.0, 0.0, 0.0};
    for (int q = 0; q < 3; ++q)
      for (int w = 0; w < 8; ++w) a[q] += red[q][w];
    if (energy) {
      const double s = sc[1], den = s * s * a[2];
      loss[0] += (float)((a[0] - 2.0 * s * a[1] + s * s * a[2]) / den);
      gscale[0] = (float)(2.0 / den);
    } else {
      loss[0] += (float)(a[0] / a[1]);
      gscale[0] = (float)(2.0 / a[1]);
    }
  }
}

// gy[c][e] = sum over the element's nodes a of gscale * dt[3a + c] / cnt(a)   (node-average backward)
__global__ void k_unet_nodes_bwd(const float* __restrict__ dt, const float* __restrict__ gscale, float out_scale,
                                 Dim3 d, float* __restrict__ gy) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.vox()) return;
  const int x = (int)(e % d.W), y = (int)((e / d.W) % d.H), z = (int)(e / ((int64_t)d.W * d.H));
  float g[3] = {0.f, 0.f, 0.f};
  for (int k = 0; k < 8; ++k) {
    const int nx = x + (k & 1), ny = y + ((k >> 1) & 1), nz = z + (k >> 2);
    const int cnt = (nx > 0 && nx < d.W ? 2 : 1) * (ny > 0 && ny < d.H ? 2 : 1) * (nz > 0 && nz < d.D ? 2 : 1);
    const int64_t a = ((int64_t)nz * (d.H + 1) + ny) * (d.W + 1) + nx;
    for (int c = 0; c < 3; ++c) g[c] += dt[3 * a + c] / (float)cnt;
  }
  for (int c = 0; c < 3; ++c) gy[(int64_t)c * d.vox() + e] = out_scale * gscale[0] * g[c];
}

// ---- optimizer ----------------------------------------------------------------------------------
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       __nv_bfloat16* __restrict__ pb, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2, float gs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = gs * g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// wt[(tap * cout + n) * Kp + k] = W[n][k][tap] (zero for k >= cin)
__global__ void k_tc_weights(const __nv_bfloat16* __restrict__ W, int cout, int cin, int Kp,
                             __nv_bfloat16* __restrict__ wt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)27 * cout * Kp) return;
  const int k = (int)(i % Kp), n = (int)((i / Kp) % cout), tap = (int)(i / ((int64_t)Kp * cout));
  wt[i] = k < cin ? W[((int64_t)n * cin + k) * 27 + tap] : __float2bfloat16(0.f);
}


uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace
}  // namespace tobk

using namespace tobk;

struct tobk_unet {
  tobk_unet_desc desc{};
  cudaStream_t stream = nullptr;
  int L = 4;
  std::vector<int> c;
  struct Layer {
    int cout, cin, taps;
    int64_t w, b;  // offsets into the flat parameter vector
  };
  std::vector<Layer> layers;  // in parameter order
  int64_t np = 0;
  std::vector<Dim3> dims;     // per level
  char* arena = nullptr;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* pb = nullptr;
  // activations [level]
  std::vector<float*> in, a, e, da, d, ge, gd, gtmp;
  float *feat = nullptr, *Ek = nullptr, *yh = nullptr, *yc = nullptr, *gy = nullptr, *gyc = nullptr, *dt = nullptr;
  float *tn = nullptr, *Kt = nullptr;  // node values of the guess and K times them (loss)
  float *scratch = nullptr, *scratch2 = nullptr;
  float *sc = nullptr, *lossd = nullptr, *gscale = nullptr;
  double* partial = nullptr;
  float* host = nullptr;  // pinned scalars
  long long step = 0;
  float out_scale = 1.f;  // t = out_scale * (node average of the network output)
  int tensor_cores = 1;   // inference convolutions: 0 direct, 1 tensor cores on large grids, 2 always
  __nv_bfloat16* wt = nullptr;  // 3x3x3 weights re-laid out for the tensor-core kernel [27][Cout][Kp]
  std::vector<int64_t> wt_off;  // per layer offset into wt (-1: not a 3x3x3 layer)
  unsigned* tc_err = nullptr;   // set by a tensor-core wait that gave up
  std::string err;
};

namespace {

int ufail(tobk_unet* u, int code, const std::string& m) {
  u->err = m;
  return code;
}

// layer indices: enc l a = 2l, enc l b = 2l + 1; dec l a / b = 2L + 2 (L - 2 - l) (+1); head, chead last
int enc_a(const tobk_unet* u, int l) { return 2 * l; }
int dec_a(const tobk_unet* u, int l) { return 2 * u->L + 2 * (u->L - 2 - l); }
int head_i(const tobk_unet* u) { return (int)u->layers.size() - 2; }
int chead_i(const tobk_unet* u) { return (int)u->layers.size() - 1; }

int kpad(int cin) { return (cin + 15) / 16 * 16; }

bool tc_fits(int cout, int cin) {
  return (cout == 16 || cout == 32 || cout == 64 || cout == 128) &&
         tc::conv3_tc_smem(cout, kpad(cin)) <= (size_t)200 * 1024;
}

// the row variant (one halo slab per 128-voxel x run) when W is a multiple of 128 and its slab
// fits, else the per-tap gather variant
template <int N>
void launch_conv3_tc(const tc::ConvTcArgs& a, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(tc::k_conv3_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024));
    cudaFuncSetAttribute(tc::k_conv3_tc_row<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024));
    configured = true;
  }
  const unsigned grid = (unsigned)((a.d.vox() + 127) / 128);
  note_launch();
  if (a.d.W % 128 == 0 && tc::conv3_tc_row_smem(N, a.Kp) <= (size_t)200 * 1024)
    tc::k_conv3_tc_row<N><<<grid, 128, tc::conv3_tc_row_smem(N, a.Kp), s>>>(a);
  else
    tc::k_conv3_tc<N><<<grid, 128, tc::conv3_tc_smem(N, a.Kp), s>>>(a);
}

void conv3_fwd_tc(tobk_unet* u, int li, const float* in1, int C1, int up1, const float* in2, int C2, float* out,
                  const Dim3& d) {
  const auto& L = u->layers[li];
  const tc::ConvTcArgs a{in1, nullptr, C1, up1, in2, C2, u->wt + u->wt_off[li], u->pb + L.b, out,
                         tc::Dim3{d.D, d.H, d.W}, kpad(L.cin), 1, u->tc_err};
  switch (L.cout) {
    case 16: launch_conv3_tc<16>(a, u->stream); break;
    case 32: launch_conv3_tc<32>(a, u->stream); break;
    case 64: launch_conv3_tc<64>(a, u->stream); break;
    default: launch_conv3_tc<128>(a, u->stream); break;
  }
}

void conv3_fwd(tobk_unet* u, int li, const float* in1, int C1, int up1, const float* in2, int C2, float* out,
               const Dim3& d, bool tensor_cores = false) {
  const auto& L = u->layers[li];
  // the tensor-core kernels serialise 27 staged taps per 128-voxel tile: below ~2 tiles per SM the
  // direct convolution (many more, smaller blocks) is faster, so mode 1 keeps it there
  const bool big = d.vox() >= (int64_t)128 * 2 * 152;
  if (tensor_cores && u->wt_off[li] >= 0 && (u->tensor_cores == 2 || big)) {
    conv3_fwd_tc(u, li, in1, C1, up1, in2, C2, out, d);
    return;
  }
  const unsigned tiles = (unsigned)(((d.W + kTX - 1) / kTX) * ((d.H + kTY - 1) / kTY) * ((d.D + kTZ - 1) / kTZ));
  note_launch();
  k_conv3<<<dim3(tiles, (L.cout + kCOT - 1) / kCOT), 256, 0, u->stream>>>(in1, nullptr, C1, up1, in2, C2, u->pb + L.w, 0,
                                                                         L.cin, u->pb + L.b, out, L.cout, d, 1);
}

// gradient with respect to the layer's input (all Cin channels) into dst [Cin][V], from the output
// gradient g and the layer's output (ReLU mask)
void conv3_bwd_data(tobk_unet* u, int li, const float* g, const float* out, float* dst, const Dim3& d) {
  const auto& L = u->layers[li];
  const unsigned tiles = (unsigned)(((d.W + kTX - 1) / kTX) * ((d.H + kTY - 1) / kTY) * ((d.D + kTZ - 1) / kTZ));
  note_launch();
  k_conv3<<<dim3(tiles, (L.cin + kCOT - 1) / kCOT), 256, 0, u->stream>>>(g, out, L.cout, 0, nullptr, 0, u->pb + L.w, 1,
                                                                        L.cin, nullptr, dst, L.cin, d, 0);
}

void conv3_wgrad(tobk_unet* u, int li, const float* g, const float* out, const float* in1, int C1, int up1,
                 const float* in2, int C2, const Dim3& d) {
  const auto& L = u->layers[li];
  const int tiles = ((d.W + kWX - 1) / kWX) * ((d.H + kTY - 1) / kTY) * ((d.D + kTZ - 1) / kTZ);
  const unsigned gx = (unsigned)std::max(1, std::min(tiles, 2 * 152));
  note_launch();
  k_conv3_wgrad<<<dim3(gx, (L.cout + 15) / 16, (L.cin + 15) / 16), 256, 0, u->stream>>>(
      g, out, in1, C1, up1, in2, C2, u->g + L.w, u->g + L.b, L.cout, d);
}

void forward(tobk_unet* u, bool tensor_cores = false) {
  cudaStream_t s = u->stream;
  const int L = u->L;
  if (tensor_cores)
    for (size_t li = 0; li < u->layers.size(); ++li)
      if (u->wt_off[li] >= 0) {
        const auto& ly = u->layers[li];
        const int64_t cnt = (int64_t)27 * ly.cout * kpad(ly.cin);
        note_launch();
        k_tc_weights<<<nb(cnt), 256, 0, s>>>(u->pb + ly.w, ly.cout, ly.cin, kpad(ly.cin), u->wt + u->wt_off[li]);
      }
  for (int l = 0; l < L; ++l) {
    const Dim3& d = u->dims[l];
    const float* inp = u->feat;
    int cin = u->desc.in_channels;
    if (l > 0) {
      note_launch();
      k_avgpool<<<nb((int64_t)u->c[l - 1] * d.vox()), 256, 0, s>>>(u->e[l - 1], u->in[l], u->c[l - 1], d);
      inp = u->in[l];
      cin = u->c[l - 1];
    }
    conv3_fwd(u, enc_a(u, l), inp, cin, 0, nullptr, 0, u->a[l], d, tensor_cores);
    conv3_fwd(u, enc_a(u, l) + 1, u->a[l], u->c[l], 0, nullptr, 0, u->e[l], d, tensor_cores);
  }
  for (int l = L - 2; l >= 0; --l) {
    const Dim3& d = u->dims[l];
    const float* coarse = (l + 1 == L - 1) ? u->e[L - 1] : u->d[l + 1];
    conv3_fwd(u, dec_a(u, l), coarse, u->c[l + 1], 1, u->e[l], u->c[l], u->da[l], d, tensor_cores);
    conv3_fwd(u, dec_a(u, l) + 1, u->da[l], u->c[l], 0, nullptr, 0, u->d[l], d, tensor_cores);
  }
  const float* d0 = L > 1 ? u->d[0] : u->e[0];
  const auto& H = u->layers[head_i(u)];
  const auto& Hc = u->layers[chead_i(u)];
  note_launch();
  k_conv1<<<nb(u->dims[0].vox()), 256, 0, s>>>(d0, u->c[0], u->pb + H.w, u->pb + H.b, u->yh, u->dims[0].vox());
  note_launch();
  k_conv1<<<nb(u->dims[L - 1].vox()), 256, 0, s>>>(u->e[L - 1], u->c[L - 1], u->pb + Hc.w, u->pb + Hc.b, u->yc,
                                                   u->dims[L - 1].vox());
}

// backward from dt (node residuals) with scale gscale; accumulates into u->g
void backward(tobk_unet* u) {
  cudaStream_t s = u->stream;
  const int L = u->L;
  const Dim3& d0 = u->dims[0];
  note_launch();
  k_unet_nodes_bwd<<<nb(d0.vox()), 256, 0, s>>>(u->dt, u->gscale, u->out_scale, d0, u->gy);
  // heads
  const float* dtop = L > 1 ? u->d[0] : u->e[0];
  const auto& H = u->layers[head_i(u)];
  const auto& Hc = u->layers[chead_i(u)];
  note_launch();
  k_conv1_wgrad<<<u->c[0] + 1, 256, 0, s>>>(u->gy, dtop, u->c[0], u->g + H.w, u->g + H.b, d0.vox());
  float* gtop = L > 1 ? u->gd[0] : u->ge[0];
  note_launch();
  k_conv1_bwd_data<<<nb(d0.vox()), 256, 0, s>>>(u->gy, u->c[0], u->pb + H.w, gtop, d0.vox(), L > 1 ? 0 : 1);
  // coarse head: gyc = sum over the 8^(L-1) descendants
  {
    const float* src = u->gy;
    for (int l = 1; l < L; ++l) {
      float* dst = (l == L - 1) ? u->gyc : (l % 2 ? u->scratch2 : u->scratch);
      note_launch();
      k_sumpool<<<nb(3 * u->dims[l].vox()), 256, 0, s>>>(src, 0, dst, 3, u->dims[l], 0);
      src = dst;
    }
    if (L == 1) cudaMemcpyAsync(u->gyc, u->gy, sizeof(float) * 3 * d0.vox(), cudaMemcpyDeviceToDevice, s);
  }
  const Dim3& dL = u->dims[L - 1];
  note_launch();
  k_conv1_wgrad<<<u->c[L - 1] + 1, 256, 0, s>>>(u->gyc, u->e[L - 1], u->c[L - 1], u->g + Hc.w, u->g + Hc.b, dL.vox());
  note_launch();
  k_conv1_bwd_data<<<nb(dL.vox()), 256, 0, s>>>(u->gyc, u->c[L - 1], u->pb + Hc.w, u->ge[L - 1], dL.vox(), 1);
  // decoder, from the top: gd[l] = dL/dd_l (post-activation)
  for (int l = 0; l <= L - 2; ++l) {
    const Dim3& d = u->dims[l];
    const int lb = dec_a(u, l) + 1, la = dec_a(u, l);
    // dec l b: input da[l], output d[l]
    conv3_wgrad(u, lb, u->gd[l], u->d[l], u->da[l], u->c[l], 0, nullptr, 0, d);
    conv3_bwd_data(u, lb, u->gd[l], u->d[l], u->gtmp[l], d);  // dL/dda (pre-mask)
    // dec l a: input [up(coarse), e_l], output da[l]
    const float* coarse = (l + 1 == L - 1) ? u->e[L - 1] : u->d[l + 1];
    conv3_wgrad(u, la, u->gtmp[l], u->da[l], coarse, u->c[l + 1], 1, u->e[l], u->c[l], d);
    conv3_bwd_data(u, la, u->gtmp[l], u->da[l], u->scratch, d);  // [c_{l+1} + c_l][V_l]
    note_launch();
    k_add_channels<<<nb((int64_t)u->c[l] * d.vox()), 256, 0, s>>>(u->scratch, u->c[l + 1], u->ge[l],
                                                                  (int64_t)u->c[l] * d.vox(), d.vox());
    float* gcoarse = (l + 1 == L - 1) ? u->ge[L - 1] : u->gd[l + 1];
    note_launch();
    k_sumpool<<<nb((int64_t)u->c[l + 1] * u->dims[l + 1].vox()), 256, 0, s>>>(u->scratch, 0, gcoarse, u->c[l + 1],
                                                                              u->dims[l + 1], l + 1 == L - 1 ? 1 : 0);
  }
  // encoder from the bottleneck up
  for (int l = L - 1; l >= 0; --l) {
    const Dim3& d = u->dims[l];
    const int la = enc_a(u, l), lb = la + 1;
    const float* inp = l == 0 ? u->feat : u->in[l];
    const int cin = l == 0 ? u->desc.in_channels : u->c[l - 1];
    conv3_wgrad(u, lb, u->ge[l], u->e[l], u->a[l], u->c[l], 0, nullptr, 0, d);
    conv3_bwd_data(u, lb, u->ge[l], u->e[l], u->gtmp[l], d);
    conv3_wgrad(u, la, u->gtmp[l], u->a[l], inp, cin, 0, nullptr, 0, d);
    if (l > 0) {
      conv3_bwd_data(u, la, u->gtmp[l], u->a[l], u->scratch, d);  // dL/din_l [c_{l-1}][V_l]
      note_launch();
      k_avgpool_bwd<<<nb((int64_t)u->c[l - 1] * u->dims[l - 1].vox()), 256, 0, s>>>(u->scratch, u->ge[l - 1], u->c[l - 1],
                                                                                    u->dims[l - 1]);
    }
  }
}

void features(tobk_unet* u, const float* xf, const double* xd, const double* f) {
  const Dim3& d0 = u->dims[0];
  note_launch();
  k_unet_features<<<nb(d0.vox()), 256, 0, u->stream>>>(xf, xd, f, d0, u->desc.penal, u->desc.E0, u->desc.Emin, u->feat,
                                                       u->Ek);
  note_launch();
  k_unet_scale<<<1, 1024, 0, u->stream>>>(u->feat, u->Ek, d0.vox(), u->sc);
  note_launch();
  k_unet_scale_load<<<nb(3 * d0.vox()), 256, 0, u->stream>>>(u->feat, d0.vox(), u->sc);
}

// loss and gradient of one sample, accumulated (gradient into u->g, loss into u->lossd[0])
void sample_grad(tobk_unet* u, const float* x, const double* f, const float* target, const uint8_t* fixed) {
  features(u, x, nullptr, f);
  forward(u);
  for (int l = 0; l < u->L; ++l) {
    cudaMemsetAsync(u->ge[l], 0, sizeof(float) * u->c[l] * u->dims[l].vox(), u->stream);
  }
  const Dim3& d0 = u->dims[0];
  const int64_t nnode = (int64_t)(d0.D + 1) * (d0.H + 1) * (d0.W + 1);
  const int64_t n = 3 * nnode;
  note_launch();
  k_unet_nodes<<<nb(nnode), 256, 0, u->stream>>>(u->yh, u->yc, d0, u->L - 1, fixed, u->sc, u->out_scale, 1, nullptr,
                                                 u->tn);
  const int energy = u->desc.loss == TOBK_UNET_LOSS_ENERGY;
  if (energy) {  // K t with the library's factored H8 operator (FP32, moduli E_kappa of the features)
    const int nel[3] = {d0.W, d0.H, d0.D};
    launch_fine_h8<float>(make_grid(3, nel), u->Ek, fixed, u->desc.nu, 0, APPLY_KV, u->tn, nullptr, nullptr, u->Kt,
                          SmoothArgs<float>{}, 1, n, u->stream);
  }
  const unsigned blocks = nb(n);
  note_launch();
  k_unet_loss_partial<<<blocks, 256, 0, u->stream>>>(u->tn, u->Kt, target, f, fixed, u->sc, n, energy, u->dt,
                                                     u->partial);
  note_launch();
  k_unet_loss_final<<<1, 256, 0, u->stream>>>(u->partial, (int)blocks, u->sc, energy, u->lossd, u->gscale);
  backward(u);
}

// Carves every device buffer of the network out of the arena (sizing pass: base == nullptr);
// returns false when a buffer does not fit.
bool unet_layout(tobk_unet* u, Arena& a) {
  const int L = u->L;
  const Dim3& d0 = u->dims[0];
  const int64_t nnode = (int64_t)(d0.D + 1) * (d0.H + 1) * (d0.W + 1);
  size_t maxcat = (size_t)3 * d0.vox();
  for (int l = 0; l < L; ++l) {
    const size_t V = (size_t)u->dims[l].vox();
    const int cprev = l == 0 ? 4 : u->c[l - 1];
    maxcat = std::max(maxcat, (size_t)((l + 1 < L ? u->c[l + 1] : 0) + u->c[l] + cprev) * V);
  }
  std::vector<void*> got;
  auto take_f = [&a, &got](size_t n) {
    float* p = a.take<float>(n);
    got.push_back(p);
    return p;
  };
  u->p = take_f(u->np);
  u->g = take_f(u->np);
  u->m = take_f(u->np);
  u->v = take_f(u->np);
  u->pb = a.take<__nv_bfloat16>(u->np);
  got.push_back(u->pb);
  u->in.clear(), u->a.clear(), u->e.clear(), u->da.clear(), u->d.clear(), u->ge.clear(), u->gd.clear(), u->gtmp.clear();
  for (int l = 0; l < L; ++l) {
    const size_t V = (size_t)u->dims[l].vox();
    const int cprev = l == 0 ? 4 : u->c[l - 1];
    u->in.push_back(take_f(cprev * V));
    u->a.push_back(take_f(u->c[l] * V));
    u->e.push_back(take_f(u->c[l] * V));
    u->da.push_back(take_f(u->c[l] * V));
    u->d.push_back(take_f(u->c[l] * V));
    u->ge.push_back(take_f(u->c[l] * V));
    u->gd.push_back(take_f(u->c[l] * V));
    u->gtmp.push_back(take_f(u->c[l] * V));
  }
  u->feat = take_f(4 * d0.vox());
  u->Ek = take_f(d0.vox());
  u->yh = take_f(3 * d0.vox());
  u->gy = take_f(3 * d0.vox());
  u->yc = take_f(3 * u->dims[L - 1].vox());
  u->gyc = take_f(3 * u->dims[L - 1].vox());
  u->dt = take_f(3 * nnode);
  u->tn = take_f(3 * nnode);
  u->Kt = take_f(3 * nnode);
  u->scratch = take_f(maxcat);
  u->scratch2 = take_f(maxcat);
  float* scal = take_f(16);
  u->sc = scal;
  u->lossd = scal + 4;
  u->gscale = scal + 8;
  u->partial = a.take<double>(3 * ((3 * nnode + 255) / 256 + 1));
  got.push_back(u->partial);
  int64_t nwt = 0;
  u->wt_off.assign(u->layers.size(), -1);
  for (size_t li = 0; li < u->layers.size(); ++li) {
    const auto& ly = u->layers[li];
    if (ly.taps == 27 && tc_fits(ly.cout, ly.cin)) {
      u->wt_off[li] = nwt;
      nwt += (int64_t)27 * ly.cout * kpad(ly.cin);
    }
  }
  u->wt = a.take<__nv_bfloat16>(std::max<int64_t>(nwt, 8));
  got.push_back(u->wt);
  u->tc_err = a.take<unsigned>(4);
  got.push_back(u->tc_err);
  if (a.base == nullptr) return true;
  for (void* p : got)
    if (p == nullptr) return false;
  return true;
}

}  // namespace

extern "C" {

int tobk_unet_default_desc(tobk_unet_desc* d) {
  if (!d) return TOBK_E_ARG;
  std::memset(d, 0, sizeof(*d));
  d->nel[0] = 128;
  d->nel[1] = 64;
  d->nel[2] = 64;
  d->levels = 4;
  d->channels[0] = 16;
  d->channels[1] = 32;
  d->channels[2] = 64;
  d->channels[3] = 64;
  d->in_channels = 4;
  d->out_channels = 3;
  d->penal = 3.0;
  d->E0 = 1.0;
  d->Emin = 1e-6;
  d->nu = 0.3;
  d->loss = TOBK_UNET_LOSS_ENERGY;
  d->seed = 1234;
  return TOBK_OK;
}

int tobk_unet_create(const tobk_unet_desc* desc, void* cuda_stream, tobk_unet** out) {
  if (!desc || !out) return TOBK_E_ARG;
  *out = nullptr;
  const int L = desc->levels;
  if (L < 1 || L > 4 || desc->in_channels != 4 || desc->out_channels != 3) return TOBK_E_ARG;
  if (desc->loss != TOBK_UNET_LOSS_MSE && desc->loss != TOBK_UNET_LOSS_ENERGY) return TOBK_E_ARG;
  if (!(desc->nu > -1.0 && desc->nu < 0.5)) return TOBK_E_ARG;
  for (int a = 0; a < 3; ++a)
    if (desc->nel[a] < 1 || desc->nel[a] % (1 << (L - 1)) != 0) return TOBK_E_ARG;
  for (int l = 0; l < L; ++l)
    if (desc->channels[l] < 16 || desc->channels[l] % 16 != 0 || desc->channels[l] > 256) return TOBK_E_ARG;
  tobk_unet* u = new tobk_unet();
  u->desc = *desc;
  u->stream = (cudaStream_t)cuda_stream;
  u->L = L;
  u->c.assign(desc->channels, desc->channels + L);
  // parameter layout
  auto add = [u](int co, int ci, int taps) {
    tobk_unet::Layer ly{co, ci, taps, u->np, 0};
    u->np += (int64_t)co * ci * taps;
    ly.b = u->np;
    u->np += co;
    u->layers.push_back(ly);
  };
  int prev = desc->in_channels;
  for (int l = 0; l < L; ++l) {
    add(u->c[l], prev, 27);
    add(u->c[l], u->c[l], 27);
    prev = u->c[l];
  }
  for (int l = L - 2; l >= 0; --l) {
    add(u->c[l], u->c[l + 1] + u->c[l], 27);
    add(u->c[l], u->c[l], 27);
  }
  add(3, u->c[0], 1);
  add(3, u->c[L - 1], 1);
  for (int l = 0; l < L; ++l) u->dims.push_back({desc->nel[2] >> l, desc->nel[1] >> l, desc->nel[0] >> l});
  // memory: one arena, laid out by the same function for the sizing pass and the real pass
  Arena sizing;
  sizing.base = nullptr;
  sizing.cap = ~size_t(0) >> 1;
  unet_layout(u, sizing);
  const size_t bytes = sizing.used;
  if (cudaMalloc(&u->arena, bytes) != cudaSuccess || cudaMallocHost(&u->host, sizeof(float) * 16) != cudaSuccess) {
    cudaGetLastError();
    tobk_unet_destroy(u);
    return TOBK_E_NOMEM;
  }
  Arena a;
  a.base = u->arena;
  a.cap = bytes;
  if (!unet_layout(u, a)) {
    tobk_unet_destroy(u);
    return TOBK_E_NOMEM;
  }
  cudaMemsetAsync(u->arena, 0, bytes, u->stream);
  // He-normal initialisation of the weights (splitmix64 + Box-Muller), zero biases
  std::vector<float> hp(u->np, 0.f);
  uint64_t st = desc->seed;
  for (const auto& ly : u->layers) {
    const double sd = std::sqrt(2.0 / (double)(ly.cin * ly.taps));
    for (int64_t i = 0; i < (int64_t)ly.cout * ly.cin * ly.taps; i += 2) {
      const double u1 = ((double)(splitmix(st) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
      const double u2 = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      const double r = std::sqrt(-2.0 * std::log(u1));
      hp[ly.w + i] = (float)(sd * r * std::cos(6.283185307179586 * u2));
      if (i + 1 < (int64_t)ly.cout * ly.cin * ly.taps) hp[ly.w + i + 1] = (float)(sd * r * std::sin(6.283185307179586 * u2));
    }
  }
  // the output heads start small, so that the initial guess is close to zero
  for (int hi : {head_i(u), chead_i(u)})
    for (int64_t i = 0; i < (int64_t)u->layers[hi].cout * u->layers[hi].cin; ++i) hp[u->layers[hi].w + i] *= 0.01f;
  cudaMemcpyAsync(u->p, hp.data(), sizeof(float) * u->np, cudaMemcpyHostToDevice, u->stream);
  note_launch();
  k_to_bf16<<<nb(u->np), 256, 0, u->stream>>>(u->p, u->pb, u->np);
  cudaStreamSynchronize(u->stream);
  if (cudaGetLastError() != cudaSuccess) {
    tobk_unet_destroy(u);
    return TOBK_E_CUDA;
  }
  *out = u;
  return TOBK_OK;
}

void tobk_unet_destroy(tobk_unet* u) {
  if (!u) return;
  if (u->stream) cudaStreamSynchronize(u->stream);
  else cudaDeviceSynchronize();
  if (u->arena) cudaFree(u->arena);
  if (u->host) cudaFreeHost(u->host);
  delete u;
}

const char* tobk_unet_last_error(const tobk_unet* u) { return u ? u->err.c_str() : "null network"; }

int64_t tobk_unet_num_params(const tobk_unet* u) { return u ? u->np : -1; }

int tobk_unet_set_tensor_cores(tobk_unet* u, int mode) {
  if (!u || mode < 0 || mode > 2) return TOBK_E_ARG;
  u->tensor_cores = mode;
  return TOBK_OK;
}

int tobk_conv3_bf16(const float* in, int Cin, int D, int H, int W, const float* weight, const float* bias,
                    int Cout, int relu, float* out, void* cuda_stream) {
  if (!in || !weight || !out || Cin <= 0 || D <= 0 || H <= 0 || W <= 0 || !tc_fits(Cout, Cin)) return TOBK_E_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int Kp = kpad(Cin);
  const int64_t nw = (int64_t)Cout * Cin * 27, nwt = (int64_t)27 * Cout * Kp;
  void* buf = nullptr;
  const size_t bytes = sizeof(__nv_bfloat16) * (size_t)(nw + nwt + Cout + 8) + 64;
  if (cudaMallocAsync(&buf, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    return TOBK_E_NOMEM;
  }
  __nv_bfloat16* wb = (__nv_bfloat16*)buf;
  __nv_bfloat16* wt = wb + ((nw + 7) / 8) * 8;
  __nv_bfloat16* bb = wt + nwt;
  unsigned* err = (unsigned*)(((uintptr_t)(bb + Cout) + 15) & ~(uintptr_t)15);
  cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  note_launch();
  k_to_bf16<<<nb(nw), 256, 0, s>>>(weight, wb, nw);
  if (bias) {
    note_launch();
    k_to_bf16<<<nb(Cout), 256, 0, s>>>(bias, bb, Cout);
  }
  note_launch();
  k_tc_weights<<<nb(nwt), 256, 0, s>>>(wb, Cout, Cin, Kp, wt);
  const tc::ConvTcArgs a{in, nullptr, Cin, 0, nullptr, 0, wt, bias ? bb : nullptr, out, tc::Dim3{D, H, W}, Kp,
                         relu ? 1 : 0, err};
  switch (Cout) {
    case 16: launch_conv3_tc<16>(a, s); break;
    case 32: launch_conv3_tc<32>(a, s); break;
    case 64: launch_conv3_tc<64>(a, s); break;
    default: launch_conv3_tc<128>(a, s); break;
  }
  unsigned flag = 0;
  cudaMemcpyAsync(&flag, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(buf, s);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return TOBK_E_CUDA;
  return flag ? TOBK_E_TIMEOUT : TOBK_OK;
}

int tobk_unet_set_output_scale(tobk_unet* u, double scale) {
  if (!u || !(scale > 0.0) || !std::isfinite(scale)) return TOBK_E_ARG;
  u->out_scale = (float)scale;
  return TOBK_OK;
}

double tobk_unet_output_scale(const tobk_unet* u) { return u ? (double)u->out_scale : 0.0; }

int tobk_unet_design_scale(tobk_unet* u, const float* x, const double* f, double* s) {
  if (!u || !x || !f || !s) return TOBK_E_ARG;
  features(u, x, nullptr, f);
  cudaMemcpyAsync(u->host, u->sc, sizeof(float) * 2, cudaMemcpyDeviceToHost, u->stream);
  cudaStreamSynchronize(u->stream);
  *s = (double)u->host[1];
  return cudaGetLastError() == cudaSuccess ? TOBK_OK : ufail(u, TOBK_E_CUDA, "design_scale");
}

int tobk_unet_get_state(tobk_unet* u, float* params, float* adam_m, float* adam_v, long long* step, int on_device) {
  if (!u) return TOBK_E_ARG;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (params) cudaMemcpyAsync(params, u->p, sizeof(float) * u->np, k, u->stream);
  if (adam_m) cudaMemcpyAsync(adam_m, u->m, sizeof(float) * u->np, k, u->stream);
  if (adam_v) cudaMemcpyAsync(adam_v, u->v, sizeof(float) * u->np, k, u->stream);
  if (step) *step = u->step;
  cudaStreamSynchronize(u->stream);
  return cudaGetLastError() == cudaSuccess ? TOBK_OK : ufail(u, TOBK_E_CUDA, "get_state");
}

int tobk_unet_set_state(tobk_unet* u, const float* params, const float* adam_m, const float* adam_v, long long step,
                        int on_device) {
  if (!u || !params) return TOBK_E_ARG;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaMemcpyAsync(u->p, params, sizeof(float) * u->np, k, u->stream);
  if (adam_m) cudaMemcpyAsync(u->m, adam_m, sizeof(float) * u->np, k, u->stream);
  else cudaMemsetAsync(u->m, 0, sizeof(float) * u->np, u->stream);
  if (adam_v) cudaMemcpyAsync(u->v, adam_v, sizeof(float) * u->np, k, u->stream);
  else cudaMemsetAsync(u->v, 0, sizeof(float) * u->np, u->stream);
  u->step = step;
  note_launch();
  k_to_bf16<<<nb(u->np), 256, 0, u->stream>>>(u->p, u->pb, u->np);
  cudaStreamSynchronize(u->stream);
  return cudaGetLastError() == cudaSuccess ? TOBK_OK : ufail(u, TOBK_E_CUDA, "set_state");
}

int tobk_unet_predict(tobk_unet* u, const double* x, const double* f, const uint8_t* fixed, double* u0) {
  if (!u || !x || !f || !fixed || !u0) return TOBK_E_ARG;
  features(u, nullptr, x, f);
  forward(u, u->tensor_cores != 0);
  if (u->tensor_cores) {
    unsigned flag = 0;
    cudaMemcpyAsync(u->host, u->tc_err, sizeof(unsigned), cudaMemcpyDeviceToHost, u->stream);
    cudaStreamSynchronize(u->stream);
    std::memcpy(&flag, u->host, sizeof(unsigned));
    if (flag) {
      cudaMemsetAsync(u->tc_err, 0, sizeof(unsigned), u->stream);
      return ufail(u, TOBK_E_TIMEOUT, "predict: a tensor-core wait gave up");
    }
  }
  const Dim3& d0 = u->dims[0];
  const int64_t nnode = (int64_t)(d0.D + 1) * (d0.H + 1) * (d0.W + 1);
  note_launch();
  k_unet_nodes<<<nb(nnode), 256, 0, u->stream>>>(u->yh, u->yc, d0, u->L - 1, fixed, u->sc, u->out_scale, 0, u0,
                                                 nullptr);
  if (cudaGetLastError() != cudaSuccess) return ufail(u, TOBK_E_CUDA, "predict: launch failed");
  return TOBK_OK;
}

int tobk_unet_loss_grad(tobk_unet* u, const float* x, const double* f, const float* target, const uint8_t* fixed,
                        float* loss, float* grad) {
  if (!u || !x || !f || !target || !fixed) return TOBK_E_ARG;
  cudaMemsetAsync(u->g, 0, sizeof(float) * u->np, u->stream);
  cudaMemsetAsync(u->lossd, 0, sizeof(float), u->stream);
  sample_grad(u, x, f, target, fixed);
  if (grad) cudaMemcpyAsync(grad, u->g, sizeof(float) * u->np, cudaMemcpyDeviceToDevice, u->stream);
  cudaMemcpyAsync(u->host, u->lossd, sizeof(float), cudaMemcpyDeviceToHost, u->stream);
  cudaStreamSynchronize(u->stream);
  if (loss) *loss = u->host[0];
  return cudaGetLastError() == cudaSuccess ? TOBK_OK : ufail(u, TOBK_E_CUDA, "loss_grad");
}

int tobk_unet_train_step(tobk_unet* u, const float* x, const double* f, const float* target, const uint8_t* fixed,
                         int nbatch, float lr, float* loss) {
  if (!u || !x || !f || !target || !fixed || nbatch < 1 || !(lr > 0.f)) return TOBK_E_ARG;
  const Dim3& d0 = u->dims[0];
  const int64_t m = d0.vox(), n = 3 * (int64_t)(d0.D + 1) * (d0.H + 1) * (d0.W + 1);
  cudaMemsetAsync(u->g, 0, sizeof(float) * u->np, u->stream);
  cudaMemsetAsync(u->lossd, 0, sizeof(float), u->stream);
  for (int b = 0; b < nbatch; ++b) sample_grad(u, x + b * m, f, target + b * n, fixed);
  u->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)u->step), c2 = 1.f - std::pow(b2, (float)u->step);
  note_launch();
  k_adam<<<nb(u->np), 256, 0, u->stream>>>(u->p, u->g, u->m, u->v, u->pb, u->np, lr, b1, b2, 1e-8f, c1, c2,
                                           1.f / (float)nbatch);
  cudaMemcpyAsync(u->host, u->lossd, sizeof(float), cudaMemcpyDeviceToHost, u->stream);
  cudaStreamSynchronize(u->stream);
  if (loss) *loss = u->host[0] / (float)nbatch;
  return cudaGetLastError() == cudaSuccess ? TOBK_OK : ufail(u, TOBK_E_CUDA, "train_step");
}

}  // extern "C"
