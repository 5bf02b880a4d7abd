// Not part of the paper's method: the learned warm start's network (mgPCG still runs to the same
// tolerance from its guess).
//
// Tensor-core (tcgen05) 3x3x3 convolution for the learned warm start's inference: an implicit GEMM
// out[v][co] = bias[co] + sum_tap sum_ci A_tap[v][ci] W_tap[co][ci] with M = 128 voxels per CTA,
// N = Cout, K = Cin per tap (padded to a multiple of 16), BF16 operands (the activations are rounded
// to bfloat16 as they are staged) and FP32 accumulation in tensor memory.
//
// Per CTA (128 threads, thread t owns voxel row t): TMEM holds the 128 x N FP32 accumulator.  For
// each of the 27 taps the threads gather the shifted activations (zero outside the grid; the
// first C1 channels optionally read at half resolution, i.e. nearest 2x upsampling, and masked)
// and the tap's weights into shared memory in the canonical K-major layout without swizzle
// (8-row x 16-byte core matrices; rows 16 bytes apart, the 8-channel column blocks `rows x 16`
// bytes apart), then one thread issues Cin/16 tcgen05.mma (M = 128, N, K = 16) and commits them to
// an mbarrier that every thread waits on before the tiles are overwritten.  The epilogue reads the
// accumulator with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31), adds the bias, applies ReLU
// and stores FP32 [Cout][V].  Every mbarrier wait is bounded; a wait that gives up sets *err and the
// CTA skips its epilogue and frees its tensor memory.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "tcgen05_common.cuh"

namespace tobk {
namespace tc {

struct Dim3 {
  int D, H, W;
  __host__ __device__ int64_t vox() const { return (int64_t)D * H * W; }
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

struct ConvTcArgs {
  const float* in1;
  const float* mask1;
  int C1, up1;
  const float* in2;
  int C2;
  const __nv_bfloat16* Wt;    // [27][N][Kp]
  const __nv_bfloat16* bias;  // [N] or null
  float* out;                 // [N][V]
  Dim3 d;
  int Kp;                     // input channels padded to a multiple of 16
  int relu;
  unsigned* err;              // set to 1 when a wait gave up
};

template <int N>
__global__ void __launch_bounds__(128) k_conv3_tc(ConvTcArgs a) {
  static_assert(N == 16 || N == 32 || N == 64 || N == 128, "output channels");
  constexpr int NCOL = N < 32 ? 32 : N;  // TMEM columns (a power of two >= 32)
  constexpr uint32_t IDESC = idesc_bf16(N);
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;                          // [Kp/8][128 rows][16 B]
  uint8_t* sB = smem + (size_t)(a.Kp / 8) * 2048;  // [Kp/8][N rows][16 B]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_s;
  const int t = threadIdx.x, warp = t >> 5;
  const int64_t V = a.d.vox();
  const int64_t vrow = (int64_t)blockIdx.x * 128 + t;  // this thread's A row / output voxel
  const bool vin = vrow < V;
  const int x = vin ? (int)(vrow % a.d.W) : 0;
  const int y = vin ? (int)((vrow / a.d.W) % a.d.H) : 0;
  const int z = vin ? (int)(vrow / ((int64_t)a.d.W * a.d.H)) : 0;
  const Dim3 dc{a.d.D / 2, a.d.H / 2, a.d.W / 2};
  const int Cin = a.C1 + a.C2;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;
  const uint32_t mb = smem_u32(&mbar);
  uint32_t phase = 0;
  bool ok = true;
  for (int tap = 0; tap < 27 && ok; ++tap) {
    const int xx = x + tap % 3 - 1, yy = y + (tap / 3) % 3 - 1, zz = z + tap / 9 - 1;
    const bool in = vin && xx >= 0 && xx < a.d.W && yy >= 0 && yy < a.d.H && zz >= 0 && zz < a.d.D;
    int64_t i1 = 0, i2 = 0;
    if (in) {
      i2 = ((int64_t)zz * a.d.H + yy) * a.d.W + xx;
      i1 = a.up1 ? ((int64_t)(zz >> 1) * dc.H + (yy >> 1)) * dc.W + (xx >> 1) : i2;
    }
    const int64_t V1 = a.up1 ? dc.vox() : V;
    for (int k8 = 0; k8 < a.Kp / 8; ++k8) {
      uint32_t pk[4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        float f[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = k8 * 8 + e + h;
          float v = 0.f;
          if (in && c < Cin) {
            if (c < a.C1) {
              v = a.in1[(int64_t)c * V1 + i1];
              if (a.mask1 && !(a.mask1[(int64_t)c * V1 + i1] > 0.f)) v = 0.f;
            } else {
              v = a.in2[(int64_t)(c - a.C1) * V + i2];
            }
          }
          f[h] = v;
        }
        pk[e / 2] = pack_bf16(f[0], f[1]);
      }
      *reinterpret_cast<uint4*>(sA + (size_t)k8 * 2048 + (size_t)t * 16) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    const int nchunk = N * (a.Kp / 8);
    for (int q = t; q < nchunk; q += 128) {
      const int n = q % N, k8 = q / N;
      const uint4 w = *reinterpret_cast<const uint4*>(a.Wt + ((size_t)tap * N + n) * a.Kp + k8 * 8);
      *reinterpret_cast<uint4*>(sB + (size_t)k8 * (N * 16) + (size_t)n * 16) = w;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int j = 0; j < a.Kp / 16; ++j) {
        const uint64_t ad = smem_desc(smem_u32(sA + (size_t)(2 * j) * 2048), 2048, 128);
        const uint64_t bd = smem_desc(smem_u32(sB + (size_t)(2 * j) * (N * 16)), N * 16, 128);
        const uint32_t acc = (tap > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    // the MMAs read sA / sB asynchronously: wait for them before the next tap overwrites the tiles
    const bool w = mbar_wait(mb, phase);
    if (!w) {
      if (t == 0) atomicExch(a.err, 1u);
      mbar_wait(mb, phase);  // one more bounded wait for the operations in flight
    }
    ok = __syncthreads_and(w) != 0;  // the same decision in every thread
    phase ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + lane_base + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (vin) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float v = __uint_as_float(r[i]) + (a.bias ? __bfloat162float(a.bias[c0 + i]) : 0.f);
          if (a.relu) v = fmaxf(v, 0.f);
          a.out[(int64_t)(c0 + i) * V + vrow] = v;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
}

inline size_t conv3_tc_smem(int N, int Kp) { return (size_t)(Kp / 8) * 2048 + (size_t)(Kp / 8) * N * 16; }

// Row variant for grids whose x extent W is a multiple of 128: a CTA's 128 voxels are 128
// consecutive x of one (y, z) line, so the activations of all 27 taps are rows of one halo slab
// (3 planes x 3 lines x 130 x, zero outside the grid) staged once in the canonical layout, and the
// A operand of tap (dz, dy, dx) is the slab seen from row ((dz + 1) 3 + dy + 1) 130 + dx + 1: a
// descriptor offset, no copy.  The weights of all taps are staged once as well, and one thread
// issues the 27 Kp / 16 MMAs back to back with a single commit.
constexpr int kSlabRows = 9 * 130;

__host__ __device__ inline size_t conv3_tc_row_smem(int N, int Kp) {
  return (size_t)(Kp / 8) * kSlabRows * 16 + (size_t)27 * (Kp / 8) * N * 16;
}

template <int N>
__global__ void __launch_bounds__(128) k_conv3_tc_row(ConvTcArgs a) {
  static_assert(N == 16 || N == 32 || N == 64 || N == 128, "output channels");
  constexpr int NCOL = N < 32 ? 32 : N;
  constexpr uint32_t IDESC = idesc_bf16(N);
  extern __shared__ __align__(128) uint8_t smem[];
  const int K8 = a.Kp / 8;
  uint8_t* sS = smem;                                   // slab [K8][9 lines][130 x][16 B]
  uint8_t* sB = smem + (size_t)K8 * kSlabRows * 16;     // weights [27][K8][N rows][16 B]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_s;
  const int t = threadIdx.x, warp = t >> 5;
  const int64_t V = a.d.vox();
  const int tiles_x = a.d.W / 128;
  const int64_t line = blockIdx.x / tiles_x;  // (z, y) line index
  const int x0 = (int)(blockIdx.x % tiles_x) * 128;
  const int y = (int)(line % a.d.H), z = (int)(line / a.d.H);
  const Dim3 dc{a.d.D / 2, a.d.H / 2, a.d.W / 2};
  const int Cin = a.C1 + a.C2;
  const int64_t V1 = a.up1 ? dc.vox() : V;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // slab: row s = (l * 130 + xi), l = 3 (dz + 1) + (dy + 1), x = x0 + xi - 1.  Work item = (8-channel
  // block k8, line l, group g): g < 32 stages the 4 interior rows xi = 1 + 4g .. 4 + 4g from one
  // float4 (float2 when upsampled) per channel, g = 32 and 33 the edge rows xi = 0 and 129.
  for (int q = t; q < K8 * 9 * 34; q += 128) {
    const int g = q % 34, l = (q / 34) % 9, k8 = q / (34 * 9);
    const int yy = y + l % 3 - 1, zz = z + l / 3 - 1;
    const bool line_in = yy >= 0 && yy < a.d.H && zz >= 0 && zz < a.d.D;
    const int64_t base2 = ((int64_t)zz * a.d.H + yy) * a.d.W;                 // full-resolution line
    const int64_t base1 = a.up1 ? ((int64_t)(zz >> 1) * dc.H + (yy >> 1)) * dc.W : base2;
    if (g < 32) {
      const int xx = x0 + 4 * g;  // 4 interior voxels, all inside the line
      float f[4][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = k8 * 8 + e;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (line_in && c < Cin) {
          if (c < a.C1) {
            if (a.up1) {
              const float2 h = __ldg(reinterpret_cast<const float2*>(a.in1 + (int64_t)c * V1 + base1 + (xx >> 1)));
              v = make_float4(h.x, h.x, h.y, h.y);
              if (a.mask1) {
                const float2 m = __ldg(reinterpret_cast<const float2*>(a.mask1 + (int64_t)c * V1 + base1 + (xx >> 1)));
                if (!(m.x > 0.f)) v.x = v.y = 0.f;
                if (!(m.y > 0.f)) v.z = v.w = 0.f;
              }
            } else {
              v = __ldg(reinterpret_cast<const float4*>(a.in1 + (int64_t)c * V1 + base1 + xx));
              if (a.mask1) {
                const float4 m = __ldg(reinterpret_cast<const float4*>(a.mask1 + (int64_t)c * V1 + base1 + xx));
                if (!(m.x > 0.f)) v.x = 0.f;
                if (!(m.y > 0.f)) v.y = 0.f;
                if (!(m.z > 0.f)) v.z = 0.f;
                if (!(m.w > 0.f)) v.w = 0.f;
              }
            }
          } else {
            v = __ldg(reinterpret_cast<const float4*>(a.in2 + (int64_t)(c - a.C1) * V + base2 + xx));
          }
        }
        f[0][e] = v.x, f[1][e] = v.y, f[2][e] = v.z, f[3][e] = v.w;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        *reinterpret_cast<uint4*>(sS + ((size_t)k8 * kSlabRows + l * 130 + 1 + 4 * g + i) * 16) =
            make_uint4(pack_bf16(f[i][0], f[i][1]), pack_bf16(f[i][2], f[i][3]), pack_bf16(f[i][4], f[i][5]),
                       pack_bf16(f[i][6], f[i][7]));
    } else {
      const int xi = g == 32 ? 0 : 129, xx = x0 + xi - 1;
      const bool in = line_in && xx >= 0 && xx < a.d.W;
      float f[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = k8 * 8 + e;
        float v = 0.f;
        if (in && c < Cin) {
          if (c < a.C1) {
            const int64_t i1 = base1 + (a.up1 ? (xx >> 1) : xx);
            v = __ldg(a.in1 + (int64_t)c * V1 + i1);
            if (a.mask1 && !(__ldg(a.mask1 + (int64_t)c * V1 + i1) > 0.f)) v = 0.f;
          } else {
            v = __ldg(a.in2 + (int64_t)(c - a.C1) * V + base2 + xx);
          }
        }
        f[e] = v;
      }
      *reinterpret_cast<uint4*>(sS + ((size_t)k8 * kSlabRows + l * 130 + xi) * 16) =
          make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]));
    }
  }
  for (int q = t; q < 27 * K8 * N; q += 128) {
    const int n = q % N, k8 = (q / N) % K8, tap = q / (N * K8);
    const uint4 w = *reinterpret_cast<const uint4*>(a.Wt + ((size_t)tap * N + n) * a.Kp + k8 * 8);
    *reinterpret_cast<uint4*>(sB + (((size_t)tap * K8 + k8) * N + n) * 16) = w;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;
  const uint32_t mb = smem_u32(&mbar);
  if (t == 0) {
    const uint32_t lbo_a = kSlabRows * 16, lbo_b = N * 16;
    for (int tap = 0; tap < 27; ++tap) {
      const int row0 = ((tap / 9) * 3 + (tap / 3) % 3) * 130 + tap % 3;
      for (int j = 0; j < a.Kp / 16; ++j) {
        const uint64_t ad = smem_desc(smem_u32(sS + ((size_t)(2 * j) * kSlabRows + row0) * 16), lbo_a, 128);
        const uint64_t bd = smem_desc(smem_u32(sB + ((size_t)tap * K8 + 2 * j) * (N * 16)), lbo_b, 128);
        const uint32_t acc = (tap > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
            : "memory");
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                 : "memory");
  }
  const bool w = mbar_wait(mb, 0);
  if (!w) {
    if (t == 0) atomicExch(a.err, 1u);
    mbar_wait(mb, 0);  // one more bounded wait for the operations in flight
  }
  const bool ok = __syncthreads_and(w) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    const int64_t vrow = (line * a.d.W) + x0 + t;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
          "%14, %15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + lane_base + (uint32_t)c0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float v = __uint_as_float(r[i]) + (a.bias ? __bfloat162float(a.bias[c0 + i]) : 0.f);
        if (a.relu) v = fmaxf(v, 0.f);
        a.out[(int64_t)(c0 + i) * V + vrow] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
}

}  // namespace tc
}  // namespace tobk
