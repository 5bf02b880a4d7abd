// FP64-accurate Gram products on the tensor cores, for the block products of the coarse
// eigensolver (eq. eigenvalueProblemCoarseScale; Appendix A asks for a residual of 1e-8, so these
// products must keep FP64 accuracy):
//     C[i][j] = sum_k A_i[k] B_j[k],   na <= 64 vectors A_i, nb <= 64 vectors B_j of length n.
//
// Error-free splitting in the manner of Ozaki, Ogita, Oishi and Rump ("Error-free transformations
// of matrix multiplication by using fast routines of matrix multiplication and its applications",
// Numer. Algorithms 59, 2012), arranged for BF16 tcgen05 MMAs with FP32 accumulators.  The vectors
// are cut into chunks of 128 entries, one chunk per CTA:
//   * every row of the chunk is scaled by a power of two 2^E (E from the row's largest entry in the
//     chunk, |entries| < 2^E) and every entry is written as a 56-bit fixed-point number
//     q = |x| 2^(56 - E) (truncated below 2^-56 of that largest entry), read straight from its IEEE
//     bits with integer arithmetic;
//   * q is cut into S = 8 digits of 7 bits, d_t = (q >> (49 - 7 t)) & 127, so x = 2^E sign(x)
//     sum_t d_t 2^(-7(t+1)); each digit is an integer of magnitude <= 127, exact in BF16;
//   * for every pair of digit planes (t, u) with t + u = L <= S - 1 the MMAs accumulate sum_k d_t d_u
//     over the chunk into the level-L accumulator (FP32 in tensor memory).  A product is below 2^14
//     and a level (at most 8 pairs) of a chunk at most 8 * 127^2 * 128 < 2^24: every accumulator holds
//     an exact integer;
//   * the chunk's contribution 2^(E_i + F_j) sum_L 2^(-7(L+2)) S_L[i][j] is formed in FP64 and the
//     chunks are added by the FP64 reduction of the CUDA-core Gram product (fixed order).
// Pairs with t + u >= S are dropped: with the input truncation this bounds the error of a chunk's
// product by about 128 2^-55 max|A_i| max|B_j| over the chunk.
//
// GB300 issues two FP64 instructions per clock per SM, so the splitting is integer work, the products
// are exact tensor-core work, and FP64 is used only to combine the eight level sums per output.
//
// Per CTA (256 threads, two tiles of 64 entries): every thread loads its entries of both tiles first;
// the warps reduce the rows' largest entries; shared memory holds the 8 digit planes of the A tile
// (128 rows, rows >= na zero) and of the B tile (N rows, rows >= nb zero) in the canonical K-major
// layout without swizzle; per tile thread 0 issues the 36 x 4 MMAs (M = 128, N, K = 16) and commits
// them to an mbarrier that every thread waits on before the next tile is staged; the 8 level
// accumulators occupy 8 N TMEM columns, read back with tcgen05.ld by the warps of the four lane
// quadrants, each quadrant's columns split over two warps.  The mbarrier waits are bounded: a wait
// that gives up sets err[0], skips the epilogue and frees the tensor memory.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "kernels.h"
#include "tcgen05_common.cuh"

namespace tobk {

constexpr int kTcSlices = 8;
constexpr int kTcTile = 64;     // entries per shared-memory tile
constexpr int kTcSub = 2;       // tiles per chunk: a level then stays below 8 * 127^2 * 128 < 2^24
constexpr int kTcThreads = 256;
constexpr int kTcPairs = 64 * (kTcTile / 2) / kTcThreads;  // entry pairs per thread and tile (64 rows)

// E with |x| < 2^E for every entry of a row whose largest magnitude has the bits m (0 for a zero row;
// a NaN / infinity has exponent field 0x7FF and sets err[1])
__device__ __forceinline__ int exponent_of(unsigned long long m, unsigned* err) {
  const int ex = (int)(m >> 52);
  if (ex == 0x7FF) {
    atomicExch(err + 1, 1u);
    return 0;
  }
  // normal x: 2^(ex-1023) <= |x| < 2^(ex-1022); subnormal: |x| < 2^-1022
  return m == 0 ? 0 : (ex == 0 ? -1022 : ex - 1022);
}

__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// the 56-bit fixed-point magnitude of x relative to 2^E and its sign
__device__ __forceinline__ unsigned long long fixed56(double x, int E, bool& neg) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  neg = (u >> 63) != 0;
  int ex = (int)((u >> 52) & 0x7FF);
  unsigned long long man = u & 0xFFFFFFFFFFFFFull;
  if (ex == 0x7FF) return 0;  // non-finite (reported by exponent_of)
  if (ex) man |= 1ull << 52;
  else ex = 1;
  const int s = ex - 1019 - E;  // |x| 2^(56-E) = man 2^(ex - 1075 + 56 - E)
  if (s >= 0) return s < 8 ? man << s : 0;
  return s > -64 ? man >> (-s) : 0;
}

// digit planes of x[k], x[k+1] of one row into the K-major tile (row stride 16 B, 8-column blocks
// `block` bytes apart, planes `plane` bytes apart)
__device__ __forceinline__ void store_digits(uint8_t* tile, int row, int k, double x0, double x1, int E, int block,
                                             int plane) {
  bool n0, n1;
  const unsigned long long q0 = fixed56(x0, E, n0), q1 = fixed56(x1, E, n1);
  uint8_t* p = tile + (size_t)(k >> 3) * block + (size_t)row * 16 + (k & 7) * 2;
#pragma unroll
  for (int t = 0; t < kTcSlices; ++t) {
    const int d0 = (int)((q0 >> (49 - 7 * t)) & 127), d1 = (int)((q1 >> (49 - 7 * t)) & 127);
    const __nv_bfloat162 h = __floats2bfloat162_rn((float)(n0 ? -d0 : d0), (float)(n1 ? -d1 : d1));
    *reinterpret_cast<__nv_bfloat162*>(p + (size_t)t * plane) = h;
  }
}

// partial [chunk][na][nb] (FP64) = the chunk's contribution to A B^T
template <int N>
__global__ void __launch_bounds__(kTcThreads) k_gram_tc(const double* __restrict__ A, int na,
                                                        const double* __restrict__ B, int nb, int64_t n,
                                                        int64_t stride, double* __restrict__ partial,
                                                        unsigned* __restrict__ err) {
  static_assert(N == 32 || N == 64, "B tile rows");
  constexpr int NCOL = kTcSlices * N;  // 256 or 512 TMEM columns: one N-wide accumulator per level
  constexpr uint32_t IDESC = tc::idesc_bf16(N);
  constexpr int KB = kTcTile / 8;      // 8-column blocks per tile
  constexpr int ABLK = 128 * 16, BBLK = N * 16;
  constexpr int APLANE = KB * ABLK, BPLANE = KB * BBLK;
  extern __shared__ __align__(128) uint8_t smem[];
  uint8_t* sA = smem;                               // [S][KB][128 rows][16 B]
  uint8_t* sB = smem + (size_t)kTcSlices * APLANE;  // [S][KB][N rows][16 B]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_s;
  __shared__ int Es[128];  // chunk exponents of the A rows [0, 64) and of the B rows [64, 128)
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int64_t c0k = (int64_t)blockIdx.x * kTcSub * kTcTile;
  // this thread's entries: tile s, pair i -> row warp + 8 i, entries 2 lane and 2 lane + 1
  double xa[kTcSub][kTcPairs][2], xb[kTcSub][kTcPairs][2];
#pragma unroll
  for (int s = 0; s < kTcSub; ++s)
#pragma unroll
    for (int i = 0; i < kTcPairs; ++i) {
      const int row = warp + 8 * i;
      const int64_t g = c0k + s * kTcTile + 2 * lane;
      const double* a = A + (int64_t)row * stride;
      const double* b = B + (int64_t)row * stride;
      xa[s][i][0] = (row < na && g < n) ? a[g] : 0.0;
      xa[s][i][1] = (row < na && g + 1 < n) ? a[g + 1] : 0.0;
      xb[s][i][0] = (row < nb && g < n) ? b[g] : 0.0;
      xb[s][i][1] = (row < nb && g + 1 < n) ? b[g + 1] : 0.0;
    }
  // zero the padding rows (A rows >= na, B rows >= nb): the MMAs read them as zero
  for (int q = t; q < kTcSlices * KB * (128 - na); q += kTcThreads) {
    const int r = na + q % (128 - na), blk = q / (128 - na);
    *reinterpret_cast<uint4*>(sA + (size_t)blk * ABLK + (size_t)r * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int q = t; q < kTcSlices * KB * (N - nb); q += kTcThreads) {
    const int r = nb + q % (N - nb), blk = q / (N - nb);
    *reinterpret_cast<uint4*>(sB + (size_t)blk * BBLK + (size_t)r * 16) = make_uint4(0u, 0u, 0u, 0u);
  }
  // largest magnitude of every row over the chunk (the 32 lanes of a warp hold one row)
#pragma unroll
  for (int i = 0; i < kTcPairs; ++i) {
    unsigned long long ma = 0, mbv = 0;
#pragma unroll
    for (int s = 0; s < kTcSub; ++s) {
      ma = max(ma, max(mag_bits(xa[s][i][0]), mag_bits(xa[s][i][1])));
      mbv = max(mbv, max(mag_bits(xb[s][i][0]), mag_bits(xb[s][i][1])));
    }
    for (int o = 16; o > 0; o >>= 1) {
      ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
      mbv = max(mbv, __shfl_xor_sync(0xffffffffu, mbv, o));
    }
    if (lane == 0) {
      Es[warp + 8 * i] = exponent_of(ma, err);
      Es[64 + warp + 8 * i] = exponent_of(mbv, err);
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_s)),
                 "r"(NCOL)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_u32(&mbar)), "r"(1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_s;
  const uint32_t mb = tc::smem_u32(&mbar);
  uint32_t phase = 0;
  bool ok = true;
  for (int s = 0; s < kTcSub && ok; ++s) {
#pragma unroll
    for (int i = 0; i < kTcPairs; ++i) {
      const int row = warp + 8 * i;
      if (row < na) store_digits(sA, row, 2 * lane, xa[s][i][0], xa[s][i][1], Es[row], ABLK, APLANE);
      if (row < nb) store_digits(sB, row, 2 * lane, xb[s][i][0], xb[s][i][1], Es[64 + row], BBLK, BPLANE);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int L = 0; L < kTcSlices; ++L)
        for (int ta = 0; ta <= L; ++ta) {
          const int tb = L - ta;
          for (int kk = 0; kk < kTcTile / 16; ++kk) {
            const uint64_t ad =
                tc::smem_desc(tc::smem_u32(sA + (size_t)ta * APLANE + (size_t)(2 * kk) * ABLK), ABLK, 128);
            const uint64_t bd =
                tc::smem_desc(tc::smem_u32(sB + (size_t)tb * BPLANE + (size_t)(2 * kk) * BBLK), BBLK, 128);
            const uint32_t acc = (s > 0 || ta > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + (uint32_t)(L * N)),
                "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
                : "memory");
          }
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                   : "memory");
    }
    // the MMAs read the planes asynchronously: wait before the next tile overwrites them
    const bool done = tc::mbar_wait(mb, phase);
    if (!done) {
      if (t == 0) atomicExch(err, 1u);
      tc::mbar_wait(mb, phase);  // one more bounded wait for the operations in flight
    }
    ok = __syncthreads_and(done) != 0;
    phase ^= 1u;
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // epilogue: warp w reads lane quadrant w % 4 (A rows 32 (w % 4) ...) and half w / 4 of the columns
  const int quad = warp & 3, half = warp >> 2;
  if (ok && quad * 32 < na) {
    const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
    const int row = quad * 32 + lane;
    for (int c0 = half * (N / 2); c0 < (half + 1) * (N / 2); c0 += 16) {
      double acc[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) acc[i] = 0.0;
      for (int L = kTcSlices - 1; L >= 0; --L) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + lane_base + (uint32_t)(L * N + c0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const double w = ldexp(1.0, -7 * (L + 2));
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[i] += w * (double)__uint_as_float(r[i]);
      }
      if (row < na) {
        double* out = partial + ((size_t)blockIdx.x * na + row) * nb;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (c0 + i < nb) out[c0 + i] = ldexp(acc[i], Es[row] + Es[64 + c0 + i]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOL) : "memory");
}

int gram_tc_chunks(int64_t n) { return (int)((n + (int64_t)kTcTile * kTcSub - 1) / ((int64_t)kTcTile * kTcSub)); }

template <int N>
static void launch_gram_tc_n(const double* A, int na, const double* B, int nb, int64_t n, int64_t stride,
                             double* partial, unsigned* err, cudaStream_t s) {
  constexpr size_t smem = (size_t)kTcSlices * (kTcTile / 8) * (128 + N) * 16;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(k_gram_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  note_launch();
  k_gram_tc<N><<<(unsigned)gram_tc_chunks(n), kTcThreads, smem, s>>>(A, na, B, nb, n, stride, partial, err);
}

void launch_gram_tc(const double* A, int na, const double* B, int nb, int64_t n, int64_t stride, double* C,
                    double* partial, unsigned* err, cudaStream_t s) {
  if (nb <= 32)
    launch_gram_tc_n<32>(A, na, B, nb, n, stride, partial, err, s);
  else
    launch_gram_tc_n<64>(A, na, B, nb, n, stride, partial, err, s);
  launch_gram_final(partial, gram_tc_chunks(n), na * nb, C, s);
}

}  // namespace tobk
