// Allocation-free residual check on the fine grid (declared as tobk_residual_noalloc in
// include/tobk.h): the relative residual ||b - K(x) x|| / ||b|| of the linear analysis (Algorithm 1
// step 3; the stopping quantity of the mgPCG solves, Appendix A).
//
// Some callers cannot allocate device memory at the point where they want to verify a solution:
// code running while a CUDA stream is being captured into a graph (cudaMalloc is not a legal
// operation there), applications whose device memory is owned by another framework's pool allocator
// and may not be grown behind its back, and latency-critical loops where cudaMalloc's implicit
// device synchronisation is not acceptable.  This entry point needs no handle and no allocation: it
// recomputes ||b_r - K(x) x_r|| / ||b_r|| for each right-hand side r, with the reduction scratch in
// a fixed-size array that lives in this file's device memory for as long as the library is loaded.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/tobk.h"
#include "device_common.cuh"
#include "unit_element.h"

namespace tobk {

void set_handleless_error(const char* msg);

constexpr int kNoAllocMaxRhs = 16;    // largest nrhs accepted
constexpr int kNoAllocBlocks = 1024;  // fixed grid width (grid-stride loop over nodes)

// Scratch shared by every call on a device: per-(RHS, block) partial sums and per-RHS arrival
// counters of the last-block reduction (256 KiB + 64 B per device).
static __device__ __align__(256) double g_noalloc_partial[kNoAllocMaxRhs * kNoAllocBlocks * 2];
static __device__ __align__(256) unsigned g_noalloc_counter[kNoAllocMaxRhs];

// Fine-grid SIMP stiffness with E_kappa evaluated from the densities inside the kernel.
template <int DIM>
struct FineOpFromDensity {
  Grid g;
  const double* x;
  const uint8_t* fixed;
  double penal, E0, Emin;
  double M[Dims<DIM>::ND * Dims<DIM>::ND];
  __device__ __forceinline__ double scale(int64_t e) const { return Emin + pow(x[e], penal) * (E0 - Emin); }
  __device__ __forceinline__ double entry(int64_t, int r, int c) const { return M[r * Dims<DIM>::ND + c]; }
};

// X read with its fixed DOFs taken as zero: the residual is that of the free-DOF system K_ff x_f
struct LoadFree {
  const double* v;
  const uint8_t* fixed;
  __device__ __forceinline__ double operator()(int64_t i) const { return fixed[i] ? 0.0 : __ldg(v + i); }
};

template <int DIM>
__global__ void __launch_bounds__(256) k_residual_noalloc(const __grid_constant__ FineOpFromDensity<DIM> op,
                                                          const double* __restrict__ B,
                                                          const double* __restrict__ X, int64_t stride,
                                                          double* __restrict__ partial, unsigned* counters,
                                                          double* __restrict__ relres) {
  __shared__ double smem[64];
  const int rhs = blockIdx.y;
  const int64_t off = (int64_t)rhs * stride;
  double v[2] = {0.0, 0.0};  // r.r, b.b over free DOFs
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < op.g.nnode;
       node += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    node_coords(op.g, node, i, j, k);
    double acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c] = 0.0;
    gather_rows<DIM, double>(op, i, j, k, LoadFree{X + off, op.fixed}, acc);
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t idx = DIM * node + c;
      if (op.fixed[idx]) continue;
      const double bi = B[off + idx];
      const double ri = bi - acc[c];
      v[0] += ri * ri;
      v[1] += bi * bi;
    }
  }
  double tot[2];
  if (grid_sum_last<2>(v, partial + (size_t)rhs * gridDim.x * 2, counters + rhs, tot, smem) && threadIdx.x == 0)
    relres[rhs] = tot[1] > 0.0 ? sqrt(tot[0] / tot[1]) : sqrt(tot[0]);
}

namespace {

std::mutex g_setup_mutex;
constexpr int kMaxDevices = 64;
double* g_partial_addr[kMaxDevices] = {nullptr};
unsigned* g_counter_addr[kMaxDevices] = {nullptr};

// Device addresses of the scratch arrays on device dev (current), looked up on the first call and
// again whenever `refresh` is set (the caller's stream is not capturing), so that a module reloaded
// after a device reset is seen.
int scratch_for_device(int dev, bool refresh, double** partial, unsigned** counters) {
  if (dev < 0 || dev >= kMaxDevices) return TOBK_E_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partial_addr[dev] || refresh) {
    void* p = nullptr;
    void* c = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess ||
        cudaGetSymbolAddress(&c, g_noalloc_counter) != cudaSuccess) {
      cudaGetLastError();
      return TOBK_E_CUDA;
    }
    g_partial_addr[dev] = static_cast<double*>(p);
    g_counter_addr[dev] = static_cast<unsigned*>(c);
  }
  *partial = g_partial_addr[dev];
  *counters = g_counter_addr[dev];
  return TOBK_OK;
}

template <int DIM>
void launch_noalloc(const tobk_desc& d, const double* x, const uint8_t* fixed, const double* B, const double* X,
                    int nrhs, double* relres, double* partial, unsigned* counters, cudaStream_t s) {
  FineOpFromDensity<DIM> op;
  int nel[3] = {d.nel[0], d.nel[1], DIM == 3 ? d.nel[2] : 1};
  op.g = make_grid(DIM, nel);
  op.x = x;
  op.fixed = fixed;
  op.penal = d.penal;
  op.E0 = d.E0;
  op.Emin = d.Emin;
  if (d.element == TOBK_ELEMENT_INCOMPATIBLE) {
    double A[unit_element::kMaxInternal * unit_element::kMaxDofs];
    unit_element::incompatible_tables(DIM, d.nu, op.M, A);
  } else {
    unit_element::stiffness(DIM, d.nu, op.M);
  }
  const int64_t want = (op.g.nnode + 255) / 256;
  const unsigned blocks = (unsigned)(want < kNoAllocBlocks ? want : kNoAllocBlocks);
  note_launch();
  k_residual_noalloc<DIM><<<dim3(blocks, nrhs), 256, 0, s>>>(op, B, X, op.g.n, partial, counters, relres);
}
}  // namespace

}  // namespace tobk

extern "C" int tobk_residual_noalloc(const tobk_desc* desc, const double* x, const uint8_t* fixed, const double* B,
                                     const double* X, int nrhs, double* relres, void* cuda_stream) {
  using namespace tobk;
  auto reject = [](int code, const char* msg) {
    set_handleless_error(msg);
    return code;
  };
  if (!desc || !x || !fixed || !B || !X || !relres) return reject(TOBK_E_ARG, "tobk_residual_noalloc: null pointer");
  if (desc->dim != 2 && desc->dim != 3) return reject(TOBK_E_ARG, "tobk_residual_noalloc: dim must be 2 or 3");
  for (int a = 0; a < desc->dim; ++a)
    if (desc->nel[a] < 1) return reject(TOBK_E_ARG, "tobk_residual_noalloc: nel must be >= 1 on every axis");
  // the material checks of tobk_create: a Poisson ratio of 1/2 or more makes the 3D Lame constant
  // infinite, a non-positive modulus or p < 1 leaves K(x) without meaning
  if (!(desc->nu > -1.0 && desc->nu < 0.5) || !(desc->E0 > 0.0) || !(desc->Emin > 0.0) || !(desc->penal >= 1.0))
    return reject(TOBK_E_ARG, "tobk_residual_noalloc: material parameters out of range");
  if (desc->element != TOBK_ELEMENT_PLAIN && desc->element != TOBK_ELEMENT_INCOMPATIBLE)
    return reject(TOBK_E_ARG, "tobk_residual_noalloc: unknown element");
  // the built-in scratch holds kNoAllocMaxRhs right-hand sides; larger blocks are rejected
  if (nrhs < 1 || nrhs > kNoAllocMaxRhs)
    return reject(TOBK_E_ARG, "tobk_residual_noalloc: nrhs must be between 1 and 16 (the size of its built-in "
                              "scratch)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return reject(TOBK_E_CUDA, "tobk_residual_noalloc: cudaGetDevice failed");
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusActive;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusActive;
  double* partial = nullptr;
  unsigned* counters = nullptr;
  if (scratch_for_device(dev, cs == cudaStreamCaptureStatusNone, &partial, &counters) != TOBK_OK) {
    return reject(TOBK_E_CUDA, "tobk_residual_noalloc: cudaGetSymbolAddress of the scratch failed");
  }
  // the arrival counters must start at zero (an interrupted earlier call could have left them set)
  cudaMemsetAsync(counters, 0, sizeof(unsigned) * kNoAllocMaxRhs, s);
  if (desc->dim == 2)
    launch_noalloc<2>(*desc, x, fixed, B, X, nrhs, relres, partial, counters, s);
  else
    launch_noalloc<3>(*desc, x, fixed, B, X, nrhs, relres, partial, counters, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    return reject(TOBK_E_CUDA, "tobk_residual_noalloc: kernel launch failed");
  }
  return TOBK_OK;
}
