// Internal declarations of the GB300 multilevel buckling solver library (not part of the C-ABI).
//
// Data layout in device memory (all levels):
//   element (i,j,k) -> e = i + nelx*(j + nely*k); node (i,j,k) -> a = i + nnx*(j + nny*k);
//   DOF c of node a -> d*a + c (node-interleaved).  Multi-RHS blocks are RHS-major: [r][n].
//   Dirichlet DOFs hold 0 in every vector the solver produces.
// Level 1 (fine) operators are matrix-free: y = sum_e E_kappa(x_e) K_e0 v_e (paper Sec. 2).
// Levels >= 2 store one dense (d 2^d)^2 element matrix per coarse element: the Galerkin product
// P^T K P of nested bi/trilinear grids assembles element by element (paper Sec. 2.1 step 1).
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

namespace tobk {

constexpr int kMaxLevels = 12;
constexpr int kMaxRhs = 64;      // RHS per multi-RHS solve (per-kernel reduction counters)
constexpr int kNumCounterSets = 6;
constexpr int kScStride = 16;  // doubles of per-RHS scalar state in the CG driver
constexpr int kMaxSmoothSteps = 8;  // smoothing steps per pre-/post-smoothing phase

// per-RHS CG scalar slots
enum ScSlot {
  SC_ZR = 0,      // z.r of the current iteration
  SC_ZQ = 1,      // z.q_old (flexible beta)
  SC_PR = 2,      // p_old.r
  SC_PQ = 3,      // p.q of the current direction
  SC_ALPHA = 4,
  SC_BETA = 5,
  SC_RR = 6,      // r.r
  SC_BB = 7,      // b.b (free DOFs)
  SC_RELRES = 8,  // sqrt(r.r / b.b)
  SC_ACTIVE = 9,  // 1: iterating, 0: converged or stopped
  SC_ITERS = 10,
  SC_ZR_OLD = 11,
  SC_PQ_OLD = 12,
  SC_STATUS = 13, // 0 ok, 1 breakdown (p.q <= 0), 2 non-finite
  SC_RTOL = 14,
};

struct Grid {
  int dim;
  int nel[3];
  int nn[3];
  int64_t m;      // elements
  int64_t nnode;  // nodes
  int64_t n;      // DOFs
};

inline Grid make_grid(int dim, const int nel[3]) {
  Grid g;
  g.dim = dim;
  for (int a = 0; a < 3; ++a) {
    g.nel[a] = (a < dim) ? nel[a] : 1;
    g.nn[a] = (a < dim) ? nel[a] + 1 : 1;
  }
  g.m = (int64_t)g.nel[0] * g.nel[1] * g.nel[2];
  g.nnode = (int64_t)g.nn[0] * g.nn[1] * g.nn[2];
  g.n = g.nnode * dim;
  return g;
}

// ------------------------------------------------------------------------------------------------
// Element tables computed on the host (Gauss quadrature written independently for this library).
// ------------------------------------------------------------------------------------------------
struct ElementTables {
  int dim, nn, nd, ngp, nv;
  int element = 0;          // tobk_element
  std::vector<double> Ke0;  // [nd*nd] unit-modulus stiffness (condensed for incompatible modes)
  std::vector<double> A;    // [d*d][nd] condensation map of the incompatible modes (empty otherwise)
  std::vector<double> dN;   // [ngp][dim][nn] shape-function gradients in physical coordinates
  std::vector<double> D;    // [nv*nv] unit-modulus constitutive matrix
  double wdet;              // Gauss weight x |J| (same at every Gauss point)
  std::vector<double> W;    // [2^dim children][nn child nodes][nn coarse nodes] interpolation weights
};
ElementTables make_element_tables(int dim, double nu, int element = 0);

// ------------------------------------------------------------------------------------------------
// device memory arena (one cudaMalloc per handle)
// ------------------------------------------------------------------------------------------------
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = ((count * sizeof(T)) + 255) & ~size_t(255);
    if (used + bytes > cap) return nullptr;
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

struct Level {
  Grid g;
  uint8_t* fixed = nullptr;   // [n]
  // stored Galerkin element matrices (levels >= 2)
  double* Ke = nullptr;       // [m][nd*nd]
  float* Ke32 = nullptr;      // FP32 copy for the mixed-precision V-cycle
  double* Ge = nullptr;       // [m][nd*nd] Galerkin G (only down to the eigen level)
  double* S = nullptr;        // assembled nodal stencil of K (levels >= 2), see stencil.cu
  float* S32 = nullptr;
  double* dinv = nullptr;     // [n] inverse diagonal (0 at fixed DOFs)
  float* dinv32 = nullptr;
  // smoother: per-step coefficients [2 * kMaxSmoothSteps] (+ lambda_max estimate at the end) and
  // the Chebyshev increment vectors (ping-pong, [rmax][n])
  double* coef = nullptr;
  float* coef32 = nullptr;
  double *dA = nullptr, *dB = nullptr;
  float *dA32 = nullptr, *dB32 = nullptr;
  // V-cycle work vectors, capacity rmax RHS: b, z, t (ping-pong), r
  double *b = nullptr, *z = nullptr, *t = nullptr, *r = nullptr;
  float *b32 = nullptr, *z32 = nullptr, *t32 = nullptr, *r32 = nullptr;
};

// Multi-RHS PCG work space for solves that start at a given level.
struct CGWork {
  double *x, *r, *z, *zt, *p0, *p1, *q;
  double* sc;          // [rmax][kScStride]
  double* partial;     // reduction partials
  unsigned* counters;  // last-block counters
  double* host_sc;     // pinned host copy of sc
};

}  // namespace tobk

namespace tobk {
// Number of kernels this library has launched (all handles); read through tobk_launch_count().
extern std::atomic<long long> g_launch_count;
inline void note_launch() { g_launch_count.fetch_add(1, std::memory_order_relaxed); }

// Programmatic dependent launch.  The solver's inner loops are long chains of short, dependent
// kernels; a kernel launched with launch_pdl may be scheduled while the previous kernel of the
// stream is still finishing, so that its launch and block scheduling overlap that kernel's tail.
// Every kernel launched this way calls pdl_wait() before its first global-memory access: the wait
// returns once the previous kernel has completed and its writes are visible (and at once when the
// kernel was launched without the attribute).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
}  // namespace tobk

// The opaque handle of the C-ABI.
struct tobk_handle;
