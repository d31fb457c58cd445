// Shared device/host definitions of the tomo library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>

namespace tomo {

// ------------------------------------------------------------------------------------
// Geometry of one grid level: nx*ny*nz hex8 elements, (nx+1)(ny+1)(nz+1) nodes.
// Elements e = i + nx*(j + ny*k); nodes n = i + nxn*(j + nyn*k); nodal vectors SoA.
// ------------------------------------------------------------------------------------
struct Geom {
  int nx, ny, nz;     // elements
  int nxn, nyn, nzn;  // nodes per axis
  int nn;             // nodes
  int nel;            // elements
};

inline Geom make_geom(int nx, int ny, int nz) {
  Geom g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.nxn = nx + 1; g.nyn = ny + 1; g.nzn = nz + 1;
  g.nn = g.nxn * g.nyn * g.nzn;
  g.nel = nx * ny * nz;
  return g;
}

// ------------------------------------------------------------------------------------
// Element operator constants.  K0 is the 24x24 stiffness of the unit cube with E = 1
// (element DOF order 3a + c, local node a = ax + 2 ay + 4 az).  In the per-component
// Walsh-Hadamard basis X_c[m] = sum_s (-1)^{popc(m & s)} x_c[s] it is block diagonal with
// eight symmetric 3x3 blocks, block k coupling the modes (c, m = k ^ (1 << c)), c = 0..2.
// blk[k][c][c'] holds that block scaled by 1/64 so that K0 x = H (blk H x) per component.
// ------------------------------------------------------------------------------------
template <typename T>
struct ElemConst {
  T blk[8][3][3];
  T k0diag;      // K0 diagonal entry (identical for all 24 DOFs of the cube)
};

template <typename T>
struct DenseK0 {
  T k[576];
};

// Status word bits written by device code (never a trap).
enum : unsigned {
  DEV_OK = 0u,
  DEV_NAN = 1u,
  DEV_BREAKDOWN = 2u,
  DEV_TIMEOUT = 4u,
};

// Scalars of one CG solve, kept in device memory so that no host round trip is needed
// between kernels.
struct CgScalars {
  double rz;       // r^T z of the current iterate
  double rz_new;
  double pq;       // p^T A p
  double rr;       // r^T r
  double ff;       // f^T f
  double alpha, beta;
  double tol2;     // (rtol ||f||)^2
  int it;          // iterations done
  int done;        // 1 once converged or stopped
  int maxit;
  unsigned status; // DEV_* bits
  int loops;       // iterations launched by the device-side loop (termination guard)
  int rr_every;    // residual replacement interval (0: off)
};

#define TOMO_CUDA_TRY(expr)                                                        \
  do {                                                                             \
    cudaError_t _e = (expr);                                                       \
    if (_e != cudaSuccess) return ::tomo::cuda_fail(_e, #expr, __FILE__, __LINE__); \
  } while (0)

int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

// Programmatic dependent launch: every kernel of the library is launched with programmatic
// stream serialisation, and starts with PDL_ENTER(): it waits for the grids it depends on
// to complete (griddepcontrol.wait, before touching any memory) and at once lets its own
// dependents be scheduled (griddepcontrol.launch_dependents), so that the launch latency of
// the next kernel overlaps this one.  A dependent still cannot read anything until this
// grid has completed and its writes are visible.
template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ------------------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------------------
#ifdef __CUDACC__

#define PDL_ENTER()                                            \
  do {                                                         \
    asm volatile("griddepcontrol.wait;" ::: "memory");         \
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
  } while (0)

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Checked build (-DTOMO_CHECKED): a computed index passes through TOMO_CHK(i, n, site); one
// outside [0, n) is recorded in this translation unit's check word (the first violation:
// site in bits 48-63, the index's low 48 bits below) and replaced by 0, so the access stays
// inside its buffer; no trap.  TOMO_AT(base, off, n, site) is the checked address base + off.
// The host reads and clears the words (tomo_check_report).  Without TOMO_CHECKED the macros
// are the index and the address themselves.
#ifdef TOMO_CHECKED
namespace {
__device__ unsigned long long g_check_word = 0ull;
}
__device__ __forceinline__ long long tomo_chk(long long i, long long n, int site) {
  if (i < 0 || i >= n) {
    atomicCAS(&g_check_word, 0ull,
              ((unsigned long long)site << 48) | ((unsigned long long)i & 0xFFFFFFFFFFFFull));
    return 0;
  }
  return i;
}
#define TOMO_CHK(i, n, site) tomo_chk((long long)(i), (long long)(n), (site))
#define TOMO_AT(base, off, n, site) ((base) + tomo_chk((long long)(off), (long long)(n), (site)))
// host accessor of this translation unit's word (read, then cleared)
#define TOMO_CHECK_ACCESSOR(fn)                                                   \
  unsigned long long fn() {                                                       \
    unsigned long long v = 0ull, z = 0ull;                                        \
    if (cudaMemcpyFromSymbol(&v, g_check_word, sizeof v) != cudaSuccess ||        \
        cudaMemcpyToSymbol(g_check_word, &z, sizeof z) != cudaSuccess) {          \
      cudaGetLastError();                                                         \
      return ~0ull;                                                               \
    }                                                                             \
    return v;                                                                     \
  }
#else
#define TOMO_CHK(i, n, site) (i)
// base + off with the tokens as written (the regular build's address arithmetic unchanged)
#define TOMO_AT(base, off, n, site) base + off
#endif

// Load of data that does not change while the kernel runs (NC: the read-only path), or, in
// the persistent lockstep iteration, where earlier phases of the same kernel write it, a
// load cached in L2 only (coherent across the SMs after the phase barrier).
template <bool NC, typename T>
__device__ __forceinline__ T ldv(const T* p) {
  if constexpr (NC) return __ldg(p);
  else return __ldcg(p);
}

// A thread's sum of FP32 terms kept as the unevaluated pair hi + lo (Knuth's TwoSum per
// term): ~44 significant bits from FP32 arithmetic alone.  FP64 runs at 1/64 of the FP32
// rate on this part, so accumulating every element in FP64 would bound the streaming
// kernels; the pair becomes a double once per thread, before the grid reduction.  The rn
// intrinsics keep nvcc from contracting the error terms.
struct FloatPairSum {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float s = __fadd_rn(hi, v);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum NV doubles over the block, then over the blocks of one grid's work: block b of nb
// writes its partial to partials[NV*b + v]; the last block to finish adds the partials in
// block order (deterministic) and calls fin(totals) with thread 0.  counter must start at 0
// and is reset by the last block.  All threads of the block must call this.  (b, nb) are
// the launch's own block index and count, or a block's place within one grid of a batched
// launch.
template <int NV, class Fin>
__device__ void grid_reduce_at(double (&v)[NV], double* partials, unsigned* counter, Fin fin,
                               unsigned b_self, unsigned nb) {
  __shared__ double s_red[32][NV];
  __shared__ bool s_last;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nthreads = blockDim.x * blockDim.y * blockDim.z;
  const int lane = tid & 31, wid = tid >> 5, nw = (nthreads + 31) >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) s_red[wid][q] = s;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = lane < nw ? s_red[lane][q] : 0.0;
      s = warp_sum(s);
      if (lane == 0) partials[(size_t)NV * b_self + q] = s;
    }
    if (lane == 0) {
      __threadfence();
      unsigned t = atomicAdd(counter, 1u);
      s_last = (t == nb - 1);
    }
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) acc[q] = 0.0;
  for (unsigned b = tid; b < nb; b += nthreads) {
#pragma unroll
    for (int q = 0; q < NV; ++q) acc[q] += __ldcg(partials + (size_t)NV * b + q);
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    double s = warp_sum(acc[q]);
    if (lane == 0) s_red[wid][q] = s;
  }
  __syncthreads();
  if (tid == 0) {
    double tot[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int w = 0; w < nw; ++w) s += s_red[w][q];
      tot[q] = s;
    }
    *counter = 0u;
    fin(tot);
  }
}

template <int NV, class Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], double* partials,
                                            unsigned* counter, Fin fin) {
  grid_reduce_at<NV>(v, partials, counter, fin,
                     blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                     gridDim.x * gridDim.y * gridDim.z);
}

// Batched launches: one launch runs the same operation for up to kBatchMax grids; grid q
// owns the launch's blocks [cta0[q], cta0[q+1]).  Returns q for block `cta` (binary search;
// cta0 is non-decreasing, cta0[0] = 0, cta < cta0[n]).
__device__ __forceinline__ int batch_owner(const int* cta0, int n, int cta) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (cta0[mid] <= cta) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

#endif  // __CUDACC__

// Grids per batched launch (bounded by the kernel parameter space the tables use).
constexpr int kBatchMax = 64;

}  // namespace tomo
