// The coarse tail of the multigrid V-cycle (the preconditioner of the state solve of Eq. 4,
// Section III-D) in one launch of a thread-block cluster: from level l0 down to the dense
// coarsest and back, the zero-start Chebyshev smoothing, the residual, the restriction, the
// coarsest solve, the prolongation and the post-smoothing, every pass separated from the
// next by a cluster barrier instead of a kernel boundary.
//
// On these levels a launched kernel does a microsecond of work or less, so a V-cycle's
// coarse levels cost the launch and drain latency of about six dependent launches per
// level.  One CTA alone does not have the issue rate for the element work (measured); a
// cluster of kVtCluster CTAs on as many SMs shares it, and its barrier is a hardware one.
// A product is two passes: element pass (each element's corner forces s_e K0 x_e, the
// Walsh-Hadamard block form, into an element buffer) and node pass (each node adds its up
// to eight elements' corners in a fixed order, then the smoother update or the residual).
// Transfers and the smoother follow the launched kernels' definitions (trilinear
// restriction and prolongation, Chebyshev-Jacobi with the per-level D^-1, the zero-start
// first step fused into the restriction, the coefficients of the grid's smoother setting),
// so the tail is the same linear operator as the launched levels; only the order in which
// a node's element contributions are added differs.
//
// Vectors live in the grid's level buffers (global memory, L2-resident at these sizes);
// data written by another CTA of the cluster is read with L2 loads after the barrier
// (release / acquire at cluster scope).
#include <cooperative_groups.h>

#include "common.cuh"
#include "host.h"
#include "march_body.cuh"

namespace tomo {

namespace cg = cooperative_groups;

namespace {

constexpr int kVtCluster = 8;   // CTAs (SMs) of the cluster, the portable maximum
constexpr int kVtThreads = 512;

__device__ __forceinline__ int vt_node(const Geom& g, int i, int j, int k) {
  return i + g.nxn * (j + g.nyn * k);
}

// Corner forces of every element: eb[(q * 3 + c) * ld + e] = (s_e K0 x_e)_{q,c} for local
// node q = qx + 2 qy + 4 qz and component c.  Thread gt of gs takes elements gt, gt + gs, ...
__device__ void vt_elements(const Geom& g, const float* __restrict__ s, const float* x,
                            float* eb, int ld, const ElemConst<float>& C, int gt, int gs) {
  const int nn = g.nn;
  const int dy = g.nxn, dz = g.nxn * g.nyn;
  for (int e = gt; e < g.nel; e += gs) {
    const int i = e % g.nx, j = (e / g.nx) % g.ny, k = e / (g.nx * g.ny);
    const int n0 = TOMO_CHK(vt_node(g, i, j, k), nn, 18);
    const int off[8] = {0, 1, dy, dy + 1, dz, dz + 1, dz + dy, dz + dy + 1};
    float X[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float* xc = x + (size_t)c * nn + n0;
      const float a0 = __ldcg(xc);
      float v[8];
      v[0] = 0.0f;
#pragma unroll
      for (int q = 1; q < 8; ++q) v[q] = __ldcg(xc + off[q]) - a0;
      fwht8(v);
#pragma unroll
      for (int m = 0; m < 8; ++m) X[c][m] = v[m];
    }
    float W[3][8];
    block_apply(C, __ldg(s + e), X, W);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = W[c][m];
      fwht8(v);
#pragma unroll
      for (int q = 0; q < 8; ++q) eb[(q * 3 + c) * ld + e] = v[q];
    }
  }
}

// (K x)_c at node (i, j, k) from the element buffer: its up to eight elements in a fixed order
__device__ __forceinline__ void vt_gather(const Geom& g, const float* eb, int ld, int i, int j,
                                          int k, float (&y)[3]) {
  y[0] = y[1] = y[2] = 0.0f;
#pragma unroll
  for (int dz = 0; dz < 2; ++dz)
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const int ei = i - dx, ej = j - dy, ek = k - dz;
        if (ei < 0 || ei >= g.nx || ej < 0 || ej >= g.ny || ek < 0 || ek >= g.nz) continue;
        const int e = TOMO_CHK(ei + g.nx * (ej + g.ny * ek), g.nel, 18);
        const int q = dx + 2 * dy + 4 * dz;  // the node is corner q of that element
#pragma unroll
        for (int c = 0; c < 3; ++c) y[c] += __ldcg(eb + (q * 3 + c) * ld + e);
      }
}

}  // namespace

namespace {

// One Chebyshev step on level L: x_new = x + c1 (x - x_prev) + c2 D^-1 (b - K x), fixed DOFs
// 0, written over x_prev; then the buffers swap roles (*cur: 0 -> the iterate is in x).
// xprev_zero: x_prev = 0 (the step after the zero-start step) is not read.
__device__ void vt_cheb(cg::cluster_group& cl, const VTailLevel& L, float* eb, int ld,
                        int* cur, float c1, float c2, bool xprev_zero,
                        const ElemConst<float>& C, int gt, int gs) {
  const Geom& g = L.g;
  const int nn = g.nn;
  float* x = *cur ? L.xp : L.x;
  float* xp = *cur ? L.x : L.xp;
  vt_elements(g, L.s, x, eb, ld, C, gt, gs);
  cl.sync();
  for (int n = gt; n < nn; n += gs) {
    const int i = n % g.nxn, j = (n / g.nxn) % g.nyn, k = n / (g.nxn * g.nyn);
    float y[3];
    vt_gather(g, eb, ld, i, j, k, y);
    const unsigned mk = L.mask[n];
    const float dinv = __ldg(L.invd + n);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t q = (size_t)c * nn + n;
      const float xv = __ldcg(x + q);
      float v = xv + c2 * (dinv * (__ldcg(L.b + q) - y[c]));
      // (x_prev = 0 after the zero-start step: the term is c1 x)
      if (c1 != 0.0f) v += c1 * (xv - (xprev_zero ? 0.0f : __ldcg(xp + q)));
      xp[q] = ((mk >> c) & 1u) ? 0.0f : v;
    }
  }
  *cur ^= 1;
  cl.sync();
}

__global__ void __launch_bounds__(kVtThreads, 1)
    k_vtail(const __grid_constant__ VTailArgs A, const __grid_constant__ ElemConst<float> C) {
  PDL_ENTER();
  cg::cluster_group cl = cg::this_cluster();
  // the stop flag is final while this kernel runs: every CTA of the cluster leaves together
  if (A.skip != nullptr && *A.skip) return;
  const int gt = (int)cl.block_rank() * blockDim.x + threadIdx.x;
  const int gs = (int)cl.num_blocks() * blockDim.x;
  const int last = A.nlev - 1;
  float* eb = A.eb;
  const int ld = A.ld;
  int cur[kVtMaxLevels];
  // ---- down: zero-start smoothing, residual, restriction ----
  for (int l = 0; l < last; ++l) {
    const VTailLevel& L = A.L[l];
    const Geom& g = L.g;
    const int nn = g.nn;
    cur[l] = 0;
    if (l == 0 && !A.first_done) {  // zero-start step x1 = c2 D^-1 b (inner levels: fused)
      for (int n = gt; n < nn; n += gs) {
        const unsigned mk = L.mask[n];
        const float dinv = __ldg(L.invd + n);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const size_t q = (size_t)c * nn + n;
          L.x[q] = ((mk >> c) & 1u) ? 0.0f : L.c2[0] * (dinv * __ldcg(L.b + q));
        }
      }
      cl.sync();
    }
    for (int s = 1; s < L.K; ++s)
      vt_cheb(cl, L, eb, ld, &cur[l], L.c1[s], L.c2[s], s == 1, C, gt, gs);
    // residual t = b - K x
    {
      const float* x = cur[l] ? L.xp : L.x;
      vt_elements(g, L.s, x, eb, ld, C, gt, gs);
      cl.sync();
      for (int n = gt; n < nn; n += gs) {
        const int i = n % g.nxn, j = (n / g.nxn) % g.nyn, k = n / (g.nxn * g.nyn);
        float y[3];
        vt_gather(g, eb, ld, i, j, k, y);
        const unsigned mk = L.mask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const size_t q = (size_t)c * nn + n;
          L.t[q] = ((mk >> c) & 1u) ? 0.0f : __ldcg(L.b + q) - y[c];
        }
      }
      cl.sync();
    }
    // restriction b_c = P^T t (weights 1, 1/2 per axis), fixed DOFs 0; below the coarsest
    // level's parent also the coarse level's zero-start step x1 = c2 D^-1 b_c
    {
      const VTailLevel& Lc = A.L[l + 1];
      const Geom& gc = Lc.g;
      const bool fuse = l + 1 < last;
      for (int N = gt; N < gc.nn; N += gs) {
        const int I = N % gc.nxn, J = (N / gc.nxn) % gc.nyn, K = N / (gc.nxn * gc.nyn);
        float acc[3] = {0.0f, 0.0f, 0.0f};
        for (int dz = 0; dz < 3; ++dz) {
          const int kk = 2 * K + dz - 1;
          if (kk < 0 || kk >= g.nzn) continue;
          const float wz = dz == 1 ? 1.0f : 0.5f;
          float az[3] = {0.0f, 0.0f, 0.0f};
          for (int dy = 0; dy < 3; ++dy) {
            const int jj = 2 * J + dy - 1;
            if (jj < 0 || jj >= g.nyn) continue;
            const float wy = dy == 1 ? 1.0f : 0.5f;
            float ay[3] = {0.0f, 0.0f, 0.0f};
            for (int dx = 0; dx < 3; ++dx) {
              const int ii = 2 * I + dx - 1;
              if (ii < 0 || ii >= g.nxn) continue;
              const float wx = dx == 1 ? 1.0f : 0.5f;
              const int n = TOMO_CHK(vt_node(g, ii, jj, kk), nn, 18);
#pragma unroll
              for (int c = 0; c < 3; ++c) ay[c] += wx * __ldcg(L.t + (size_t)c * nn + n);
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) az[c] += wy * ay[c];
          }
#pragma unroll
          for (int c = 0; c < 3; ++c) acc[c] += wz * az[c];
        }
        const unsigned mk = Lc.mask[N];
        const float dinv = fuse ? __ldg(Lc.invd + N) : 0.0f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const size_t q = (size_t)c * gc.nn + N;
          const bool fx = (mk >> c) & 1u;
          Lc.b[q] = fx ? 0.0f : acc[c];
          if (fuse) Lc.x[q] = fx ? 0.0f : Lc.c2[0] * (dinv * acc[c]);
        }
      }
      cl.sync();
    }
  }
  // ---- coarsest: z = D^-1/2 Ainv D^-1/2 b (the dense inverse of the scaled matrix); every
  // CTA stages D^-1/2 b in its shared memory and takes every cluster-size-th row ----
  {
    const VTailLevel& L = A.L[last];
    extern __shared__ float vt_rs[];
    const int n = A.nc;
    for (int q = threadIdx.x; q < n; q += blockDim.x) vt_rs[q] = A.dsc[q] * __ldcg(L.b + q);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int w0 = (int)cl.block_rank() * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nw = (int)cl.num_blocks() * (blockDim.x >> 5);
    for (int row = w0; row < n; row += nw) {
      const float* a = A.Ainv + (size_t)row * n;
      float acc = 0.0f;
      for (int c = lane; c < n; c += 32) acc += __ldg(a + TOMO_CHK(c, n, 18)) * vt_rs[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) L.x[row] = A.dsc[row] * acc;
    }
    cl.sync();
  }
  // ---- up: prolongation x += P x_c (fixed DOFs unchanged), post-smoothing ----
  for (int l = last - 1; l >= 0; --l) {
    const VTailLevel& L = A.L[l];
    const VTailLevel& Lc = A.L[l + 1];
    const Geom& g = L.g;
    const Geom& gc = Lc.g;
    {
      const float* xc = (l + 1 == last || !cur[l + 1]) ? Lc.x : Lc.xp;
      float* x = cur[l] ? L.xp : L.x;
      for (int n = gt; n < g.nn; n += gs) {
        const int i = n % g.nxn, j = (n / g.nxn) % g.nyn, k = n / (g.nxn * g.nyn);
        const int i0 = i >> 1, i1 = (i + 1) >> 1;
        const int j0 = j >> 1, j1 = (j + 1) >> 1;
        const int k0 = k >> 1, k1 = (k + 1) >> 1;
        const float wi0 = (i & 1) ? 0.5f : 1.0f, wi1 = (i & 1) ? 0.5f : 0.0f;
        const float wj0 = (j & 1) ? 0.5f : 1.0f, wj1 = (j & 1) ? 0.5f : 0.0f;
        const float wk0 = (k & 1) ? 0.5f : 1.0f, wk1 = (k & 1) ? 0.5f : 0.0f;
        const int r00 = gc.nxn * (j0 + gc.nyn * k0), r10 = gc.nxn * (j1 + gc.nyn * k0);
        const int r01 = gc.nxn * (j0 + gc.nyn * k1), r11 = gc.nxn * (j1 + gc.nyn * k1);
        const unsigned mk = L.mask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float* v = xc + (size_t)c * gc.nn;
          const float a00 = wi0 * __ldcg(v + TOMO_CHK(r00 + i0, gc.nn, 18)) +
                            wi1 * __ldcg(v + TOMO_CHK(r00 + i1, gc.nn, 18));
          const float a10 = wi0 * __ldcg(v + TOMO_CHK(r10 + i0, gc.nn, 18)) +
                            wi1 * __ldcg(v + TOMO_CHK(r10 + i1, gc.nn, 18));
          const float a01 = wi0 * __ldcg(v + TOMO_CHK(r01 + i0, gc.nn, 18)) +
                            wi1 * __ldcg(v + TOMO_CHK(r01 + i1, gc.nn, 18));
          const float a11 = wi0 * __ldcg(v + TOMO_CHK(r11 + i0, gc.nn, 18)) +
                            wi1 * __ldcg(v + TOMO_CHK(r11 + i1, gc.nn, 18));
          const float acc = wk0 * (wj0 * a00 + wj1 * a10) + wk1 * (wj0 * a01 + wj1 * a11);
          const size_t q = (size_t)c * g.nn + n;
          if (!((mk >> c) & 1u)) x[q] = __ldcg(x + q) + acc;
        }
      }
      cl.sync();
    }
    for (int s = 0; s < L.K; ++s)
      vt_cheb(cl, L, eb, ld, &cur[l], s == 0 ? 0.0f : L.c1[s], L.c2[s], false, C, gt, gs);
  }
}

}  // namespace

int vtail_ctas() {
  int dev = 0, ok = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&ok, cudaDevAttrClusterLaunch, dev) != cudaSuccess || !ok) {
    cudaGetLastError();
    return 0;
  }
  return kVtCluster;
}

cudaError_t launch_vtail(cudaStream_t st, const VTailArgs& A, const ElemConst<float>& C) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(kVtCluster);
  cfg.blockDim = dim3(kVtThreads);
  cfg.dynamicSmemBytes = sizeof(float) * (size_t)A.nc;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kVtCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_vtail, A, C);
}

#ifdef TOMO_CHECKED
TOMO_CHECK_ACCESSOR(check_word_vtail)
#endif

}  // namespace tomo
