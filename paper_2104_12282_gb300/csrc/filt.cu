// Density filter, SIMP material, compliance sensitivity and the optimality-criteria update
// (Eq. 4 and Eq. 5, Section III-D).
#include "common.cuh"
#include "host.h"

namespace tomo {

// ---------------------------------------------------------------------------------------
// Filter: mode 0 out = (H in)/Hs, mode 1 out = H (in/Hs), mode 2 out = H in.
// H_ij = max(0, rmin - |x_i - x_j|) over element centroids, taps (di, dj, dk) with their
// weights, truncated at the domain boundary.  Optional fused material for mode 0:
// s = h (Emin + rho^p (E0 - Emin)).
// ---------------------------------------------------------------------------------------
template <typename T, int MODE, bool MAT>
__global__ void k_filter(Geom g, const int4* __restrict__ taps, const T* __restrict__ tapw,
                         int ntaps, const T* __restrict__ in, const T* __restrict__ Hs,
                         T* __restrict__ out, T E0, T Emin, T penal, T h, T* __restrict__ s_out) {
  PDL_ENTER();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.nel; e += gridDim.x * blockDim.x) {
    const int i = e % g.nx, j = (e / g.nx) % g.ny, k = e / (g.nx * g.ny);
    T acc = T(0);
    for (int t = 0; t < ntaps; ++t) {
      const int4 d = taps[t];
      const int ii = i + d.x, jj = j + d.y, kk = k + d.z;
      if (ii < 0 || ii >= g.nx || jj < 0 || jj >= g.ny || kk < 0 || kk >= g.nz) continue;
      const int nb = TOMO_CHK(ii + g.nx * (jj + g.ny * kk), g.nel, 14);
      T v = ldg(in + nb);
      if (MODE == 1) v = v / ldg(Hs + nb);
      acc += tapw[t] * v;
    }
    if (MODE == 0) acc = acc / Hs[e];
    out[e] = acc;
    if (MAT) s_out[e] = h * (Emin + pow(acc, penal) * (E0 - Emin));
  }
}

// Tiled form of the same filter for tap radius R <= 3: a CTA stages a 32 x 8 x 8 element
// tile with an R-element halo in shared memory (mode 1 divides by Hs once per staged
// element, not once per tap), builds the (2R+1)^3 weight table from the tap list, and each
// thread accumulates a column of 8 outputs along z, reusing each staged column for all
// (2R+1) z-offsets.  Elements outside the domain stage as 0 (the filter is truncated).
constexpr int kFtX = 32, kFtY = 8, kFtZ = 8;

template <typename T, int R, int MODE, bool MAT>
__global__ void __launch_bounds__(kFtX * kFtY)
    k_filter_tiled(Geom g, const int4* __restrict__ taps, const T* __restrict__ tapw, int ntaps,
                   const T* __restrict__ in, const T* __restrict__ Hs, T* __restrict__ out,
                   T E0, T Emin, T penal, T h, T* __restrict__ s_out) {
  constexpr int W = 2 * R + 1;
  constexpr int SX = kFtX + 2 * R, SY = kFtY + 2 * R, SZ = kFtZ + 2 * R;
  __shared__ T tile[SZ][SY][SX];
  __shared__ T wt[W * W * W];
  PDL_ENTER();
  const int tid = threadIdx.x + kFtX * threadIdx.y;
  const int i0 = blockIdx.x * kFtX, j0 = blockIdx.y * kFtY, k0 = blockIdx.z * kFtZ;
  for (int q = tid; q < W * W * W; q += kFtX * kFtY) wt[q] = T(0);
  __syncthreads();
  for (int t = tid; t < ntaps; t += kFtX * kFtY) {
    const int4 d = taps[t];
    wt[(d.z + R) * W * W + (d.y + R) * W + (d.x + R)] = tapw[t];
  }
  for (int q = tid; q < SX * SY * SZ; q += kFtX * kFtY) {
    const int x = q % SX, y = (q / SX) % SY, z = q / (SX * SY);
    const int i = i0 + x - R, j = j0 + y - R, k = k0 + z - R;
    T v = T(0);
    if (i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz) {
      const int e = TOMO_CHK(i + g.nx * (j + g.ny * k), g.nel, 14);
      v = ldg(in + e);
      if (MODE == 1) v = v / ldg(Hs + e);
    }
    tile[z][y][x] = v;
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  T acc[kFtZ];
#pragma unroll
  for (int z = 0; z < kFtZ; ++z) acc[z] = T(0);
#pragma unroll 1
  for (int dj = 0; dj < W; ++dj) {
#pragma unroll
    for (int di = 0; di < W; ++di) {
      T col[SZ];
#pragma unroll
      for (int z = 0; z < SZ; ++z) col[z] = tile[z][ty + dj][tx + di];
#pragma unroll
      for (int dk = 0; dk < W; ++dk) {
        const T w = wt[dk * W * W + dj * W + di];
#pragma unroll
        for (int z = 0; z < kFtZ; ++z) acc[z] += w * col[z + dk];
      }
    }
  }
  const int i = i0 + tx, j = j0 + ty;
  if (i >= g.nx || j >= g.ny) return;
#pragma unroll
  for (int z = 0; z < kFtZ; ++z) {
    const int k = k0 + z;
    if (k >= g.nz) break;
    const int e = TOMO_CHK(i + g.nx * (j + g.ny * k), g.nel, 14);
    T v = acc[z];
    if (MODE == 0) v = v / Hs[e];
    out[e] = v;
    if (MAT) s_out[e] = h * (Emin + pow(v, penal) * (E0 - Emin));
  }
}

// The same tiling for radii 4..8 (rmin up to 9 elements; the paper's R = 0.08 on Mesh 3 is
// 7.2 elements): radius at run time, tile and weight table in dynamic shared memory.
constexpr int kFtMaxR = 8;
template <int MODE, bool MAT>
__global__ void __launch_bounds__(kFtX * kFtY)
    k_filter_tiled_wide(Geom g, int R, const int4* __restrict__ taps,
                        const float* __restrict__ tapw, int ntaps, const float* __restrict__ in,
                        const float* __restrict__ Hs, float* __restrict__ out, float E0,
                        float Emin, float penal, float h, float* __restrict__ s_out) {
  extern __shared__ __align__(16) float ft_smem[];
  const int W = 2 * R + 1;
  const int SX = kFtX + 2 * R, SY = kFtY + 2 * R, SZ = kFtZ + 2 * R;
  float* tile = ft_smem;                 // [SZ][SY][SX]
  float* wt = ft_smem + SX * SY * SZ;    // [W][W][W]
  PDL_ENTER();
  const int tid = threadIdx.x + kFtX * threadIdx.y;
  const int i0 = blockIdx.x * kFtX, j0 = blockIdx.y * kFtY, k0 = blockIdx.z * kFtZ;
  for (int q = tid; q < W * W * W; q += kFtX * kFtY) wt[q] = 0.0f;
  __syncthreads();
  for (int t = tid; t < ntaps; t += kFtX * kFtY) {
    const int4 d = taps[t];
    wt[(d.z + R) * W * W + (d.y + R) * W + (d.x + R)] = tapw[t];
  }
  for (int q = tid; q < SX * SY * SZ; q += kFtX * kFtY) {
    const int x = q % SX, y = (q / SX) % SY, z = q / (SX * SY);
    const int i = i0 + x - R, j = j0 + y - R, k = k0 + z - R;
    float v = 0.0f;
    if (i >= 0 && i < g.nx && j >= 0 && j < g.ny && k >= 0 && k < g.nz) {
      const int e = TOMO_CHK(i + g.nx * (j + g.ny * k), g.nel, 14);
      v = __ldg(in + e);
      if (MODE == 1) v = v / __ldg(Hs + e);
    }
    tile[q] = v;
  }
  __syncthreads();
  const int tx = threadIdx.x, ty = threadIdx.y;
  float acc[kFtZ];
#pragma unroll
  for (int z = 0; z < kFtZ; ++z) acc[z] = 0.0f;
  for (int dj = 0; dj < W; ++dj) {
    for (int di = 0; di < W; ++di) {
      const float* col = tile + (ty + dj) * SX + (tx + di);
      for (int dk = 0; dk < W; ++dk) {
        const float w = wt[dk * W * W + dj * W + di];
        if (w == 0.0f) continue;  // uniform over the CTA
#pragma unroll
        for (int z = 0; z < kFtZ; ++z) acc[z] = fmaf(w, col[(z + dk) * SX * SY], acc[z]);
      }
    }
  }
  const int i = i0 + tx, j = j0 + ty;
  if (i >= g.nx || j >= g.ny) return;
#pragma unroll
  for (int z = 0; z < kFtZ; ++z) {
    const int k = k0 + z;
    if (k >= g.nz) break;
    const int e = TOMO_CHK(i + g.nx * (j + g.ny * k), g.nel, 14);
    float v = acc[z];
    if (MODE == 0) v = v / Hs[e];
    out[e] = v;
    if (MAT) s_out[e] = h * (Emin + powf(v, penal) * (E0 - Emin));
  }
}

template <int MODE, bool MAT>
cudaError_t launch_wide(dim3 grid, dim3 block, size_t smem, cudaStream_t st, Geom g, int R,
                        const int4* taps, const float* tapw, int ntaps, const float* in,
                        const float* Hs, float* out, float E0, float Emin, float penal, float h,
                        float* s_out) {
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(k_filter_tiled_wide<MODE, MAT>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  return pdl_launch(k_filter_tiled_wide<MODE, MAT>, grid, block, smem, st, g, R, taps, tapw,
                    ntaps, in, Hs, out, E0, Emin, penal, h, s_out);
}

template <typename T, int R>
bool launch_filter_tiled(cudaStream_t st, Geom g, const int4* taps, const T* tapw, int ntaps,
                         const T* in, const T* Hs, T* out, int mode, int material, T E0,
                         T Emin, T penal, T h, T* s_out) {
  const dim3 grid((g.nx + kFtX - 1) / kFtX, (g.ny + kFtY - 1) / kFtY, (g.nz + kFtZ - 1) / kFtZ);
  const dim3 block(kFtX, kFtY);
  if (grid.y > 65535 || grid.z > 65535) return false;
  if (mode == 0 && material)
    pdl_launch(k_filter_tiled<T, R, 0, true>, grid, block, 0, st, g, taps, tapw, ntaps, in, Hs,
               out, E0, Emin, penal, h, s_out);
  else if (mode == 0)
    pdl_launch(k_filter_tiled<T, R, 0, false>, grid, block, 0, st, g, taps, tapw, ntaps, in, Hs,
               out, E0, Emin, penal, h, s_out);
  else if (mode == 1)
    pdl_launch(k_filter_tiled<T, R, 1, false>, grid, block, 0, st, g, taps, tapw, ntaps, in, Hs,
               out, E0, Emin, penal, h, s_out);
  else
    pdl_launch(k_filter_tiled<T, R, 2, false>, grid, block, 0, st, g, taps, tapw, ntaps, in, Hs,
               out, E0, Emin, penal, h, s_out);
  return true;
}

template <typename T>
cudaError_t launch_filter(cudaStream_t st, Geom g, const int4* taps, const T* tapw, int ntaps,
                          int radius, const T* in, const T* Hs, T* out, int mode, int material,
                          T E0, T Emin, T penal, T h, T* s_out) {
  bool done = false;
  if (radius == 0)
    done = launch_filter_tiled<T, 0>(st, g, taps, tapw, ntaps, in, Hs, out, mode, material, E0,
                                     Emin, penal, h, s_out);
  else if (radius == 1)
    done = launch_filter_tiled<T, 1>(st, g, taps, tapw, ntaps, in, Hs, out, mode, material, E0,
                                     Emin, penal, h, s_out);
  else if (radius == 2)
    done = launch_filter_tiled<T, 2>(st, g, taps, tapw, ntaps, in, Hs, out, mode, material, E0,
                                     Emin, penal, h, s_out);
  else if (radius == 3 && sizeof(T) == 4)
    done = launch_filter_tiled<T, 3>(st, g, taps, tapw, ntaps, in, Hs, out, mode, material, E0,
                                     Emin, penal, h, s_out);
  if constexpr (sizeof(T) == 4) {
    if (!done && radius > 3 && radius <= kFtMaxR) {
      const int W = 2 * radius + 1;
      const size_t smem = sizeof(float) * ((size_t)(kFtX + 2 * radius) * (kFtY + 2 * radius) *
                                               (kFtZ + 2 * radius) + (size_t)W * W * W);
      const dim3 grid((g.nx + kFtX - 1) / kFtX, (g.ny + kFtY - 1) / kFtY,
                      (g.nz + kFtZ - 1) / kFtZ);
      const dim3 block(kFtX, kFtY);
      if (smem <= 200 * 1024 && grid.y <= 65535 && grid.z <= 65535) {
        cudaError_t e;
        if (mode == 0 && material)
          e = launch_wide<0, true>(grid, block, smem, st, g, radius, taps, tapw, ntaps, in, Hs,
                                   out, E0, Emin, penal, h, s_out);
        else if (mode == 0)
          e = launch_wide<0, false>(grid, block, smem, st, g, radius, taps, tapw, ntaps, in, Hs,
                                    out, E0, Emin, penal, h, s_out);
        else if (mode == 1)
          e = launch_wide<1, false>(grid, block, smem, st, g, radius, taps, tapw, ntaps, in, Hs,
                                    out, E0, Emin, penal, h, s_out);
        else
          e = launch_wide<2, false>(grid, block, smem, st, g, radius, taps, tapw, ntaps, in, Hs,
                                    out, E0, Emin, penal, h, s_out);
        return e != cudaSuccess ? e : cudaGetLastError();
      }
    }
  }
  if (done) return cudaGetLastError();
  int blocks = (g.nel + 255) / 256;
  if (blocks > 16384) blocks = 16384;
  if (mode == 0 && material)
    pdl_launch(k_filter<T, 0, true>, blocks, 256, 0, st, g, taps, tapw, ntaps, in, Hs, out, E0, Emin,
                                                 penal, h, s_out);
  else if (mode == 0)
    pdl_launch(k_filter<T, 0, false>, blocks, 256, 0, st, g, taps, tapw, ntaps, in, Hs, out, E0, Emin,
                                                  penal, h, s_out);
  else if (mode == 1)
    pdl_launch(k_filter<T, 1, false>, blocks, 256, 0, st, g, taps, tapw, ntaps, in, Hs, out, E0, Emin,
                                                  penal, h, s_out);
  else
    pdl_launch(k_filter<T, 2, false>, blocks, 256, 0, st, g, taps, tapw, ntaps, in, Hs, out, E0, Emin,
                                                  penal, h, s_out);
  return cudaGetLastError();
}

// s = h (Emin + rho^p (E0 - Emin)) for given physical densities.
template <typename T>
__global__ void k_material(int n, const T* __restrict__ rho, T E0, T Emin, T penal, T h,
                           T* __restrict__ s) {
  PDL_ENTER();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    s[e] = h * (Emin + pow(rho[e], penal) * (E0 - Emin));
}

template <typename T>
cudaError_t launch_material(cudaStream_t st, int n, const T* rho, T E0, T Emin, T penal, T h,
                            T* s) {
  int blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  pdl_launch(k_material<T>, blocks, 256, 0, st, n, rho, E0, Emin, penal, h, s);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Sensitivity (Eq. 5 with the SIMP chain rule): dc_e = -p rho^(p-1) (E0-Emin) h u_e^T K0 u_e.
// u_e^T K0 u_e = sum_k X_k^T blk_k X_k with X the per-component Walsh-Hadamard transform of
// the element's node values minus local node 0 (differences first).
// ---------------------------------------------------------------------------------------
// Per-component Walsh-Hadamard modes of an element's node values minus local node 0 (the
// differences first, so FP32 rounding stays relative to the differences), optionally of
// the unevaluated pair v + vlo.
template <typename T, bool PAIR>
__device__ __forceinline__ void element_modes(const Geom& g, const T* __restrict__ v,
                                              const T* __restrict__ vlo, int i, int j, int k,
                                              T (&X)[3][8]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    T w[8];
    const T* vc = v + (size_t)c * g.nn;
    const T* vlc = PAIR ? vlo + (size_t)c * g.nn : nullptr;
    const int n0 = TOMO_CHK(i + g.nxn * (j + g.nyn * k), g.nn, 15);
    const T a0 = ldg(vc + n0);
    const T al = PAIR ? ldg(vlc + n0) : T(0);
#pragma unroll
    for (int s = 1; s < 8; ++s) {
      const int ns = TOMO_CHK(
          (i + (s & 1)) + g.nxn * ((j + ((s >> 1) & 1)) + g.nyn * (k + (s >> 2))), g.nn, 15);
      T d = ldg(vc + ns) - a0;
      if (PAIR) d += ldg(vlc + ns) - al;
      w[s] = d;
    }
    w[0] = T(0);
#pragma unroll
    for (int st = 1; st < 8; st <<= 1)
#pragma unroll
      for (int s = 0; s < 8; ++s)
        if ((s & st) == 0) {
          const T a = w[s], b = w[s + st];
          w[s] = a + b;
          w[s + st] = a - b;
        }
#pragma unroll
    for (int m = 0; m < 8; ++m) X[c][m] = w[m];
  }
}

// dc_e = -p rho^(p-1) (E0-Emin) h w_e^T K0 u_e with w = u (compliance, Eq. 5) or w = the
// adjoint state lambda (BILIN; the general objective of Eq. 3).  w_e^T K0 u_e = sum_k
// Y_k^T blk_k X_k in the Hadamard basis (X, Y the modes of u, w).
template <typename T, bool PAIR, bool BILIN>
__global__ void k_sensitivity(Geom g, const T* __restrict__ rho, const T* __restrict__ u,
                              const T* __restrict__ ulo, const T* __restrict__ w,
                              const T* __restrict__ wlo, const __grid_constant__ ElemConst<T> C,
                              T penal, T E0, T Emin, T h, T* __restrict__ dc) {
  PDL_ENTER();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.nel; e += gridDim.x * blockDim.x) {
    const int i = e % g.nx, j = (e / g.nx) % g.ny, k = e / (g.nx * g.ny);
    T X[3][8];
    element_modes<T, PAIR>(g, u, ulo, i, j, k, X);
    T Y[3][8];
    if constexpr (BILIN) element_modes<T, PAIR>(g, w, wlo, i, j, k, Y);
    T ce = T(0);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const T x0 = (kk ^ 1) ? X[0][kk ^ 1] : T(0);
      const T x1 = (kk ^ 2) ? X[1][kk ^ 2] : T(0);
      const T x2 = (kk ^ 4) ? X[2][kk ^ 4] : T(0);
      const T y0 = C.blk[kk][0][0] * x0 + C.blk[kk][0][1] * x1 + C.blk[kk][0][2] * x2;
      const T y1 = C.blk[kk][1][0] * x0 + C.blk[kk][1][1] * x1 + C.blk[kk][1][2] * x2;
      const T y2 = C.blk[kk][2][0] * x0 + C.blk[kk][2][1] * x1 + C.blk[kk][2][2] * x2;
      if constexpr (BILIN) {
        const T w0 = (kk ^ 1) ? Y[0][kk ^ 1] : T(0);
        const T w1 = (kk ^ 2) ? Y[1][kk ^ 2] : T(0);
        const T w2 = (kk ^ 4) ? Y[2][kk ^ 4] : T(0);
        ce += w0 * y0 + w1 * y1 + w2 * y2;
      } else {
        ce += x0 * y0 + x1 * y1 + x2 * y2;
      }
    }
    const T r = rho[e];
    dc[e] = -penal * pow(r, penal - T(1)) * (E0 - Emin) * h * ce;
  }
}

template <typename T>
cudaError_t launch_sensitivity(cudaStream_t st, Geom g, const T* rho, const T* u, const T* ulo,
                               const T* w, const T* wlo, const ElemConst<T>& c, T penal, T E0,
                               T Emin, T h, T* dc) {
  int blocks = (g.nel + 127) / 128;
  if (blocks > 16384) blocks = 16384;
  if ((ulo != nullptr) != (w != nullptr && wlo != nullptr) && w != nullptr)
    return cudaErrorInvalidValue;  // u and w must both be pairs or both plain
  if (ulo) {
    if constexpr (sizeof(T) == 4) {
      if (w)
        pdl_launch(k_sensitivity<T, true, true>, blocks, 128, 0, st, g, rho, u, ulo, w, wlo, c,
                   penal, E0, Emin, h, dc);
      else
        pdl_launch(k_sensitivity<T, true, false>, blocks, 128, 0, st, g, rho, u, ulo, w, wlo, c,
                   penal, E0, Emin, h, dc);
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }
  if (w)
    pdl_launch(k_sensitivity<T, false, true>, blocks, 128, 0, st, g, rho, u, nullptr, w, nullptr,
               c, penal, E0, Emin, h, dc);
  else
    pdl_launch(k_sensitivity<T, false, false>, blocks, 128, 0, st, g, rho, u, nullptr, nullptr,
               nullptr, c, penal, E0, Emin, h, dc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Optimality criteria (Section III-D).  With q_e = z_e sqrt(max(-dc_e, 0)/w_e), the update at
// multiplier lam is z_new = clamp(q_e lam^-1/2, max(0, z-m), min(1, z+m)) and the filtered
// volume is V(lam) = sum_e w_e z_new_e, non-increasing in lam.  lam is searched in log2
// space on [-100, 100]: each pass evaluates kOcCand candidates spread over the current
// bracket and keeps the cell where V crosses V_max, shrinking the bracket kOcCand-1 fold,
// until its relative width is below 1e-10; the update uses the bracket's centre.
// ---------------------------------------------------------------------------------------
constexpr int kOcCand = 32;
constexpr int kOcThreads = 256;
constexpr int kOcPerThread = 8;

template <typename T>
__global__ void __launch_bounds__(kOcThreads)
    k_oc_pass(int n, const T* __restrict__ z, const T* __restrict__ dc, const T* __restrict__ w,
              double vmax, T move, double* bracket, double* partials, unsigned* counter,
              int first) {
  PDL_ENTER();
  __shared__ T s_scale[kOcCand];
  __shared__ double s_w[kOcThreads / 32][kOcCand];
  __shared__ bool s_last;
  // the first pass starts from the full search range; later passes read the bracket the
  // previous pass left
  const double a = first ? -100.0 : bracket[0], b = first ? 100.0 : bracket[1];
  if (a >= b) return;  // converged (uniform across the grid)
  if (threadIdx.x < kOcCand) {
    const double e = a + (b - a) * (double)threadIdx.x / (double)(kOcCand - 1);
    s_scale[threadIdx.x] = (T)exp2(-0.5 * e);
  }
  __syncthreads();
  T acc[kOcCand];
#pragma unroll
  for (int t = 0; t < kOcCand; ++t) acc[t] = T(0);
  const int base = (blockIdx.x * kOcThreads) * kOcPerThread + threadIdx.x;
#pragma unroll
  for (int u = 0; u < kOcPerThread; ++u) {
    const int e = base + u * kOcThreads;
    if (e < n) {
      const T ze = z[e], we = w[e];
      const T neg = dc[e] < T(0) ? -dc[e] : T(0);
      const T q = ze * sqrt(neg / we);
      const T lo = ze - move > T(0) ? ze - move : T(0);
      const T hi = ze + move < T(1) ? ze + move : T(1);
#pragma unroll
      for (int t = 0; t < kOcCand; ++t) {
        T zt = q * s_scale[t];
        zt = zt < lo ? lo : (zt > hi ? hi : zt);
        acc[t] += we * zt;
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kOcCand; ++t) {
    T v = acc[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_w[wid][t] = (double)v;
  }
  __syncthreads();
  if (threadIdx.x < kOcCand) {
    double s = 0.0;
    for (int q = 0; q < kOcThreads / 32; ++q) s += s_w[q][threadIdx.x];
    partials[(size_t)blockIdx.x * kOcCand + threadIdx.x] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: totals in block order, then the new bracket
  __shared__ double s_tot[kOcCand];
  {
    // thread (t, part): candidate t, blocks part, part + 8, ...; then fixed-order sum
    const int t = threadIdx.x % kOcCand, part = threadIdx.x / kOcCand;
    constexpr int parts = kOcThreads / kOcCand;
    double s = 0.0;
    for (unsigned q = part; q < gridDim.x; q += parts)
      s += __ldcg(partials + (size_t)q * kOcCand + t);
    s_w[part][t] = s;
    __syncthreads();
    if (threadIdx.x < kOcCand) {
      double tot = 0.0;
      for (int q = 0; q < parts; ++q) tot += s_w[q][threadIdx.x];
      s_tot[threadIdx.x] = tot;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *counter = 0u;
    int t = 0;
    while (t < kOcCand && s_tot[t] > vmax) ++t;
    double na, nb;
    if (t == 0) { na = a; nb = a; }                        // root at or below a
    else if (t == kOcCand) { na = b; nb = b; }             // V(b) > Vmax: root at or above b
    else {
      na = a + (b - a) * (double)(t - 1) / (double)(kOcCand - 1);
      nb = a + (b - a) * (double)t / (double)(kOcCand - 1);
    }
    // relative width of the lam bracket: 2^(nb-na) - 1 ~ (nb-na) ln 2
    if ((nb - na) * 0.6931471805599453 <= 1e-10) { na = nb = 0.5 * (na + nb); }
    bracket[0] = na;
    bracket[1] = nb;
  }
}

template <typename T>
__global__ void __launch_bounds__(kOcThreads)
    k_oc_final(int n, const T* __restrict__ z, const T* __restrict__ dc, const T* __restrict__ w,
               T move, const double* bracket, T* __restrict__ znew, double* partials,
               unsigned* counter, double* change_out) {
  PDL_ENTER();
  __shared__ float s_m[kOcThreads / 32];
  __shared__ bool s_last;
  const double ec = 0.5 * (bracket[0] + bracket[1]);
  const T scale = (T)exp2(-0.5 * ec);
  float mx = 0.0f;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const T ze = z[e], we = w[e];
    const T neg = dc[e] < T(0) ? -dc[e] : T(0);
    const T q = ze * sqrt(neg / we);
    const T lo = ze - move > T(0) ? ze - move : T(0);
    const T hi = ze + move < T(1) ? ze + move : T(1);
    T zt = q * scale;
    zt = zt < lo ? lo : (zt > hi ? hi : zt);
    znew[e] = zt;
    const float d = (float)(zt > ze ? zt - ze : ze - zt);
    mx = fmaxf(mx, d);
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.0f;
    for (int q = 0; q < kOcThreads / 32; ++q) m = fmaxf(m, s_m[q]);
    partials[blockIdx.x] = (double)m;
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  float m = 0.0f;
  for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x)
    m = fmaxf(m, (float)__ldcg(partials + q));
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float mm = 0.0f;
    for (int q = 0; q < kOcThreads / 32; ++q) mm = fmaxf(mm, s_m[q]);
    *change_out = (double)mm;
    *counter = 0u;
  }
}

// The change is reduced in float; for FP64 grids it is recomputed exactly below.
template <typename T>
__global__ void k_oc_change64(int n, const T* __restrict__ z, const T* __restrict__ znew,
                              double* partials, unsigned* counter, double* change_out) {
  PDL_ENTER();
  __shared__ double s_m[kOcThreads / 32];
  __shared__ bool s_last;
  double mx = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    mx = fmax(mx, fabs((double)znew[e] - (double)z[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int q = 0; q < kOcThreads / 32; ++q) m = fmax(m, s_m[q]);
    partials[blockIdx.x] = m;
    __threadfence();
    const unsigned t = atomicAdd(counter, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double m = 0.0;
  for (unsigned q = threadIdx.x; q < gridDim.x; q += blockDim.x) m = fmax(m, __ldcg(partials + q));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = 0.0;
    for (int q = 0; q < kOcThreads / 32; ++q) mm = fmax(mm, s_m[q]);
    *change_out = mm;
    *counter = 0u;
  }
}

template <typename T>
cudaError_t launch_oc(cudaStream_t st, int n, const T* z, const T* dc, const T* w, double vmax,
                      double move, T* znew, double* partials, unsigned* counter,
                      double* bracket, double* change_out, int max_blocks) {
  const int per_block = kOcThreads * kOcPerThread;
  const int blocks = (n + per_block - 1) / per_block;
  if (blocks > max_blocks) return cudaErrorInvalidValue;
  // 31^9 > 200 / (1e-10 / ln 2): nine passes always reach the tolerance
  for (int pass = 0; pass < 9; ++pass)
    pdl_launch(k_oc_pass<T>, blocks, kOcThreads, 0, st, n, z, dc, w, vmax, (T)move, bracket,
               partials, counter, pass == 0 ? 1 : 0);
  int fb = (n + kOcThreads - 1) / kOcThreads;
  if (fb > 2 * 152 * 4) fb = 2 * 152 * 4;
  pdl_launch(k_oc_final<T>, fb, kOcThreads, 0, st, n, z, dc, w, (T)move, bracket, znew, partials,
                                           counter, change_out);
  if (sizeof(T) == 8)
    pdl_launch(k_oc_change64<T>, fb, kOcThreads, 0, st, n, z, znew, partials, counter, change_out);
  return cudaGetLastError();
}

int oc_partials_needed(int n) {
  const int per_block = kOcThreads * kOcPerThread;
  const int blocks = (n + per_block - 1) / per_block;
  const int a = blocks * kOcCand;
  const int b = 2 * 152 * 4;
  return a > b ? a : b;
}

int oc_max_blocks(int n) {
  const int per_block = kOcThreads * kOcPerThread;
  return (n + per_block - 1) / per_block;
}

#define INST(T)                                                                                \
  template cudaError_t launch_filter<T>(cudaStream_t, Geom, const int4*, const T*, int, int,   \
                                        const T*, const T*, T*, int, int, T, T, T, T, T*);     \
  template cudaError_t launch_material<T>(cudaStream_t, int, const T*, T, T, T, T, T*);       \
  template cudaError_t launch_sensitivity<T>(cudaStream_t, Geom, const T*, const T*, const T*, \
                                             const T*, const T*, const ElemConst<T>&, T, T, T, \
                                             T, T*);                                           \
  template cudaError_t launch_oc<T>(cudaStream_t, int, const T*, const T*, const T*, double,   \
                                    double, T*, double*, unsigned*, double*, double*, int);
INST(float)
INST(double)
#undef INST

#ifdef TOMO_CHECKED
TOMO_CHECK_ACCESSOR(check_word_filt)
#endif

}  // namespace tomo
