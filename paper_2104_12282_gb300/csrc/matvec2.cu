// FP32 matrix-free hex8 product and Chebyshev smoother step, two node rows per thread in
// packed FP32x2 arithmetic (state equation of Eq. 4, Section III-D; K = sum_e s_e K0).
//
// Same operator and the same differences-first accuracy as k_march, fewer instructions:
// * a thread owns node column i and node rows (j0, j0+1) and evaluates the two elements
//   (i, j0, k) and (i, j0+1, k) at once, one in each half of a float2;
// * the Walsh-Hadamard modes of an element come from its twelve edge differences
//   (x-, y- and z-edges), each a difference of neighbouring node values, so FP32 rounding
//   stays relative to displacement differences;
// * K0 acts in the mode basis through its four block kinds (see element.cu), 41 packed
//   operations for the pair of elements;
// * the inverse transform is staged: its x-stage runs per element, the sx = 1 halves go to
//   lane i+1 by shuffle, the y-stage runs on the summed node-column values, the sy = 1 half
//   of the upper element goes to the next thread row through shared memory, the z-stage
//   splits plane k (output) from plane k+1 (carried in registers).
// CTA = 32 lanes x 8 thread rows = node columns 32 x 16; lanes 0, 31 and node rows 0, 15
// are halo.  Each z-chunk recomputes one element layer below it.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "host.h"
#include "march2_body.cuh"

namespace tomo {

namespace {

template <int MODE, bool DOT>
__global__ void __launch_bounds__(32 * TYP, TOMO_MARCH2_MIN_BLOCKS)
    k_march2(const __grid_constant__ March2Args A, const __grid_constant__ March2Const K) {
  march2_body<MODE, DOT>(A, K, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.x,
                         blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                         gridDim.x * gridDim.y * gridDim.z, threadIdx.x, threadIdx.y);
}

// The same operation for several grids in one launch: block b belongs to grid q with
// cta0[q] <= b < cta0[q+1] and is that grid's block b - cta0[q] in the order of k_march2's
// (x, y, z) grid, so each grid sees exactly the blocks (and the dot partials) of its own
// launch.
// TY thread rows per CTA: 8 as k_march2, or 4 (tiles of 6 element rows, for batches of
// small grids whose y extent the 14-row tile covers poorly; chosen by measurement).
template <int MODE, bool DOT, int TY>
__global__ void __launch_bounds__(32 * TY, TOMO_MARCH2_MIN_BLOCKS * TYP / TY)
    k_march2_batch(const __grid_constant__ March2Batch B, const __grid_constant__ March2Const K) {
  const int q = batch_owner(B.cta0, B.n, (int)blockIdx.x);
  const int loc = (int)blockIdx.x - B.cta0[q];
  const int gx = B.gx[q], gy = B.gy[q];
  march2_body<MODE, DOT, true, TY>(B.a[q], K, loc % gx, (loc / gx) % gy, loc / (gx * gy), gx,
                                   (unsigned)loc, (unsigned)(B.cta0[q + 1] - B.cta0[q]),
                                   threadIdx.x, threadIdx.y);
}

template <int TY>
cudaError_t launch_march2_batch_ty(cudaStream_t st, int mode, bool dot, int ctas,
                                   const March2Batch& B, const March2Const& c) {
  dim3 grid(ctas), block(32, TY);
  if (mode == M_APPLY) {
    if (dot) pdl_launch(k_march2_batch<M_APPLY, true, TY>, grid, block, 0, st, B, c);
    else pdl_launch(k_march2_batch<M_APPLY, false, TY>, grid, block, 0, st, B, c);
  } else if (mode == M_RESID) {
    if (dot) return cudaErrorInvalidValue;
    pdl_launch(k_march2_batch<M_RESID, false, TY>, grid, block, 0, st, B, c);
  } else {
    if (dot) pdl_launch(k_march2_batch<M_CHEB, true, TY>, grid, block, 0, st, B, c);
    else pdl_launch(k_march2_batch<M_CHEB, false, TY>, grid, block, 0, st, B, c);
  }
  return cudaGetLastError();
}

}  // namespace

std::vector<uint8_t> march2_tile_flags(const Geom& g, const std::vector<uint8_t>& hmask) {
  const int gx = (g.nxn + 29) / 30;
  const int gy = (g.nyn + 2 * TYP - 3) / (2 * TYP - 2);
  std::vector<uint8_t> f((size_t)gx * gy, 0);
  for (int k = 0; k < g.nzn; ++k)
    for (int j = 0; j < g.nyn; ++j)
      for (int i = 0; i < g.nxn; ++i) {
        if (!hmask[(size_t)i + (size_t)g.nxn * (j + (size_t)g.nyn * k)]) continue;
        // every tile whose node columns (halo included) contain (i, j)
        for (int bx = std::max(0, (i - 30) / 30); bx <= std::min(gx - 1, (i + 1) / 30); ++bx) {
          if (i < bx * 30 - 1 || i > bx * 30 + 30) continue;
          for (int by = std::max(0, (j - 14) / 14); by <= std::min(gy - 1, (j + 1) / 14); ++by)
            if (j >= by * 14 - 1 && j <= by * 14 + 14) f[bx + (size_t)gx * by] = 1;
        }
      }
  return f;
}

namespace {

struct March2Shape {
  int gx, gy, kz, nzc;
};

// Tiles and z-chunks of one grid's launch (the same for a single and a batched launch, so
// that a grid's arithmetic does not depend on how it was launched).
March2Shape march2_shape(int mode, bool dot, const Geom& g, int num_sms) {
  March2Shape m;
  m.gx = (g.nxn + 29) / 30;
  m.gy = (g.nyn + 2 * TYP - 3) / (2 * TYP - 2);
  const int tiles = m.gx * m.gy;
  // one wave of resident CTAs (occupancy of the single-grid instance)
  int per_sm = 0;
  cudaError_t oe;
  if (mode == M_APPLY)
    oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, dot ? k_march2<M_APPLY, true> : k_march2<M_APPLY, false>, 32 * TYP, 0);
  else if (mode == M_RESID)
    oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_march2<M_RESID, false>,
                                                       32 * TYP, 0);
  else
    oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, dot ? k_march2<M_CHEB, true> : k_march2<M_CHEB, false>, 32 * TYP, 0);
  if (oe != cudaSuccess) cudaGetLastError();
  if (oe != cudaSuccess || per_sm < 1) per_sm = 2;
  const int target = per_sm * (num_sms > 0 ? num_sms : 152);
  // Each CTA marches kz + 1 element layers one after another, so a launch takes at least
  // (kz + 1) step latencies.  Large grids fill one wave with long chunks (little halo);
  // grids too small to fill the GPU take the shortest chunks that still fit in one wave.
  int kz = (int)(((long long)g.nzn * tiles + target - 1) / target);
  if (kz < 1) kz = 1;
  if (kz > g.nzn) kz = g.nzn;
  m.kz = kz;
  m.nzc = (g.nzn + kz - 1) / kz;
  return m;
}

}  // namespace

cudaError_t launch_march2_batch(cudaStream_t st, int mode, const March2Args* a, int n,
                                const March2Const& c, int num_sms, int ty) {
  if (n <= 0) return cudaSuccess;
  if (ty != TYP && ty != 4) return cudaErrorInvalidValue;
  const bool dot = a[0].dot_kind != 0;
  for (int q = 0; q < n; ++q)
    if ((a[q].dot_kind != 0) != dot) return cudaErrorInvalidValue;
  for (int q0 = 0; q0 < n; q0 += kBatchMax) {
    March2Batch B{};
    B.n = std::min(kBatchMax, n - q0);
    int ctas = 0;
    for (int q = 0; q < B.n; ++q) {
      March2Shape m = march2_shape(mode, dot, a[q0 + q].g, num_sms);
      if (a[q0 + q].kz > 0) {  // z-chunk length chosen by the caller for the whole batch
        m.kz = std::min(a[q0 + q].kz, a[q0 + q].g.nzn);
        m.nzc = (a[q0 + q].g.nzn + m.kz - 1) / m.kz;
      }
      B.a[q] = a[q0 + q];
      B.a[q].kz = m.kz;
      if (ty != TYP) {
        m.gy = (a[q0 + q].g.nyn + 2 * ty - 3) / (2 * ty - 2);
        B.a[q].tile_fixed = nullptr;  // the flags are per TYP-row tile: test every mask
      }
      B.gx[q] = m.gx;
      B.gy[q] = m.gy;
      B.cta0[q] = ctas;
      ctas += m.gx * m.gy * m.nzc;
    }
    B.cta0[B.n] = ctas;
    if (g_phase_rec) {  // recorded for the persistent lockstep iteration (TYP rows)
      if ((mode == M_RESID && dot) || ty != TYP) return cudaErrorInvalidValue;
      const int kind = mode == M_APPLY ? (dot ? PH_M2_APPLY_DOT : PH_M2_APPLY)
                       : mode == M_RESID ? PH_M2_RESID
                                         : (dot ? PH_M2_CHEB_DOT : PH_M2_CHEB);
      record_phase(kind, ctas, B, q0 > 0);
      continue;
    }
    const cudaError_t e = ty == TYP ? launch_march2_batch_ty<TYP>(st, mode, dot, ctas, B, c)
                                    : launch_march2_batch_ty<4>(st, mode, dot, ctas, B, c);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_march2(cudaStream_t st, int mode, const March2Args& a, const March2Const& c,
                          int num_sms) {
  const Geom& g = a.g;
  March2Args args = a;
  const March2Shape m = march2_shape(mode, a.dot_kind != 0, g, num_sms);
  const int gx = m.gx, gy = m.gy, nzc = m.nzc;
  args.kz = m.kz;
  dim3 grid(gx, gy, nzc), block(32, TYP);
  const bool dot = a.dot_kind != 0;
  if (mode == M_APPLY) {
    if (dot) pdl_launch(k_march2<M_APPLY, true>, grid, block, 0, st, args, c);
    else pdl_launch(k_march2<M_APPLY, false>, grid, block, 0, st, args, c);
  } else if (mode == M_RESID) {
    pdl_launch(k_march2<M_RESID, false>, grid, block, 0, st, args, c);
  } else {
    if (dot) pdl_launch(k_march2<M_CHEB, true>, grid, block, 0, st, args, c);
    else pdl_launch(k_march2<M_CHEB, false>, grid, block, 0, st, args, c);
  }
  return cudaGetLastError();
}

#ifdef TOMO_CHECKED
TOMO_CHECK_ACCESSOR(check_word_matvec2)
#endif

}  // namespace tomo
