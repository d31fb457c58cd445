// Matrix-free hex8 stiffness product y = K(rho) x and the multigrid smoother step built on
// it (state equation of Eq. 4, Section III-D).  K = sum_e s_e K0 with s_e = h E_e.
//
// Design (GB300): one thread per node column (i, j), marching along z through the node
// planes of a z-chunk.  A CTA is 32 lanes (x) by kTY rows (y).  Element (i, j, k) is
// evaluated by thread (i, j) from the raw 2x2x2 block of node values:
//   own column (planes k, k+1, registers), row j+1 (shared memory), lane i+1 (shuffle).
// Per element, per component, the 8 node values minus the value at local node 0 are
// transformed by an 8-point Walsh-Hadamard transform (differences first, so FP32 rounding
// is relative to the displacement differences, not to the displacements), multiplied by
// K0's eight 3x3 Hadamard-basis blocks scaled by s_e, and transformed back to the eight
// corner forces.  Corner forces reach their nodes without atomics: +x corners by shuffle,
// +y corners through shared memory, +z corners carried in registers to the next plane.
// Lanes 0 and 31 and rows 0 and kTY-1 are halo (their outputs are not written); each
// z-chunk recomputes one element layer below it.
#include <algorithm>

#include "common.cuh"
#include "host.h"
#include "march_body.cuh"

namespace tomo {

template <typename T, int MODE, bool PAIR, bool DOT>
__global__ void __launch_bounds__(32 * kTY, sizeof(T) == 4 ? 2 : 1)
    k_march(const __grid_constant__ MarchArgs<T> A, const __grid_constant__ ElemConst<T> C) {
  march_body<T, MODE, PAIR, DOT>(A, C, blockIdx.x, blockIdx.y, blockIdx.z,
                                 blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z),
                                 gridDim.x * gridDim.y * gridDim.z, threadIdx.x, threadIdx.y);
}

// The FP64 residual of a float pair (r = f - K (x_hi + x_lo), gated residual replacement)
// for several grids in one launch; block b belongs to grid q with cta0[q] <= b < cta0[q+1].
__global__ void __launch_bounds__(32 * kRrTY, 1)
    k_march_rr_batch(const __grid_constant__ MarchRrBatch B,
                     const __grid_constant__ ElemConst<double> C) {
  const int q = batch_owner(B.cta0, B.n, (int)blockIdx.x);
  const int loc = (int)blockIdx.x - B.cta0[q];
  const int gx = B.gx[q], gy = B.gy[q];
  march_body<double, M_RESID, true, false, kRrTY>(B.a[q], C, loc % gx, (loc / gx) % gy,
                                                  loc / (gx * gy), (unsigned)loc,
                                                  (unsigned)(B.cta0[q + 1] - B.cta0[q]),
                                                  threadIdx.x, threadIdx.y);
}

namespace {

struct MarchShape {
  int gx, gy, kz, nzc;
};

template <typename T>
MarchShape march_shape(const Geom& g, int num_sms, int ty = kTY) {
  MarchShape m;
  m.gx = (g.nxn + 29) / 30;
  m.gy = (g.nyn + ty - 3) / (ty - 2);
  // z-chunks: about one full wave of resident CTAs (2 per SM), chunks of >= 4 planes
  const int tiles = m.gx * m.gy;
  const int target = (sizeof(T) == 4 ? 2 : 1) * (num_sms > 0 ? num_sms : 152);
  int nzc = target / tiles;
  if (nzc < 1) nzc = 1;
  int kz = (g.nzn + nzc - 1) / nzc;
  if (kz < 4) kz = 4;
  if (kz > g.nzn) kz = g.nzn;
  m.kz = kz;
  m.nzc = (g.nzn + kz - 1) / kz;
  return m;
}

}  // namespace

cudaError_t launch_march_rr_batch(cudaStream_t st, const MarchArgs<double>* a, int n,
                                  const ElemConst<double>& c, int num_sms) {
  for (int q0 = 0; q0 < n; q0 += kBatchMax) {
    MarchRrBatch B{};
    B.n = std::min(kBatchMax, n - q0);
    int ctas = 0;
    for (int q = 0; q < B.n; ++q) {
      const MarchShape m = march_shape<double>(a[q0 + q].g, num_sms, kRrTY);
      B.a[q] = a[q0 + q];
      B.a[q].kz = m.kz;
      B.gx[q] = m.gx;
      B.gy[q] = m.gy;
      B.cta0[q] = ctas;
      ctas += m.gx * m.gy * m.nzc;
    }
    B.cta0[B.n] = ctas;
    if (g_phase_rec) {  // recorded for the persistent lockstep iteration
      record_phase(PH_RR, ctas, B, q0 > 0);
      continue;
    }
    pdl_launch(k_march_rr_batch, dim3(ctas), dim3(32, kRrTY), 0, st, B, c);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_march(cudaStream_t st, int mode, const MarchArgs<T>& a, const ElemConst<T>& c,
                         int num_sms, int* grid_ctas) {
  const Geom& g = a.g;
  MarchArgs<T> args = a;
  const MarchShape m = march_shape<T>(g, num_sms);
  const int gx = m.gx, gy = m.gy, nzc = m.nzc;
  args.kz = m.kz;
  dim3 grid(gx, gy, nzc), block(32, kTY);
  if (grid_ctas) *grid_ctas = gx * gy * nzc;
  const bool pair = sizeof(T) == 4 ? a.xlo != nullptr : a.xf_hi != nullptr;
  const bool dot = a.dot_kind != 0;
  if (mode == M_APPLY) {
    if (dot) pdl_launch(k_march<T, M_APPLY, false, true>, grid, block, 0, st, args, c);
    else pdl_launch(k_march<T, M_APPLY, false, false>, grid, block, 0, st, args, c);
  } else if (mode == M_RESID) {
    if (pair) pdl_launch(k_march<T, M_RESID, true, false>, grid, block, 0, st, args, c);
    else pdl_launch(k_march<T, M_RESID, false, false>, grid, block, 0, st, args, c);
  } else {
    if (dot) pdl_launch(k_march<T, M_CHEB, false, true>, grid, block, 0, st, args, c);
    else pdl_launch(k_march<T, M_CHEB, false, false>, grid, block, 0, st, args, c);
  }
  return cudaGetLastError();
}

template cudaError_t launch_march<float>(cudaStream_t, int, const MarchArgs<float>&,
                                         const ElemConst<float>&, int, int*);
template cudaError_t launch_march<double>(cudaStream_t, int, const MarchArgs<double>&,
                                          const ElemConst<double>&, int, int*);

#ifdef TOMO_CHECKED
TOMO_CHECK_ACCESSOR(check_word_matvec)
#endif

}  // namespace tomo
