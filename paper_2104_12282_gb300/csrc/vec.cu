// Multigrid transfers, coarse operators, the coarsest dense solve, CG recurrences and
// reductions.  The solve of the state equation of Eq. 4 (Section III-D) is preconditioned
// CG, the standard solver the paper names (PCG; multigrid is the stated alternative).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "host.h"
#include "march2_body.cuh"
#include "march_body.cuh"

namespace tomo {

constexpr int kRedBlocks = 304;  // reduction grid (2 x 152 SMs)
// float4 groups a thread loads before using them (the x/r update moves five arrays per
// group, the p update two)
constexpr int kIlpXr = 2, kIlpP = 4;
constexpr int kRedThreads = 256;

__device__ __forceinline__ bool skipped(const int* skip) { return skip != nullptr && *skip; }

// ---------------------------------------------------------------------------------------
// First Chebyshev step from a zero guess: x1 = c2 D^-1 b, x0 = 0.  D = k0diag * (sum of s_e
// over the elements around the node) is the diagonal of K (all three components equal).
// Optional dot b.x1 for the Jacobi-preconditioned CG (dot_kind 2).
// ---------------------------------------------------------------------------------------
// (vb, vnb): the block's index and the block count of this grid's launch (grid-stride loop
// and dot partials); batched launches pass a block's place within its grid.
template <typename T, bool DOT>
__device__ __forceinline__ void jacobi_body(int vb, int vnb, Geom g, const T* __restrict__ s,
                                            const uint8_t* __restrict__ mask,
                                            const T* __restrict__ b, T c2, T k0diag,
                                            T* __restrict__ x1, T* __restrict__ x0,
                                            double* partials, unsigned* counter,
                                            CgScalars* sc, const int* skip,
                                            T* __restrict__ invd = nullptr) {
  PDL_ENTER();
  if (skipped(skip)) return;
  double dot = 0.0;       // FP64 grids
  FloatPairSum dotf;      // FP32 grids
  for (int n = vb * blockDim.x + threadIdx.x; n < g.nn; n += vnb * blockDim.x) {
    const int i = n % g.nxn, j = (n / g.nxn) % g.nyn, k = n / (g.nxn * g.nyn);
    // the (up to) eight elements around the node: indices clamped, absent ones weighted 0
    const int xa = max(i - 1, 0), xb = min(i, g.nx - 1);
    const int ya = g.nx * max(j - 1, 0), yb = g.nx * min(j, g.ny - 1);
    const int za = g.nx * g.ny * max(k - 1, 0), zb = g.nx * g.ny * min(k, g.nz - 1);
    const T wxa = i > 0 ? T(1) : T(0), wxb = i < g.nx ? T(1) : T(0);
    const T wya = j > 0 ? T(1) : T(0), wyb = j < g.ny ? T(1) : T(0);
    const T wza = k > 0 ? T(1) : T(0), wzb = k < g.nz ? T(1) : T(0);
    auto row = [&](int off) {
      return wxa * s[TOMO_CHK(off + xa, g.nel, 7)] + wxb * s[TOMO_CHK(off + xb, g.nel, 7)];
    };
    const T S = wza * (wya * row(za + ya) + wyb * row(za + yb)) +
                wzb * (wya * row(zb + ya) + wyb * row(zb + yb));
    const T dg = k0diag * S;
    if (invd) invd[n] = dg > T(0) ? T(1) / dg : T(0);  // kept for the fused later steps
    const unsigned mk = mask[n];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const size_t idx = (size_t)c * g.nn + n;
      const T bv = b[idx];
      const T v = (((mk >> c) & 1u) || !(dg > T(0))) ? T(0) : c2 * bv / dg;
      x1[idx] = v;
      if (x0) x0[idx] = T(0);
      if (DOT) {
        if constexpr (sizeof(T) == 4) dotf.add(__fmul_rn(bv, v));
        else dot += bv * v;
      }
    }
  }
  if (DOT) {
    if constexpr (sizeof(T) == 4) dot = dotf.value();
    double v[1] = {dot};
    grid_reduce_at<1>(v, partials, counter, [sc](const double* tot) {
      sc->rz_new = tot[0];
      if (!isfinite(tot[0])) { sc->status |= DEV_NAN; sc->done = 1; }
      sc->beta = sc->rz != 0.0 ? tot[0] / sc->rz : 0.0;
      sc->rz = tot[0];
    }, vb, vnb);
  }
}

template <typename T, bool DOT>
__global__ void k_jacobi(Geom g, const T* __restrict__ s, const uint8_t* __restrict__ mask,
                         const T* __restrict__ b, T c2, T k0diag, T* __restrict__ x1,
                         T* __restrict__ x0, double* partials, unsigned* counter, CgScalars* sc,
                         const int* skip, T* __restrict__ invd) {
  jacobi_body<T, DOT>(blockIdx.x, gridDim.x, g, s, mask, b, c2, k0diag, x1, x0, partials,
                      counter, sc, skip, invd);
}

template <typename T>
cudaError_t launch_jacobi(cudaStream_t st, Geom g, const T* s, const uint8_t* mask, const T* b,
                          T c2, T k0diag, T* x1, T* x0zero, double* partials,
                          unsigned* counter, CgScalars* sc, int dot_kind, const int* skip,
                          T* invd) {
  int blocks = (g.nn + 255) / 256;
  if (dot_kind) {
    if (blocks > kRedBlocks) blocks = kRedBlocks;
    pdl_launch(k_jacobi<T, true>, blocks, 256, 0, st, g, s, mask, b, c2, k0diag, x1, x0zero,
               partials, counter, sc, skip, invd);
  } else {
    if (blocks > 4096) blocks = 4096;
    pdl_launch(k_jacobi<T, false>, blocks, 256, 0, st, g, s, mask, b, c2, k0diag, x1, x0zero,
               nullptr, nullptr, nullptr, skip, invd);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Restriction r_c = P^T r_f (trilinear, weights 1, 1/2 per axis), masked on the coarse grid.
// Fine node i maps to coarse node i/2 (even) or to (i-1)/2 and (i+1)/2 (odd).
// ---------------------------------------------------------------------------------------
// Optionally fused with the first (zero-start) Chebyshev step on the coarse level:
// x1 = c2 D^-1 r_c, D from the coarse moduli sc.
template <typename T>
__device__ __forceinline__ void restrict_body(int vb, int vnb, Geom gf, Geom gc,
                                              const T* __restrict__ rf, T* __restrict__ rc,
                                              const uint8_t* __restrict__ mask_c,
                                              const int* skip, T* __restrict__ x1,
                                              const T* __restrict__ sc, T c2, T k0diag) {
  PDL_ENTER();
  if (skipped(skip)) return;
  for (int n = vb * blockDim.x + threadIdx.x; n < gc.nn; n += vnb * blockDim.x) {
    const int I = n % gc.nxn, J = (n / gc.nxn) % gc.nyn, K = n / (gc.nxn * gc.nyn);
    // fine indices 2I-1, 2I, 2I+1 per axis with weights 1/2, 1, 1/2; indices outside the
    // fine grid are clamped and weighted 0 (same code path for every node)
    int ix[3], iy[3], iz[3];
    T wx[3], wy[3], wz[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int a = 2 * I + d - 1, b = 2 * J + d - 1, e = 2 * K + d - 1;
      const T w = d == 1 ? T(1) : T(0.5);
      wx[d] = (a >= 0 && a < gf.nxn) ? w : T(0);
      wy[d] = (b >= 0 && b < gf.nyn) ? w : T(0);
      wz[d] = (e >= 0 && e < gf.nzn) ? w : T(0);
      ix[d] = min(max(a, 0), gf.nxn - 1);
      iy[d] = gf.nxn * min(max(b, 0), gf.nyn - 1);
      iz[d] = gf.nxn * gf.nyn * min(max(e, 0), gf.nzn - 1);
    }
    T acc[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* v = rf + (size_t)c * gf.nn;
#pragma unroll
      for (int dz = 0; dz < 3; ++dz) {
        T az = T(0);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          const int row = iz[dz] + iy[dy];
          const T ay = wx[0] * v[TOMO_CHK(row + ix[0], gf.nn, 8)] +
                       wx[1] * v[TOMO_CHK(row + ix[1], gf.nn, 8)] +
                       wx[2] * v[TOMO_CHK(row + ix[2], gf.nn, 8)];
          az += wy[dy] * ay;
        }
        acc[c] += wz[dz] * az;
      }
    }
    const unsigned mk = mask_c[n];
#pragma unroll
    for (int c = 0; c < 3; ++c) rc[(size_t)c * gc.nn + n] = ((mk >> c) & 1u) ? T(0) : acc[c];
    if (x1 != nullptr) {
      T S = T(0);
      for (int dz = -1; dz <= 0; ++dz)
        for (int dy = -1; dy <= 0; ++dy)
          for (int dx = -1; dx <= 0; ++dx) {
            const int ei = I + dx, ej = J + dy, ek = K + dz;
            if (ei >= 0 && ei < gc.nx && ej >= 0 && ej < gc.ny && ek >= 0 && ek < gc.nz)
              S += sc[TOMO_CHK(ei + gc.nx * (ej + gc.ny * ek), gc.nel, 8)];
          }
      const T dg = k0diag * S;
#pragma unroll
      for (int c = 0; c < 3; ++c)
        x1[(size_t)c * gc.nn + n] = (((mk >> c) & 1u) || !(dg > T(0))) ? T(0) : c2 * acc[c] / dg;
    }
  }
}

template <typename T>
__global__ void k_restrict(Geom gf, Geom gc, const T* __restrict__ rf, T* __restrict__ rc,
                           const uint8_t* __restrict__ mask_c, const int* skip,
                           T* __restrict__ x1, const T* __restrict__ sc, T c2, T k0diag) {
  restrict_body<T>(blockIdx.x, gridDim.x, gf, gc, rf, rc, mask_c, skip, x1, sc, c2, k0diag);
}

template <typename T>
cudaError_t launch_restrict(cudaStream_t st, Geom gf, Geom gc, const T* rf, T* rc,
                            const uint8_t* mask_c, const int* skip, T* x1, const T* sc, T c2,
                            T k0diag) {
  int blocks = (gc.nn + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  pdl_launch(k_restrict<T>, blocks, 256, 0, st, gf, gc, rf, rc, mask_c, skip, x1, sc, c2, k0diag);
  return cudaGetLastError();
}

// x_f += P x_c (trilinear interpolation), masked on the fine grid.  Every fine node takes
// the same 2x2x2 form (an even index uses one coarse node with weights 1 and 0), so the
// warp does not diverge on index parity.
template <typename T>
__device__ __forceinline__ void prolong_body(int vb, int vnb, Geom gf, Geom gc,
                                             const T* __restrict__ xc, T* __restrict__ xf,
                                             const uint8_t* __restrict__ mask_f,
                                             const int* skip) {
  PDL_ENTER();
  if (skipped(skip)) return;
  for (int n = vb * blockDim.x + threadIdx.x; n < gf.nn; n += vnb * blockDim.x) {
    const int i = n % gf.nxn, j = (n / gf.nxn) % gf.nyn, k = n / (gf.nxn * gf.nyn);
    const int i0 = i >> 1, i1 = (i + 1) >> 1;
    const int j0 = j >> 1, j1 = (j + 1) >> 1;
    const int k0 = k >> 1, k1 = (k + 1) >> 1;
    const T h = T(0.5);
    const T wi0 = (i & 1) ? h : T(1), wi1 = (i & 1) ? h : T(0);
    const T wj0 = (j & 1) ? h : T(1), wj1 = (j & 1) ? h : T(0);
    const T wk0 = (k & 1) ? h : T(1), wk1 = (k & 1) ? h : T(0);
    const int r00 = gc.nxn * (j0 + gc.nyn * k0), r10 = gc.nxn * (j1 + gc.nyn * k0);
    const int r01 = gc.nxn * (j0 + gc.nyn * k1), r11 = gc.nxn * (j1 + gc.nyn * k1);
    const unsigned mk = mask_f[n];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T* v = xc + (size_t)c * gc.nn;
      const T a00 = wi0 * v[TOMO_CHK(r00 + i0, gc.nn, 9)] + wi1 * v[TOMO_CHK(r00 + i1, gc.nn, 9)];
      const T a10 = wi0 * v[TOMO_CHK(r10 + i0, gc.nn, 9)] + wi1 * v[TOMO_CHK(r10 + i1, gc.nn, 9)];
      const T a01 = wi0 * v[TOMO_CHK(r01 + i0, gc.nn, 9)] + wi1 * v[TOMO_CHK(r01 + i1, gc.nn, 9)];
      const T a11 = wi0 * v[TOMO_CHK(r11 + i0, gc.nn, 9)] + wi1 * v[TOMO_CHK(r11 + i1, gc.nn, 9)];
      const T acc = wk0 * (wj0 * a00 + wj1 * a10) + wk1 * (wj0 * a01 + wj1 * a11);
      const size_t idx = (size_t)c * gf.nn + n;
      if (!((mk >> c) & 1u)) xf[idx] += acc;
    }
  }
}

template <typename T>
__global__ void k_prolong_add(Geom gf, Geom gc, const T* __restrict__ xc, T* __restrict__ xf,
                              const uint8_t* __restrict__ mask_f, const int* skip) {
  prolong_body<T>(blockIdx.x, gridDim.x, gf, gc, xc, xf, mask_f, skip);
}

template <typename T>
cudaError_t launch_prolong_add(cudaStream_t st, Geom gf, Geom gc, const T* xc, T* xf,
                               const uint8_t* mask_f, const int* skip) {
  int blocks = (gf.nn + 255) / 256;
  if (blocks > 16384) blocks = 16384;
  pdl_launch(k_prolong_add<T>, blocks, 256, 0, st, gf, gc, xc, xf, mask_f, skip);
  return cudaGetLastError();
}

// Coarse element (edge 2h) modulus = mean of its (up to 8) children; with s = h E this is
// s_c = (sum of children s_f) / 4.  Children outside the fine grid count as void.
template <typename T>
__global__ void k_coarsen_s(Geom gf, Geom gc, const T* __restrict__ sf, T* __restrict__ sc) {
  PDL_ENTER();
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < gc.nel; e += gridDim.x * blockDim.x) {
    const int I = e % gc.nx, J = (e / gc.nx) % gc.ny, K = e / (gc.nx * gc.ny);
    T acc = T(0);
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int i = 2 * I + dx, j = 2 * J + dy, k = 2 * K + dz;
          if (i < gf.nx && j < gf.ny && k < gf.nz)
            acc += sf[TOMO_CHK(i + gf.nx * (j + gf.ny * k), gf.nel, 10)];
        }
    sc[e] = acc * T(0.25);
  }
}

// D^-1 per node, D = k0diag * (sum of s_e over the node's elements), 0 where that sum is not
// positive: the same sum, in the same order, as the zero-start Jacobi step above, for the
// Chebyshev steps of the product kernel (computed once per level and gradient).
template <typename T>
__global__ void k_invdiag(Geom g, const T* __restrict__ s, T k0diag, T* __restrict__ invd) {
  PDL_ENTER();
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < g.nn; n += gridDim.x * blockDim.x) {
    const int i = n % g.nxn, j = (n / g.nxn) % g.nyn, k = n / (g.nxn * g.nyn);
    const int xa = max(i - 1, 0), xb = min(i, g.nx - 1);
    const int ya = g.nx * max(j - 1, 0), yb = g.nx * min(j, g.ny - 1);
    const int za = g.nx * g.ny * max(k - 1, 0), zb = g.nx * g.ny * min(k, g.nz - 1);
    const T wxa = i > 0 ? T(1) : T(0), wxb = i < g.nx ? T(1) : T(0);
    const T wya = j > 0 ? T(1) : T(0), wyb = j < g.ny ? T(1) : T(0);
    const T wza = k > 0 ? T(1) : T(0), wzb = k < g.nz ? T(1) : T(0);
    auto row = [&](int off) {
      return wxa * s[TOMO_CHK(off + xa, g.nel, 11)] + wxb * s[TOMO_CHK(off + xb, g.nel, 11)];
    };
    const T S = wza * (wya * row(za + ya) + wyb * row(za + yb)) +
                wzb * (wya * row(zb + ya) + wyb * row(zb + yb));
    const T dg = k0diag * S;
    invd[n] = dg > T(0) ? T(1) / dg : T(0);
  }
}

template <typename T>
cudaError_t launch_invdiag(cudaStream_t st, Geom g, const T* s, T k0diag, T* invd) {
  int blocks = (g.nn + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  pdl_launch(k_invdiag<T>, blocks, 256, 0, st, g, s, k0diag, invd);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarsen_s(cudaStream_t st, Geom gf, Geom gc, const T* sf, T* sc) {
  int blocks = (gc.nel + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  pdl_launch(k_coarsen_s<T>, blocks, 256, 0, st, gf, gc, sf, sc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Coarsest level: assemble the dense K (fixed DOFs -> identity), scale symmetrically by
// D^-1/2, invert in place by Gauss-Jordan (SPD: no pivoting), one CTA.
// A holds D^-1/2 K^-1 D^-1/2 ... stored as inv(D^-1/2 K D^-1/2); dscale = D^-1/2.
// ---------------------------------------------------------------------------------------
template <typename T, bool SMEM>
__global__ void __launch_bounds__(1024) k_coarse_factor(Geom g, const T* __restrict__ s,
                                                        const uint8_t* __restrict__ mask,
                                                        const __grid_constant__ DenseK0<T> K0,
                                                        T* __restrict__ A, T* __restrict__ dscale,
                                                        unsigned* status) {
  PDL_ENTER();
  const int n = 3 * g.nn;
  const int tid = threadIdx.x, nt = blockDim.x;
  extern __shared__ unsigned char smem_raw[];
  T* col = reinterpret_cast<T*>(smem_raw);  // 4n: pivot column and row snapshots
  T* M = SMEM ? col + 4 * n : A;            // the working matrix: shared memory when it fits
  T* s_sm = SMEM ? M + (size_t)n * n : col + 4 * n;           // element moduli
  uint8_t* m_sm = reinterpret_cast<uint8_t*>(s_sm + g.nel);  // fixed bits per node
  for (int e = tid; e < g.nel; e += nt) s_sm[e] = s[e];
  for (int q = tid; q < g.nn; q += nt) m_sm[q] = mask[q];
  __syncthreads();
  // Entry (r, c), r = cr N_n + nr: sum over the elements shared by nodes nr and nc of
  // s_e K0[(a_r, cr), (a_c, cc)]; rows and columns of fixed DOFs are those of the identity.
  for (int q = tid; q < n * n; q += nt) {
    const int r = q / n, c = q - (q / n) * n;
    const int cr = r / g.nn, nr = r - cr * g.nn, cc = c / g.nn, nc = c - cc * g.nn;
    T v = T(0);
    if (((m_sm[nr] >> cr) & 1u) || ((m_sm[nc] >> cc) & 1u)) {
      v = (r == c) ? T(1) : T(0);
    } else {
      const int ir = nr % g.nxn, jr = (nr / g.nxn) % g.nyn, kr = nr / (g.nxn * g.nyn);
      const int ic = nc % g.nxn, jc = (nc / g.nxn) % g.nyn, kc = nc / (g.nxn * g.nyn);
      const int x0 = max(max(ir, ic) - 1, 0), x1 = min(min(ir, ic), g.nx - 1);
      const int y0 = max(max(jr, jc) - 1, 0), y1 = min(min(jr, jc), g.ny - 1);
      const int z0 = max(max(kr, kc) - 1, 0), z1 = min(min(kr, kc), g.nz - 1);
      for (int ez = z0; ez <= z1; ++ez)
        for (int ey = y0; ey <= y1; ++ey)
          for (int ex = x0; ex <= x1; ++ex) {
            const int ar = (ir - ex) + 2 * (jr - ey) + 4 * (kr - ez);
            const int ac = (ic - ex) + 2 * (jc - ey) + 4 * (kc - ez);
            v += s_sm[ex + g.nx * (ey + g.ny * ez)] * K0.k[(3 * ar + cr) * 24 + 3 * ac + cc];
          }
    }
    M[q] = v;
  }
  __syncthreads();
  T* ds = col;  // D^-1/2 (the snapshot buffers are free until the elimination)
  for (int q = tid; q < n; q += nt) {
    T dv = M[(size_t)q * n + q];
    if (!(dv > T(0))) {
      atomicOr(status, DEV_BREAKDOWN);
      dv = T(1);
      M[(size_t)q * n + q] = T(1);
    }
    ds[q] = T(1) / sqrt(dv);
    dscale[q] = ds[q];
  }
  __syncthreads();
  for (int q = tid; q < n * n; q += nt) {
    const int a = q / n, b = q - (q / n) * n;
    M[q] *= ds[a] * ds[b];
  }
  __syncthreads();
  // In-place Gauss-Jordan inversion of the scaled SPD matrix (no pivoting).  Each thread
  // owns the entries of one column j at rows i0, i0 + R, ...; pivot step k needs column k
  // and row k as they were before the step, which the owners of column k+1 and row k+1
  // write into the other half of a double buffer while updating, so one barrier per step.
  T* colb = col;          // [2][n] snapshots of the pivot column
  T* rowb = col + 2 * n;  // [2][n] snapshots of the pivot row
  const int R = nt / n > 0 ? nt / n : 1;
  const bool own = tid < R * n;
  const int j = own ? tid % n : 0, i0 = own ? tid / n : 0;
  if (own)
    for (int i = i0; i < n; i += R) {
      const T v = M[(size_t)i * n + j];
      if (j == 0) colb[i] = v;
      if (i == 0) rowb[j] = v;
    }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const T* cs = colb + (k & 1) * n;
    const T* rs = rowb + (k & 1) * n;
    T* cn = colb + ((k + 1) & 1) * n;
    T* rn = rowb + ((k + 1) & 1) * n;
    T p = rs[k];
    if (!(p > T(0))) {
      if (tid == 0) atomicOr(status, DEV_BREAKDOWN);
      p = T(1);
    }
    const T ip = T(1) / p;
    if (own) {
      const T rj = (j == k) ? T(1) : rs[j] * ip;
      for (int i = i0; i < n; i += R) {
        const size_t q = (size_t)i * n + j;
        T v;
        if (i == k) v = (j == k) ? ip : rj;
        else if (j == k) v = -cs[i] * ip;
        else v = M[q] - cs[i] * rj;
        M[q] = v;
        if (j == k + 1) cn[i] = v;
        if (i == k + 1) rn[j] = v;
      }
    }
    __syncthreads();
  }
  if (SMEM)
    for (int q = tid; q < n * n; q += nt) A[q] = M[q];
}

template <typename T>
cudaError_t launch_coarse_factor(cudaStream_t st, Geom g, const T* s, const uint8_t* mask,
                                 const DenseK0<T>& K0, T* A, T* dscale, unsigned* status) {
  const int n = 3 * g.nn;
  const size_t extra = sizeof(T) * (size_t)g.nel + (size_t)g.nn + 16;
  const size_t full = sizeof(T) * ((size_t)n * n + 4 * n) + extra;
  if (full <= 200 * 1024) {
    static cudaError_t attr = cudaFuncSetAttribute(
        k_coarse_factor<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
        200 * 1024 + 1024);  // once per process (and per type)
    if (attr != cudaSuccess) return attr;
    pdl_launch(k_coarse_factor<T, true>, 1, 1024, full, st, g, s, mask, K0, A, dscale, status);
  } else {
    pdl_launch(k_coarse_factor<T, false>, 1, 1024, sizeof(T) * 4 * (size_t)n + extra, st, g, s,
               mask, K0, A, dscale,
                                                                      status);
  }
  return cudaGetLastError();
}

// z = D^-1/2 Ainv D^-1/2 r.  One warp per row: the lanes split the row's columns (row-major
// reads of the stored inverse, coalesced; every warp's row loads are independent, so a row
// costs about one L2 round trip instead of one per few columns), then a fixed-order warp
// sum; accumulated in T.
// (w0, nw): the warp's place among the warps that share the rows (default: this block's
// warps); a row's result does not depend on which warp computes it.
template <typename T>
__device__ __forceinline__ void coarse_apply_body(int n, const T* __restrict__ Ainv,
                                                  const T* __restrict__ dsc,
                                                  const T* __restrict__ r, T* __restrict__ z,
                                                  const int* skip, int w0 = -1, int nw = 0) {
  PDL_ENTER();
  if (skipped(skip)) return;
  extern __shared__ unsigned char smem_raw[];
  T* rs = reinterpret_cast<T*>(smem_raw);
  for (int q = threadIdx.x; q < n; q += blockDim.x) rs[q] = dsc[q] * r[q];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  if (w0 < 0) {
    w0 = threadIdx.x >> 5;
    nw = blockDim.x >> 5;
  }
  for (int row = w0; row < n; row += nw) {
    const T* a = Ainv + (size_t)row * n;
    T acc = T(0);
    for (int c = lane; c < n; c += 32) acc += __ldg(a + TOMO_CHK(c, n, 12)) * rs[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) z[row] = dsc[row] * acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_apply(int n, const T* __restrict__ Ainv,
                                                       const T* __restrict__ dsc,
                                                       const T* __restrict__ r, T* __restrict__ z,
                                                       const int* skip) {
  coarse_apply_body<T>(n, Ainv, dsc, r, z, skip);
}

template <typename T>
cudaError_t launch_coarse_apply(cudaStream_t st, int n, const T* Ainv, const T* dscale,
                                const T* r, T* z, const int* skip) {
  pdl_launch(k_coarse_apply<T>, 1, 1024, sizeof(T) * (size_t)n, st, n, Ainv, dscale, r, z, skip);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// CG: x += alpha p, r -= alpha q, rr = r.r; convergence test in the finaliser.
// With xlo the iterate is the unevaluated pair xhi + xlo (float): the product alpha*p is
// formed exactly as prod + err (FMA) and added with TwoSum, so the pair keeps ~48 bits.
// ---------------------------------------------------------------------------------------
// x (+)= alpha p as the float pair (hi, lo): the product alpha*p is formed exactly as
// prod + perr (FMA) and added to hi with TwoSum; the rn intrinsics keep the compiler from
// contracting these steps into FMAs (that would break the error terms)
__device__ __forceinline__ void pair_axpy(float alpha, float pv, float& hi, float& lo) {
  const float prod = __fmul_rn(alpha, pv);
  const float perr = __fmaf_rn(alpha, pv, -prod);
  const float s = __fadd_rn(hi, prod);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(prod, bb));
  const float l2 = __fadd_rn(__fadd_rn(lo, err), perr);
  const float hi2 = __fadd_rn(s, l2);
  lo = __fsub_rn(l2, __fsub_rn(hi2, s));
  hi = hi2;
}

// x1 != nullptr: also the finest level's zero-start Jacobi step from the new residual,
// x1[c nn + m] = c2 r[c nn + m] invd[m] (the first smoothing step of the next V-cycle).
template <typename T, bool PAIRX>
__device__ __forceinline__ void cg_xr_body(int vb, int vnb, int n, T* __restrict__ xhi,
                                           T* __restrict__ xlo, T* __restrict__ r,
                                           const T* __restrict__ p, const T* __restrict__ q,
                                           double* partials, unsigned* counter,
                                           CgScalars* sc, T* __restrict__ x1 = nullptr,
                                           const T* __restrict__ invd = nullptr, T c2 = T(0)) {
  const int nn = n / 3;
  PDL_ENTER();
  if (sc->done) return;
  const double alpha_d = sc->alpha;
  const T alpha = (T)alpha_d;
  double acc = 0.0;      // FP64 grids
  FloatPairSum accf;     // FP32 grids
  const int tid = vb * blockDim.x + threadIdx.x, nt = vnb * blockDim.x;
  int i0 = 0;
  if constexpr (sizeof(T) == 4) {
    // float4 body: 16-byte accesses, and up to kIlpXr of a thread's float4 groups loaded
    // before any is used, keep enough bytes in flight to stream at HBM rate also with few
    // resident warps; every group is then updated (and added to the dot) in index order
    const int n4 = n >> 2;
    for (int v0 = tid; v0 < n4; v0 += kIlpXr * nt) {
      float4 pv[kIlpXr], qv[kIlpXr], rv[kIlpXr], hv[kIlpXr], lv[kIlpXr];
#pragma unroll
      for (int u = 0; u < kIlpXr; ++u) {
        const int v = v0 + u * nt;
        if (v < n4) {
          pv[u] = reinterpret_cast<const float4*>(p)[v];
          qv[u] = reinterpret_cast<const float4*>(q)[v];
          rv[u] = reinterpret_cast<const float4*>(r)[v];
          hv[u] = reinterpret_cast<const float4*>(xhi)[v];
          if constexpr (PAIRX) lv[u] = reinterpret_cast<const float4*>(xlo)[v];
        }
      }
#pragma unroll
      for (int u = 0; u < kIlpXr; ++u) {
        const int v = v0 + u * nt;
        if (v >= n4) break;
        if constexpr (PAIRX) {
          pair_axpy(alpha, pv[u].x, hv[u].x, lv[u].x);
          pair_axpy(alpha, pv[u].y, hv[u].y, lv[u].y);
          pair_axpy(alpha, pv[u].z, hv[u].z, lv[u].z);
          pair_axpy(alpha, pv[u].w, hv[u].w, lv[u].w);
          reinterpret_cast<float4*>(xlo)[v] = lv[u];
        } else {
          hv[u].x += alpha * pv[u].x;
          hv[u].y += alpha * pv[u].y;
          hv[u].z += alpha * pv[u].z;
          hv[u].w += alpha * pv[u].w;
        }
        reinterpret_cast<float4*>(xhi)[v] = hv[u];
        float4 rr = rv[u];
        rr.x = rr.x - alpha * qv[u].x;
        rr.y = rr.y - alpha * qv[u].y;
        rr.z = rr.z - alpha * qv[u].z;
        rr.w = rr.w - alpha * qv[u].w;
        reinterpret_cast<float4*>(r)[v] = rr;
        if (x1) {
          const int i = v << 2;
          int m = i - (i / nn) * nn;   // node of DOF i; the next three follow (wrapping at nn)
          float4 xv;
          xv.x = c2 * rr.x * invd[TOMO_CHK(m, nn, 13)];
          m = (m + 1 == nn) ? 0 : m + 1;
          xv.y = c2 * rr.y * invd[TOMO_CHK(m, nn, 13)];
          m = (m + 1 == nn) ? 0 : m + 1;
          xv.z = c2 * rr.z * invd[TOMO_CHK(m, nn, 13)];
          m = (m + 1 == nn) ? 0 : m + 1;
          xv.w = c2 * rr.w * invd[TOMO_CHK(m, nn, 13)];
          reinterpret_cast<float4*>(x1)[v] = xv;
        }
        accf.add(__fmul_rn(rr.x, rr.x));
        accf.add(__fmul_rn(rr.y, rr.y));
        accf.add(__fmul_rn(rr.z, rr.z));
        accf.add(__fmul_rn(rr.w, rr.w));
      }
    }
    i0 = n4 << 2;
  }
  for (int i = i0 + tid; i < n; i += nt) {
    const T pv = p[i];
    if constexpr (PAIRX) {
      float hi = xhi[i], lo = xlo[i];
      pair_axpy(alpha, pv, hi, lo);
      xhi[i] = hi;
      xlo[i] = lo;
    } else {
      xhi[i] += alpha * pv;
    }
    const T rv = r[i] - alpha * q[i];
    r[i] = rv;
    if (x1) x1[i] = c2 * rv * invd[i - (i / nn) * nn];
    if constexpr (sizeof(T) == 4) accf.add(__fmul_rn(rv, rv));
    else acc += rv * rv;
  }
  if constexpr (sizeof(T) == 4) acc = accf.value();
  double v[1] = {acc};
  grid_reduce_at<1>(v, partials, counter, [sc](const double* tot) {
    sc->rr = tot[0];
    sc->it += 1;
    if (!isfinite(tot[0])) { sc->status |= DEV_NAN; sc->done = 1; }
    else if (tot[0] <= sc->tol2 || sc->it >= sc->maxit) sc->done = 1;
  }, vb, vnb);
}

template <typename T, bool PAIRX>
__global__ void k_cg_xr(int n, T* __restrict__ xhi, T* __restrict__ xlo, T* __restrict__ r,
                        const T* __restrict__ p, const T* __restrict__ q, double* partials,
                        unsigned* counter, CgScalars* sc, T* __restrict__ x1,
                        const T* __restrict__ invd, T c2) {
  cg_xr_body<T, PAIRX>(blockIdx.x, gridDim.x, n, xhi, xlo, r, p, q, partials, counter, sc, x1,
                       invd, c2);
}

// Blocks of the x/r update of an n-vector: enough for 16-byte accesses at HBM rate on large
// grids (two waves of 304), fewer on small ones (one float4 per thread and pass); the same
// count whether the grid is launched alone or in a batch, so that the reduction order and
// the result do not depend on it.
int cg_xr_blocks(int n) {
  const int b = ((n >> 2) + kRedThreads - 1) / kRedThreads;
  return b < 1 ? 1 : (b > 2 * kRedBlocks ? 2 * kRedBlocks : b);
}

template <typename T>
cudaError_t launch_cg_xr(cudaStream_t st, int n, T* xhi, T* xlo, T* r, const T* p, const T* q,
                         double* partials, unsigned* counter, CgScalars* sc, T* x1,
                         const T* invd, T c2) {
  const int blocks = cg_xr_blocks(n);
  if (xlo) {
    if constexpr (sizeof(T) == 4) {
      pdl_launch(k_cg_xr<T, true>, blocks, kRedThreads, 0, st, n, xhi, xlo, r, p, q, partials,
                 counter, sc, x1, invd, c2);
      return cudaGetLastError();
    }
    return cudaErrorInvalidValue;
  }
  pdl_launch(k_cg_xr<T, false>, blocks, kRedThreads, 0, st, n, xhi, nullptr, r, p, q, partials,
             counter, sc, x1, invd, c2);
  return cudaGetLastError();
}


// p = z + beta p
template <typename T>
__device__ __forceinline__ void cg_p_body(int vb, int vnb, int n, T* __restrict__ p,
                                          const T* __restrict__ z, CgScalars* sc) {
  PDL_ENTER();
  if (sc->done) return;
  const T beta = (T)sc->beta;
  const int tid = vb * blockDim.x + threadIdx.x, nt = vnb * blockDim.x;
  int i0 = 0;
  if constexpr (sizeof(T) == 4) {
    const int n4 = n >> 2;
    for (int v0 = tid; v0 < n4; v0 += kIlpP * nt) {
      float4 zv[kIlpP], pv[kIlpP];
#pragma unroll
      for (int u = 0; u < kIlpP; ++u)
        if (v0 + u * nt < n4) {
          zv[u] = reinterpret_cast<const float4*>(z)[v0 + u * nt];
          pv[u] = reinterpret_cast<const float4*>(p)[v0 + u * nt];
        }
#pragma unroll
      for (int u = 0; u < kIlpP; ++u)
        if (v0 + u * nt < n4) {
          float4 w = pv[u];
          w.x = zv[u].x + beta * w.x;
          w.y = zv[u].y + beta * w.y;
          w.z = zv[u].z + beta * w.z;
          w.w = zv[u].w + beta * w.w;
          reinterpret_cast<float4*>(p)[v0 + u * nt] = w;
        }
    }
    i0 = n4 << 2;
  }
  for (int i = i0 + tid; i < n; i += nt) p[i] = z[i] + beta * p[i];
}

template <typename T>
__global__ void k_cg_p(int n, T* __restrict__ p, const T* __restrict__ z, CgScalars* sc) {
  cg_p_body<T>(blockIdx.x, gridDim.x, n, p, z, sc);
}

template <typename T>
cudaError_t launch_cg_p(cudaStream_t st, int n, T* p, const T* z, CgScalars* sc) {
  int blocks = (n + 255) / 256;
  if (blocks > 8 * 152) blocks = 8 * 152;
  pdl_launch(k_cg_p<T>, blocks, 256, 0, st, n, p, z, sc);
  return cudaGetLastError();
}

// The p update as the last kernel of the device-side loop's iteration, with the loop's
// control in its last block (no launch of its own): continue while CG has not stopped; the
// iteration counter bounds the loop even if a reduction never reported.  counter: a zeroed
// word, reset by the last block.
template <typename T>
__global__ void k_cg_p_cond(int n, T* __restrict__ p, const T* __restrict__ z, CgScalars* sc,
                            cudaGraphConditionalHandle h, unsigned* counter) {
  cg_p_body<T>(blockIdx.x, gridDim.x, n, p, z, sc);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(counter, 1u) == gridDim.x - 1) {
      *counter = 0u;
      sc->loops += 1;
      const bool go = !sc->done && sc->loops < sc->maxit + 8;
      if (!go) sc->done = 1;
      cudaGraphSetConditional(h, go ? 1u : 0u);
    }
  }
}

template <typename T>
cudaError_t launch_cg_p_cond(cudaStream_t st, int n, T* p, const T* z, CgScalars* sc,
                             cudaGraphConditionalHandle h, unsigned* counter) {
  int blocks = (n + 255) / 256;
  if (blocks > 8 * 152) blocks = 8 * 152;
  pdl_launch(k_cg_p_cond<T>, blocks, 256, 0, st, n, p, z, sc, h, counter);
  return cudaGetLastError();
}

// p[0..n) = v
template <typename T>
__global__ void k_fill(int64_t n, T* __restrict__ p, T v) {
  PDL_ENTER();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

template <typename T>
cudaError_t launch_fill(cudaStream_t st, int64_t n, T* p, T v) {
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  pdl_launch(k_fill<T>, (int)blocks, 256, 0, st, n, p, v);
  return cudaGetLastError();
}

// the load from its nonzero entries: fT[idx[k]] = val[k], f64[idx[k]] = val[k] (the vectors
// are zeroed before)
template <typename T>
__global__ void k_scatter_load(int nnz, const int64_t* __restrict__ idx,
                               const double* __restrict__ val, T* __restrict__ fT,
                               double* __restrict__ f64) {
  PDL_ENTER();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x) {
    fT[idx[k]] = (T)val[k];
    f64[idx[k]] = val[k];
  }
}

template <typename T>
cudaError_t launch_scatter_load(cudaStream_t st, int nnz, const int64_t* idx, const double* val,
                                T* fT, double* f64) {
  if (nnz <= 0) return cudaSuccess;
  int blocks = (nnz + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  pdl_launch(k_scatter_load<T>, blocks, 256, 0, st, nnz, idx, val, fT, f64);
  return cudaGetLastError();
}

// out = sum_k val[k] (u + ulo)[idx[k]] in FP64 (one block, fixed order): f^T u for a sparse
// load f given by its nonzero entries.
template <typename T>
__global__ void __launch_bounds__(256) k_sparse_dot(int nnz, const int64_t* __restrict__ idx,
                                                    const double* __restrict__ val,
                                                    const T* __restrict__ u,
                                                    const T* __restrict__ ulo,
                                                    double* partials, unsigned* counter,
                                                    double* out) {
  PDL_ENTER();
  double acc = 0.0;
  // a thread's entries k = t, t + nt, ... in that order, kSpIlp of them with their index,
  // value and u loads in flight together (one dependent round trip per group)
  constexpr int kSpIlp = 4;
  const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  for (int k0 = t; k0 < nnz; k0 += kSpIlp * nt) {
    int64_t ii[kSpIlp];
    double vv[kSpIlp], uu[kSpIlp];
#pragma unroll
    for (int q = 0; q < kSpIlp; ++q) {
      const int k = k0 + q * nt;
      ii[q] = k < nnz ? idx[k] : -1;
      vv[q] = k < nnz ? val[k] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kSpIlp; ++q) {
      uu[q] = 0.0;
      if (ii[q] >= 0) {
        uu[q] = (double)u[ii[q]];
        if (ulo) uu[q] += (double)ulo[ii[q]];
      }
    }
#pragma unroll
    for (int q = 0; q < kSpIlp; ++q)
      if (ii[q] >= 0) acc += vv[q] * uu[q];
  }
  double v[1] = {acc};
  grid_reduce_at<1>(v, partials, counter, [out](const double* tot) { *out = tot[0]; },
                    blockIdx.x, gridDim.x);
}

// f^T u over the load's nonzero entries: blocks by the entry count alone (about 1024
// entries each, at most 152), so the fixed-order block sum is the same on every call
template <typename T>
cudaError_t launch_sparse_dot(cudaStream_t st, int nnz, const int64_t* idx, const double* val,
                              const T* u, const T* ulo, double* partials, unsigned* counter,
                              double* out) {
  int blocks = (nnz + 1023) / 1024;
  blocks = blocks < 1 ? 1 : (blocks > 152 ? 152 : blocks);
  pdl_launch(k_sparse_dot<T>, blocks, 256, 0, st, nnz, idx, val, u, ulo, partials, counter,
             out);
  return cudaGetLastError();
}

// r = 0 on every DOF, then r[idx[k]] = val[k]: the CG start residual f (masked) from the load's
// nonzero entries
template <typename T>
__global__ void k_scatter_vec(int nnz, const int64_t* __restrict__ idx,
                              const double* __restrict__ val, T* __restrict__ r) {
  PDL_ENTER();
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nnz; k += gridDim.x * blockDim.x)
    r[idx[k]] = (T)val[k];
}

template <typename T>
cudaError_t launch_scatter_vec(cudaStream_t st, int nnz, const int64_t* idx, const double* val,
                               T* r) {
  if (nnz <= 0) return cudaSuccess;
  int blocks = (nnz + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  pdl_launch(k_scatter_vec<T>, blocks, 256, 0, st, nnz, idx, val, r);
  return cudaGetLastError();
}

template cudaError_t launch_sparse_dot<float>(cudaStream_t, int, const int64_t*, const double*,
                                              const float*, const float*, double*, unsigned*,
                                              double*);
template cudaError_t launch_sparse_dot<double>(cudaStream_t, int, const int64_t*, const double*,
                                               const double*, const double*, double*,
                                               unsigned*, double*);
template cudaError_t launch_scatter_vec<float>(cudaStream_t, int, const int64_t*, const double*,
                                               float*);
template cudaError_t launch_scatter_vec<double>(cudaStream_t, int, const int64_t*,
                                                const double*, double*);
// Start of a CG solve in one launch: the non-null vectors among x_hi, x_lo, r, p (n each) are
// zeroed and *sc = h (the solve's scalars, passed by value).
template <typename T>
__global__ void k_cg_start(int n, T* __restrict__ xhi, T* __restrict__ xlo, T* __restrict__ r,
                           T* __restrict__ p, CgScalars* sc, CgScalars h) {
  PDL_ENTER();
  if (blockIdx.x == 0 && threadIdx.x == 0) *sc = h;
  T* v[4] = {xhi, xlo, r, p};
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    T* x = v[a];
    if (!x) continue;
    int i0 = 0;
    if constexpr (sizeof(T) == 4) {
      const int n4 = n >> 2;
      for (int i = tid; i < n4; i += nt)
        reinterpret_cast<float4*>(x)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      i0 = n4 << 2;
    }
    for (int i = i0 + tid; i < n; i += nt) x[i] = T(0);
  }
}

template <typename T>
cudaError_t launch_cg_start(cudaStream_t st, int n, T* xhi, T* xlo, T* r, T* p, CgScalars* sc,
                            const CgScalars& h) {
  int blocks = ((n >> 2) + 255) / 256;
  if (blocks > 8 * 152) blocks = 8 * 152;
  if (blocks < 1) blocks = 1;
  pdl_launch(k_cg_start<T>, blocks, 256, 0, st, n, xhi, xlo, r, p, sc, h);
  return cudaGetLastError();
}

template cudaError_t launch_cg_start<float>(cudaStream_t, int, float*, float*, float*, float*,
                                            CgScalars*, const CgScalars&);
template cudaError_t launch_cg_start<double>(cudaStream_t, int, double*, double*, double*,
                                             double*, CgScalars*, const CgScalars&);
template cudaError_t launch_fill<float>(cudaStream_t, int64_t, float*, float);
template cudaError_t launch_fill<double>(cudaStream_t, int64_t, double*, double);
template cudaError_t launch_scatter_load<float>(cudaStream_t, int, const int64_t*,
                                                const double*, float*, double*);
template cudaError_t launch_scatter_load<double>(cudaStream_t, int, const int64_t*,
                                                 const double*, double*, double*);

// ---------------------------------------------------------------------------------------
// Batched launches (FP32): block b belongs to grid q with cta0[q] <= b < cta0[q+1] and acts
// as block b - cta0[q] of cta0[q+1] - cta0[q]; each grid gets the block count its own launch
// would use, so its results do not depend on the batch.
// ---------------------------------------------------------------------------------------
__global__ void k_jacobi_batch(const __grid_constant__ FlatBatch<JacobiItem> B) {
  const int q = batch_owner(B.cta0, B.n, (int)blockIdx.x);
  const JacobiItem& a = B.a[q];
  jacobi_body<float, false>((int)blockIdx.x - B.cta0[q], B.cta0[q + 1] - B.cta0[q], a.g, a.s,
                            a.mask, a.b, a.c2, a.k0diag, a.x1, nullptr, nullptr, nullptr,
                            nullptr, a.skip, a.invd);
}

__global__ void k_restrict_batch(const __grid_constant__ FlatBatch<RestrictItem> B) {
  const int q = batch_owner(B.cta0, B.n, (int)blockIdx.x);
  const RestrictItem& a = B.a[q];
  restrict_body<float>((int)blockIdx.x - B.cta0[q], B.cta0[q + 1] - B.cta0[q], a.gf, a.gc,
                       a.rf, a.rc, a.mask_c, a.skip, a.x1, a.sc, a.c2, a.k0diag);
}

__global__ void k_prolong_batch(const __grid_constant__ FlatBatch<ProlongItem> B) {
  const int q = batch_owner(B.cta0, B.n, (int)blockIdx.x);
  const ProlongItem& a = B.a[q];
  prolong_body<float>((int)blockIdx.x - B.cta0[q], B.cta0[q + 1] - B.cta0[q], a.gf, a.gc,
                      a.xc, a.xf, a.mask_f, a.skip);
}

// one block per grid
__global__ void __launch_bounds__(1024)
    k_coarse_apply_batch(const __grid_constant__ FlatBatch<CoarseItem> B) {
  const CoarseItem& a = B.a[blockIdx.x];
  coarse_apply_body<float>(a.n, a.Ainv, a.dsc, a.r, a.z, a.skip);
}

__global__ void k_cg_xr_batch(const __grid_constant__ FlatBatch<CgXrItem> B) {
  const int q = batch_owner(B.cta0, B.n, (int)blockIdx.x);
  const CgXrItem& a = B.a[q];
  cg_xr_body<float, true>((int)blockIdx.x - B.cta0[q], B.cta0[q + 1] - B.cta0[q], a.n, a.xhi,
                          a.xlo, a.r, a.p, a.q, a.partials, a.counter, a.sc, a.x1, a.invd,
                          a.c2);
}

__global__ void k_cg_p_batch(const __grid_constant__ FlatBatch<CgPItem> B) {
  const int q = batch_owner(B.cta0, B.n, (int)blockIdx.x);
  const CgPItem& a = B.a[q];
  cg_p_body<float>((int)blockIdx.x - B.cta0[q], B.cta0[q + 1] - B.cta0[q], a.n, a.p, a.z, a.sc);
}

__global__ void k_loop_cond_batch(cudaGraphConditionalHandle h, CgScalars* const* scs, int n) {
  PDL_ENTER();
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    CgScalars* sc = scs[q];
    if (sc->done) continue;
    sc->loops += 1;
    if (sc->loops < sc->maxit + 8) atomicOr(&any, 1);
    else sc->done = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

namespace {

// Fill tables of up to kBatchMax entries and launch them.  blocks(item): the block count of
// the item's own launch; work(item) > 0: the launch shares about kBatchBlocks blocks among
// the items in proportion to their work (at most their own count, at least one), since a
// batch of small grids at their own counts carries thousands of nearly empty blocks.  Only
// for kernels whose results do not depend on the block count (grid-stride pointwise work),
// or whose reduction order may follow the batch.
constexpr int kBatchBlocks = 2 * 8 * 152;  // two waves of 256-thread blocks
template <class Item, class Blocks, class Work, class Launch>
cudaError_t flat_batches(const Item* a, int n, Blocks blocks, Work work, Launch launch) {
  for (int q0 = 0; q0 < n; q0 += kBatchMax) {
    FlatBatch<Item> B{};
    B.n = std::min(kBatchMax, n - q0);
    double wsum = 0.0;
    for (int q = 0; q < B.n; ++q) wsum += (double)work(a[q0 + q]);
    int ctas = 0;
    for (int q = 0; q < B.n; ++q) {
      B.a[q] = a[q0 + q];
      B.cta0[q] = ctas;
      int b = blocks(B.a[q]);
      const double w = (double)work(B.a[q]);
      if (w > 0.0 && wsum > 0.0) {
        const int share = (int)std::ceil(kBatchBlocks * w / wsum);
        b = std::max(1, std::min(b, share));
      }
      ctas += b;
    }
    B.cta0[B.n] = ctas;
    if (ctas > 0) {
      launch(B, ctas, q0 > 0);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

int clamp_blocks(int n, int cap) {
  const int b = (n + 255) / 256;
  return b < 1 ? 1 : (b > cap ? cap : b);
}

}  // namespace

cudaError_t launch_jacobi_batch(cudaStream_t st, const JacobiItem* a, int n) {
  return flat_batches(a, n, [](const JacobiItem& it) { return clamp_blocks(it.g.nn, 4096); },
                      [](const JacobiItem& it) { return it.g.nn; },
                      [st](const FlatBatch<JacobiItem>& B, int ctas, bool cont) {
                        if (g_phase_rec) record_phase(PH_JACOBI, ctas, B, cont);
                        else pdl_launch(k_jacobi_batch, ctas, 256, 0, st, B);
                      });
}

cudaError_t launch_restrict_batch(cudaStream_t st, const RestrictItem* a, int n) {
  return flat_batches(a, n, [](const RestrictItem& it) { return clamp_blocks(it.gc.nn, 8192); },
                      [](const RestrictItem& it) { return it.gc.nn; },
                      [st](const FlatBatch<RestrictItem>& B, int ctas, bool cont) {
                        if (g_phase_rec) record_phase(PH_RESTRICT, ctas, B, cont);
                        else pdl_launch(k_restrict_batch, ctas, 256, 0, st, B);
                      });
}

cudaError_t launch_prolong_batch(cudaStream_t st, const ProlongItem* a, int n) {
  return flat_batches(a, n, [](const ProlongItem& it) { return clamp_blocks(it.gf.nn, 16384); },
                      [](const ProlongItem& it) { return it.gf.nn; },
                      [st](const FlatBatch<ProlongItem>& B, int ctas, bool cont) {
                        if (g_phase_rec) record_phase(PH_PROLONG, ctas, B, cont);
                        else pdl_launch(k_prolong_batch, ctas, 256, 0, st, B);
                      });
}

cudaError_t launch_coarse_apply_batch(cudaStream_t st, const CoarseItem* a, int n) {
  int nmax = 0;
  for (int q = 0; q < n; ++q) nmax = std::max(nmax, a[q].n);
  const size_t smem = sizeof(float) * (size_t)nmax;
  return flat_batches(a, n, [](const CoarseItem&) { return 1; },
                      [](const CoarseItem&) { return 0; },
                      [st, smem](const FlatBatch<CoarseItem>& B, int ctas, bool cont) {
                        if (g_phase_rec) record_phase(PH_COARSE, ctas, B, cont);
                        else pdl_launch(k_coarse_apply_batch, ctas, 1024, smem, st, B);
                      });
}

cudaError_t launch_cg_xr_batch(cudaStream_t st, const CgXrItem* a, int n) {
  return flat_batches(a, n, [](const CgXrItem& it) { return cg_xr_blocks(it.n); },
                      [](const CgXrItem& it) { return it.n; },
                      [st](const FlatBatch<CgXrItem>& B, int ctas, bool cont) {
                        if (g_phase_rec) record_phase(PH_CGXR, ctas, B, cont);
                        else pdl_launch(k_cg_xr_batch, ctas, kRedThreads, 0, st, B);
                      });
}

cudaError_t launch_cg_p_batch(cudaStream_t st, const CgPItem* a, int n) {
  return flat_batches(a, n, [](const CgPItem& it) { return clamp_blocks(it.n, 8 * 152); },
                      [](const CgPItem& it) { return it.n; },
                      [st](const FlatBatch<CgPItem>& B, int ctas, bool cont) {
                        if (g_phase_rec) record_phase(PH_CGP, ctas, B, cont);
                        else pdl_launch(k_cg_p_batch, ctas, 256, 0, st, B);
                      });
}

cudaError_t launch_loop_cond_batch(cudaStream_t st, cudaGraphConditionalHandle h,
                                   CgScalars* const* scs, int n) {
  pdl_launch(k_loop_cond_batch, 1, 256, 0, st, h, scs, n);
  return cudaGetLastError();
}

// out = a . (b + blo), accumulated in double.
template <typename TA, typename TB>
__global__ void k_dot(int n, const TA* __restrict__ a, const TB* __restrict__ b,
                      const TB* __restrict__ blo, double* partials, unsigned* counter,
                      double* out) {
  PDL_ENTER();
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double bv = (double)b[i];
    if (blo) bv += (double)blo[i];
    acc += (double)a[i] * bv;
  }
  double v[1] = {acc};
  grid_reduce<1>(v, partials, counter, [out](const double* tot) { *out = tot[0]; });
}

template <typename TA, typename TB>
cudaError_t launch_dot(cudaStream_t st, int n, const TA* a, const TB* b, const TB* blo,
                       double* partials, unsigned* counter, double* out) {
  pdl_launch(k_dot<TA, TB>, kRedBlocks, kRedThreads, 0, st, n, a, b, blo, partials, counter, out);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_mask_copy(Geom g, const T* __restrict__ in, const uint8_t* __restrict__ mask,
                            T* __restrict__ out) {
  PDL_ENTER();
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 3 * g.nn; q += gridDim.x * blockDim.x) {
    const int c = q / g.nn, node = q % g.nn;
    out[q] = ((mask[node] >> c) & 1u) ? T(0) : in[q];
  }
}

template <typename T>
cudaError_t launch_mask_copy(cudaStream_t st, Geom g, const T* in, const uint8_t* mask, T* out) {
  int blocks = (3 * g.nn + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  pdl_launch(k_mask_copy<T>, blocks, 256, 0, st, g, in, mask, out);
  return cudaGetLastError();
}

template <typename TO, typename TI>
__global__ void k_convert(int n, const TI* __restrict__ in, const TI* __restrict__ inlo,
                          TO* __restrict__ out, const CgScalars* gate) {
  PDL_ENTER();
  if (gate != nullptr &&
      (gate->done || gate->rr_every <= 0 || (gate->it % gate->rr_every) != 0))
    return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (inlo) out[i] = (TO)((double)in[i] + (double)inlo[i]);
    else out[i] = (TO)in[i];
  }
}

template <typename TO, typename TI>
cudaError_t launch_convert(cudaStream_t st, int n, const TI* in, const TI* inlo, TO* out,
                           const CgScalars* gate) {
  int blocks = (n + 255) / 256;
  if (blocks > 8192) blocks = 8192;
  pdl_launch(k_convert<TO, TI>, blocks, 256, 0, st, n, in, inlo, out, gate);
  return cudaGetLastError();
}

#define INST(T)                                                                               \
  template cudaError_t launch_jacobi<T>(cudaStream_t, Geom, const T*, const uint8_t*, const T*, \
                                        T, T, T*, T*, double*, unsigned*, CgScalars*, int,     \
                                        const int*, T*);                                     \
  template cudaError_t launch_restrict<T>(cudaStream_t, Geom, Geom, const T*, T*,             \
                                          const uint8_t*, const int*, T*, const T*, T, T);   \
  template cudaError_t launch_prolong_add<T>(cudaStream_t, Geom, Geom, const T*, T*,          \
                                             const uint8_t*, const int*);                    \
  template cudaError_t launch_coarsen_s<T>(cudaStream_t, Geom, Geom, const T*, T*);           \
  template cudaError_t launch_invdiag<T>(cudaStream_t, Geom, const T*, T, T*);               \
  template cudaError_t launch_coarse_factor<T>(cudaStream_t, Geom, const T*, const uint8_t*,  \
                                               const DenseK0<T>&, T*, T*, unsigned*);        \
  template cudaError_t launch_coarse_apply<T>(cudaStream_t, int, const T*, const T*, const T*, \
                                              T*, const int*);                               \
  template cudaError_t launch_cg_xr<T>(cudaStream_t, int, T*, T*, T*, const T*, const T*,     \
                                       double*, unsigned*, CgScalars*, T*, const T*, T);     \
  template cudaError_t launch_cg_p<T>(cudaStream_t, int, T*, const T*, CgScalars*);           \
  template cudaError_t launch_cg_p_cond<T>(cudaStream_t, int, T*, const T*, CgScalars*,       \
                                           cudaGraphConditionalHandle, unsigned*);            \
  template cudaError_t launch_mask_copy<T>(cudaStream_t, Geom, const T*, const uint8_t*, T*);
INST(float)
INST(double)
#undef INST
template cudaError_t launch_dot<double, float>(cudaStream_t, int, const double*, const float*,
                                               const float*, double*, unsigned*, double*);
template cudaError_t launch_dot<double, double>(cudaStream_t, int, const double*, const double*,
                                                const double*, double*, unsigned*, double*);
template cudaError_t launch_dot<float, float>(cudaStream_t, int, const float*, const float*,
                                              const float*, double*, unsigned*, double*);
template cudaError_t launch_convert<float, float>(cudaStream_t, int, const float*, const float*,
                                                  float*, const CgScalars*);
template cudaError_t launch_convert<double, float>(cudaStream_t, int, const float*, const float*,
                                                   double*, const CgScalars*);
template cudaError_t launch_convert<float, double>(cudaStream_t, int, const double*,
                                                   const double*, float*, const CgScalars*);
template cudaError_t launch_convert<double, double>(cudaStream_t, int, const double*,
                                                    const double*, double*, const CgScalars*);


// ---------------------------------------------------------------------------------------
// Persistent lockstep iteration: the recorded batched launches of one CG iteration run as
// the phases of one cooperative kernel of 256-thread CTAs (every phase's CTA work is 256
// threads: the product's 32 x 8, the FP64 residual replacement's 32 x 8, the flat kernels'
// 256; the coarsest apply, launched with 1024 threads, strides over its rows with 256).
// Unit u of a phase is CTA u of the launch it replaces, so every grid sees the same blocks
// (and dot partials, in the same order) as in the launched loop: the results are bitwise
// the launched loop's.  Data written by an earlier phase is read through L2 (ldcg) or by
// plain loads after the barrier's fences, never through the read-only path.
// ---------------------------------------------------------------------------------------
thread_local std::vector<PhaseRec>* g_phase_rec = nullptr;

namespace {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier over all CTAs of the launch (count, generation words).  Returns false if
// this CTA waited longer than limit_ns for the others.
__device__ bool grid_barrier(unsigned* bar, long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();  // the CTA's writes happen before thread 0's fence (cumulative)
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      while (*gen == g) {
        if ((long long)(global_ns() - t0) > limit_ns) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();  // ... and thread 0's acquire happens before the CTA's later reads
  return s_ok != 0;
}

// One unit of each phase kind (a CTA of the recorded launch).
template <int MODE, bool DOT>
__device__ __forceinline__ void m2_unit(const unsigned char* tab, const UnitDesc& ud,
                                     const March2Const& K) {
  const March2Batch& B = *reinterpret_cast<const March2Batch*>(tab);
  const int loc = ud.vb, gx = ud.gx, gy = ud.gy;
  march2_body<MODE, DOT, false>(B.a[ud.q], K, loc % gx, (loc / gx) % gy, loc / (gx * gy), gx,
                                (unsigned)loc, (unsigned)ud.vnb, threadIdx.x & 31,
                                threadIdx.x >> 5);
}

template <class Item>
__device__ __forceinline__ const Item& flat_item(const unsigned char* tab, int q) {
  return reinterpret_cast<const FlatBatch<Item>*>(tab)->a[q];
}

__device__ __forceinline__ void rr_unit(const unsigned char* tab, const UnitDesc& ud,
                                     const ElemConst<double>& K1) {
  const MarchRrBatch& B = *reinterpret_cast<const MarchRrBatch*>(tab);
  const int loc = ud.vb, gx = ud.gx, gy = ud.gy;
  march_body<double, M_RESID, true, false, kRrTY, false>(
      B.a[ud.q], K1, loc % gx, (loc / gx) % gy, loc / (gx * gy), (unsigned)loc,
      (unsigned)ud.vnb, threadIdx.x & 31, threadIdx.x >> 5);
}

__device__ __forceinline__ void jacobi_unit(const unsigned char* tab, const UnitDesc& ud) {
  const JacobiItem& a = flat_item<JacobiItem>(tab, ud.q);
  jacobi_body<float, false>(ud.vb, ud.vnb, a.g, a.s, a.mask, a.b, a.c2, a.k0diag, a.x1,
                            nullptr, nullptr, nullptr, nullptr, a.skip, a.invd);
}

__device__ __forceinline__ void restrict_unit(const unsigned char* tab, const UnitDesc& ud) {
  const RestrictItem& a = flat_item<RestrictItem>(tab, ud.q);
  restrict_body<float>(ud.vb, ud.vnb, a.gf, a.gc, a.rf, a.rc, a.mask_c, a.skip, a.x1, a.sc,
                       a.c2, a.k0diag);
}

__device__ __forceinline__ void prolong_unit(const unsigned char* tab, const UnitDesc& ud) {
  const ProlongItem& a = flat_item<ProlongItem>(tab, ud.q);
  prolong_body<float>(ud.vb, ud.vnb, a.gf, a.gc, a.xc, a.xf, a.mask_f, a.skip);
}

__device__ __forceinline__ void coarse_unit(const unsigned char* tab, const UnitDesc& ud) {
  const CoarseItem& a = flat_item<CoarseItem>(tab, ud.q);
  // the launched coarsest solve is one 1024-thread block per grid: unit vb of vnb takes
  // its warps vb * 8 .. vb * 8 + 7 (of vnb * 8)
  coarse_apply_body<float>(a.n, a.Ainv, a.dsc, a.r, a.z, a.skip,
                           ud.vb * 8 + (int)(threadIdx.x >> 5), ud.vnb * 8);
}

__device__ __forceinline__ void cgxr_unit(const unsigned char* tab, const UnitDesc& ud) {
  const CgXrItem& a = flat_item<CgXrItem>(tab, ud.q);
  cg_xr_body<float, true>(ud.vb, ud.vnb, a.n, a.xhi, a.xlo, a.r, a.p, a.q, a.partials,
                          a.counter, a.sc, a.x1, a.invd, a.c2);
}

__device__ __forceinline__ void cgp_unit(const unsigned char* tab, const UnitDesc& ud) {
  const CgPItem& a = flat_item<CgPItem>(tab, ud.q);
  cg_p_body<float>(ud.vb, ud.vnb, a.n, a.p, a.z, a.sc);
}

__global__ void __launch_bounds__(256, 2)
    k_persist(const DevPhase* __restrict__ phases, int nph,
              const unsigned char* __restrict__ tables, const __grid_constant__ March2Const K2,
              const __grid_constant__ ElemConst<double> K1, unsigned* barrier,
              long long limit_ns, CgScalars* const* scs, int nscs,
              unsigned long long* acc) {
  // acc (optional): acc[p] += device ns of phase p as CTA 0 sees it (start or previous
  // barrier exit to this phase's barrier exit; a final barrier closes the last phase),
  // acc[nph] += 1 per launch
  unsigned long long t_last = 0;
  if (acc != nullptr && blockIdx.x == 0 && threadIdx.x == 0) t_last = global_ns();
  // The loop state lives in shared memory across a unit (one slot pair per thread, reread
  // after the unit), so that no register is held across the bodies: the product body alone
  // uses all but one of the 128 registers two CTAs per SM allow.
  __shared__ int s_loop[2][256];
  volatile int* const sp = &s_loop[0][threadIdx.x];
  volatile int* const su = &s_loop[1][threadIdx.x];
  for (int p = 0; p < nph; ++p) {
    for (int u = blockIdx.x;; u += gridDim.x) {
      const DevPhase ph = phases[p];
      if (u >= ph.units) break;
      const unsigned char* tab = tables + ph.offset;
      // the unit's place, precomputed on the host: grid q, block vb of vnb, product tile
      // counts gx, gy
      UnitDesc ud = reinterpret_cast<const UnitDesc*>(tables + ph.units_offset)[u];
      ud.q = (int)TOMO_CHK(ud.q, *reinterpret_cast<const int*>(tab), 17);
      *sp = p;
      *su = u;
      switch (ph.kind) {
        case PH_M2_APPLY: m2_unit<M_APPLY, false>(tab, ud, K2); break;
        case PH_M2_APPLY_DOT: m2_unit<M_APPLY, true>(tab, ud, K2); break;
        case PH_M2_RESID: m2_unit<M_RESID, false>(tab, ud, K2); break;
        case PH_M2_CHEB: m2_unit<M_CHEB, false>(tab, ud, K2); break;
        case PH_M2_CHEB_DOT: m2_unit<M_CHEB, true>(tab, ud, K2); break;
        case PH_RR: rr_unit(tab, ud, K1); break;
        case PH_JACOBI: jacobi_unit(tab, ud); break;
        case PH_RESTRICT: restrict_unit(tab, ud); break;
        case PH_PROLONG: prolong_unit(tab, ud); break;
        case PH_COARSE: coarse_unit(tab, ud); break;
        case PH_CGXR: cgxr_unit(tab, ud); break;
        case PH_CGP: cgp_unit(tab, ud); break;
        default: break;
      }
      __syncthreads();  // the next unit reuses this CTA's shared memory
      p = *sp;
      u = *su;
    }
    if (p + 1 < nph && phases[p + 1].join) continue;
    if (p + 1 == nph && acc == nullptr) break;  // the launch's end closes the last phase
    if (!grid_barrier(barrier, limit_ns)) {
      // a CTA did not arrive in time: every grid stops with the timeout status (the
      // remaining CTAs time out at their own next barrier and leave too)
      if (threadIdx.x == 0)
        for (int q = 0; q < nscs; ++q) {
          atomicOr(&scs[q]->status, DEV_TIMEOUT);
          scs[q]->done = 1;
        }
      return;
    }
    if (acc != nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
      const unsigned long long t = global_ns();
      acc[p] += t - t_last;
      t_last = t;
      if (p + 1 == nph) acc[nph] += 1;
    }
  }
}

}  // namespace

int persist_ctas(int num_sms, size_t smem) {
  int per_sm = 0;
  int dev = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_persist, 256, smem) !=
          cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * (num_sms > 0 ? num_sms : 152);
}

cudaError_t launch_persist(cudaStream_t st, const DevPhase* phases, int nph,
                           const unsigned char* tables, const March2Const& k2,
                           const ElemConst<double>& k1, unsigned* barrier, long long limit_ns,
                           CgScalars* const* scs, int nscs, int ctas, size_t smem,
                           unsigned long long* acc) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_persist, phases, nph, tables, k2, k1, barrier, limit_ns,
                            scs, nscs, acc);
}

#ifdef TOMO_CHECKED
TOMO_CHECK_ACCESSOR(check_word_vec)
#endif

}  // namespace tomo
