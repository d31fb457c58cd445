// The body of the generic product kernel (k_march, FP64 grids and the FP64 residual of the
// float-pair iterate): one CTA of 32 lanes x TY thread rows, thread (l, r).  Shared by the
// launched kernels (matvec.cu) and the persistent lockstep iteration (vec.cu).
#pragma once

#include "common.cuh"
#include "host.h"

namespace tomo {

template <typename T>
__device__ __forceinline__ void fwht8(T (&v)[8]) {
#pragma unroll
  for (int st = 1; st < 8; st <<= 1) {
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      if ((s & st) == 0) {
        const T a = v[s], b = v[s + st];
        v[s] = a + b;
        v[s + st] = a - b;
      }
    }
  }
}

// W_c[m] = s * sum_c' blk[k][c][c'] X_c'[k ^ (1 << c')] for k = m ^ (1 << c); translation
// modes (m = 0) and structural zeros skipped.
template <typename T>
__device__ __forceinline__ void block_apply(const ElemConst<T>& C, T se, const T (&X)[3][8],
                                            T (&W)[3][8]) {
  T Xs[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Xs[c][0] = T(0);
#pragma unroll
    for (int m = 1; m < 8; ++m) Xs[c][m] = se * X[c][m];
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) W[c][0] = T(0);
  // classes 0 and 7: full 3x3
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const int k = kk ? 7 : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T acc = C.blk[k][c][0] * Xs[0][k ^ 1];
      acc += C.blk[k][c][1] * Xs[1][k ^ 2];
      acc += C.blk[k][c][2] * Xs[2][k ^ 4];
      W[c][k ^ (1 << c)] = acc;
    }
  }
  // classes 1, 2, 4: the translation member (c == log2 k) is decoupled and zero
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int k = 1 << t;
    const int ca = (t + 1) % 3, cb = (t + 2) % 3;
    const T xa = Xs[ca][k ^ (1 << ca)], xb = Xs[cb][k ^ (1 << cb)];
    W[ca][k ^ (1 << ca)] = C.blk[k][ca][ca] * xa + C.blk[k][ca][cb] * xb;
    W[cb][k ^ (1 << cb)] = C.blk[k][cb][ca] * xa + C.blk[k][cb][cb] * xb;
  }
  // classes 3, 5, 6: the member with m = 7 (component t below) is decoupled
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int k = 7 ^ (1 << t);  // t=2 -> 3, t=1 -> 5, t=0 -> 6
    const int ca = (t + 1) % 3, cb = (t + 2) % 3;
    const T xa = Xs[ca][k ^ (1 << ca)], xb = Xs[cb][k ^ (1 << cb)];
    W[ca][k ^ (1 << ca)] = C.blk[k][ca][ca] * xa + C.blk[k][ca][cb] * xb;
    W[cb][k ^ (1 << cb)] = C.blk[k][cb][ca] * xa + C.blk[k][cb][cb] * xb;
    W[t][7] = C.blk[k][t][t] * Xs[t][7];
  }
}

// One CTA: tile (bx, by), z-chunk bz; blin / nblk: the CTA's linear index and the CTA count
// of this grid's launch (for the fused dot).
template <typename T, int MODE, bool PAIR, bool DOT, int TY = kTY, bool NC = true>
__device__ __forceinline__ void march_body(const MarchArgs<T>& A, const ElemConst<T>& C, int bx,
                                           int by, int bz, unsigned blin, unsigned nblk,
                                           int l, int r) {
  PDL_ENTER();
  if (A.skip != nullptr && *A.skip) return;
  if (A.gate != nullptr && (A.gate->rr_every <= 0 || (A.gate->it % A.gate->rr_every) != 0))
    return;
  const Geom g = A.g;
  const int i = bx * 30 - 1 + l;
  const int j = by * (TY - 2) - 1 + r;
  const int kb = bz * A.kz;
  const int ke = min(kb + A.kz, g.nzn);
  const int nn = g.nn;
  const bool col_in = (i >= 0 && i < g.nxn && j >= 0 && j < g.nyn);
  const bool el_col = (i >= 0 && i < g.nx && j >= 0 && j < g.ny && l < 31);
  const bool out_col = col_in && l >= 1 && l <= 30 && r >= 1 && r <= TY - 2;
  const int colbase = col_in ? i + g.nxn * j : 0;
  const int plane = g.nxn * g.nyn;
  const int ecol = el_col ? i + g.nx * j : 0;
  const int eplane = g.nx * g.ny;

  // PAIR with T = float: the input pair is carried as two arrays and differenced separately;
  // PAIR with T = double: the float pair is joined into one double on load (exact: 48 bits)
  constexpr bool SPLIT = PAIR && sizeof(T) == 4;
  constexpr bool JOIN = PAIR && sizeof(T) == 8;
  constexpr int NA = SPLIT ? 6 : 3;
  __shared__ T sA[NA][TY][32];
  __shared__ T sG[6][TY][32];
  __shared__ T sS[TY][32];

  auto load_plane = [&](int k, T (&v)[NA]) {
#pragma unroll
    for (int q = 0; q < NA; ++q) v[q] = T(0);
    if (col_in && k >= 0 && k < g.nzn) {
      const int n = TOMO_CHK(colbase + plane * k, nn, 5);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if constexpr (JOIN) {
          v[c] = (T)ldv<NC>(A.xf_hi + (size_t)c * nn + n) +
                 (T)ldv<NC>(A.xf_lo + (size_t)c * nn + n);
        } else {
          v[c] = ldv<NC>(A.x + (size_t)c * nn + n);
          if constexpr (SPLIT) v[3 + c] = ldv<NC>(A.xlo + (size_t)c * nn + n);
        }
      }
    }
  };
  auto load_s = [&](int k) -> T {
    return (el_col && k >= 0 && k < g.nz) ? ldv<NC>(A.s + TOMO_CHK(ecol + eplane * k, g.nel, 5))
                                          : T(0);
  };

  // raw node values: A* own column, B* row j+1; *0 plane k, *1 plane k+1
  T A0[NA], B0[NA];
  load_plane(kb - 1, A0);
#pragma unroll
  for (int q = 0; q < NA; ++q) sA[q][r][l] = A0[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NA; ++q) B0[q] = (r + 1 < TY) ? sA[q][r + 1][l] : T(0);
  __syncthreads();
  // one-step-ahead prefetch of the next plane and element layer
  T A1n[NA];
  load_plane(kb, A1n);
  T sen = load_s(kb - 1);

  T carry[3] = {T(0), T(0), T(0)};
  T carryS = T(0);
  double dot = 0.0;

  for (int k = kb - 1; k < ke; ++k) {
    T A1[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) A1[q] = A1n[q];
    const T se = sen;
    load_plane(k + 2, A1n);
    sen = load_s(k + 1);
    // epilogue operands of node (i, j, k), consumed at the end of this step
    const bool emit = out_col && k >= kb;
    const int n_out = emit ? TOMO_CHK(colbase + plane * (k < 0 ? 0 : k), nn, 6)
                           : colbase + plane * (k < 0 ? 0 : k);
    unsigned mk = 0u;
    T bv[3] = {T(0), T(0), T(0)}, xp[3] = {T(0), T(0), T(0)};
    if (emit) {
      mk = A.mask[n_out];
      if (MODE != M_APPLY) {
#pragma unroll
        for (int c = 0; c < 3; ++c) bv[c] = ldv<NC>(A.b + (size_t)c * nn + n_out);
      }
      if (MODE == M_CHEB && A.c1 != T(0) && !A.xprev_zero) {
#pragma unroll
        for (int c = 0; c < 3; ++c) xp[c] = A.xprev[(size_t)c * nn + n_out];
      }
    }

#pragma unroll
    for (int q = 0; q < NA; ++q) sA[q][r][l] = A1[q];
    __syncthreads();
    T B1[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) B1[q] = (r + 1 < TY) ? sA[q][r + 1][l] : T(0);

    // ---- forward: differences against local node 0, Walsh-Hadamard per component ----
    T X[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // local node s = sx + 2 sy + 4 sz
      T v[8];
      const T a0 = A0[c];
      const T c0 = __shfl_down_sync(0xffffffffu, A0[c], 1);
      const T c1v = __shfl_down_sync(0xffffffffu, A1[c], 1);
      const T d0 = __shfl_down_sync(0xffffffffu, B0[c], 1);
      const T d1 = __shfl_down_sync(0xffffffffu, B1[c], 1);
      v[0] = T(0);
      v[1] = c0 - a0;
      v[2] = B0[c] - a0;
      v[3] = d0 - a0;
      v[4] = A1[c] - a0;
      v[5] = c1v - a0;
      v[6] = B1[c] - a0;
      v[7] = d1 - a0;
      if constexpr (SPLIT) {
        const T al = A0[3 + c];
        const T cl0 = __shfl_down_sync(0xffffffffu, A0[3 + c], 1);
        const T cl1 = __shfl_down_sync(0xffffffffu, A1[3 + c], 1);
        const T dl0 = __shfl_down_sync(0xffffffffu, B0[3 + c], 1);
        const T dl1 = __shfl_down_sync(0xffffffffu, B1[3 + c], 1);
        v[1] += cl0 - al;
        v[2] += B0[3 + c] - al;
        v[3] += dl0 - al;
        v[4] += A1[3 + c] - al;
        v[5] += cl1 - al;
        v[6] += B1[3 + c] - al;
        v[7] += dl1 - al;
      }
      fwht8(v);
#pragma unroll
      for (int m = 0; m < 8; ++m) X[c][m] = v[m];
    }
    T W[3][8];
    block_apply(C, se, X, W);
    // ---- inverse: corner forces y_c[s] = sum_m chi_m(s) W_c[m] ----
    T G[3][4];  // contributions to node column i for corners (sy, sz) -> index sy + 2 sz
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      T v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = W[c][m];
      fwht8(v);
      // +x corners (sx = 1) belong to node column i+1: send to lane + 1
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T fromleft = __shfl_up_sync(0xffffffffu, v[2 * q + 1], 1);
        G[c][q] = v[2 * q] + (l > 0 ? fromleft : T(0));
      }
    }
    T Sx = T(0);
    if (MODE == M_CHEB) {
      const T fromleft = __shfl_up_sync(0xffffffffu, se, 1);
      Sx = se + (l > 0 ? fromleft : T(0));
    }
    // +y corners (sy = 1) belong to node row j+1: through shared memory
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      sG[2 * c + 0][r][l] = G[c][1];  // sy=1, sz=0
      sG[2 * c + 1][r][l] = G[c][3];  // sy=1, sz=1
    }
    if (MODE == M_CHEB) sS[r][l] = Sx;
    __syncthreads();
    T Tz[3][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const T b0 = r > 0 ? sG[2 * c + 0][r - 1][l] : T(0);
      const T b1 = r > 0 ? sG[2 * c + 1][r - 1][l] : T(0);
      Tz[c][0] = G[c][0] + b0;  // sz = 0: node plane k
      Tz[c][1] = G[c][2] + b1;  // sz = 1: node plane k+1
    }
    T Sy = T(0);
    if (MODE == M_CHEB) Sy = Sx + (r > 0 ? sS[r - 1][l] : T(0));

    // ---- node (i, j, k) is complete ----
    T out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      out[c] = carry[c] + Tz[c][0];
      carry[c] = Tz[c][1];
    }
    const T Stot = carryS + Sy;
    carryS = Sy;
    if (emit) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const bool fx = (mk >> c) & 1u;
        const size_t idx = (size_t)c * nn + n_out;
        if (MODE == M_APPLY) {
          const T yv = fx ? T(0) : out[c];
          A.y[idx] = yv;
          if (DOT) dot += (double)(A0[c] * yv);
        } else if (MODE == M_RESID) {
          const T rv = fx ? T(0) : (bv[c] - out[c]);
          if constexpr (JOIN) {
            const float rf = (float)rv;
            A.yf[idx] = rf;
            if (A.x1f) A.x1f[idx] = A.c2f * rf * A.invdf[n_out];
          } else {
            A.y[idx] = rv;
          }
        } else {
          const T dg = C.k0diag * Stot;
          const T w = dg > T(0) ? (bv[c] - out[c]) / dg : T(0);
          T xn = A0[c] + A.c2 * w;
          if (A.c1 != T(0)) xn += A.c1 * (A0[c] - xp[c]);
          xn = fx ? T(0) : xn;
          A.xprev[idx] = xn;
          if (DOT) dot += (double)(bv[c] * xn);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      A0[q] = A1[q];
      B0[q] = B1[q];
    }
  }
  if (DOT) {
    double v[1] = {dot};
    CgScalars* sc = A.sc;
    const int kind = A.dot_kind;
    grid_reduce_at<1>(v, A.partials, A.counter, [sc, kind](const double* tot) {
      if (kind == 1) {
        sc->pq = tot[0];
        if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
          sc->status |= isfinite(tot[0]) ? DEV_BREAKDOWN : DEV_NAN;
          sc->done = 1;
          sc->alpha = 0.0;
        } else {
          sc->alpha = sc->rz / tot[0];
        }
      } else if (kind == 2) {
        sc->rz_new = tot[0];
        if (!isfinite(tot[0])) {
          sc->status |= DEV_NAN;
          sc->done = 1;
        } else if (!(tot[0] > 0.0)) {  // r^T M r <= 0: the preconditioner is not positive
          sc->status |= DEV_BREAKDOWN;
          sc->done = 1;
        }
        sc->beta = sc->rz != 0.0 ? tot[0] / sc->rz : 0.0;
        sc->rz = tot[0];
      }
    }, blin, nblk);
  }
}

}  // namespace tomo
