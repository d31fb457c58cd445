// The body of the FP32 product kernel (k_march2): one CTA of 32 x TY threads (TY = 8 thread
// rows, or 4 for batches of small grids), thread (l, t) = lane l of thread row t.  Shared by
// the launched kernels (matvec2.cu) and the persistent lockstep iteration (vec.cu), which
// runs the same CTA work as one unit of its phases.
#pragma once

#include "common.cuh"
#include "host.h"

namespace tomo {

namespace {

constexpr int TYP = 8;            // thread rows per CTA (two node rows each)
// resident CTAs per SM the register allocation aims at (2: 128 registers, no spills)
#ifndef TOMO_MARCH2_MIN_BLOCKS
#define TOMO_MARCH2_MIN_BLOCKS 2
#endif
#ifndef TOMO_MARCH2_CHEB_UNROLL
#define TOMO_MARCH2_CHEB_UNROLL 1
#endif
constexpr int kChebUnroll = TOMO_MARCH2_CHEB_UNROLL;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return __ffma2_rn(a, b, c);
}
__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 shdn2(float2 v) {
  return make_float2(__shfl_down_sync(FULL, v.x, 1), __shfl_down_sync(FULL, v.y, 1));
}
__device__ __forceinline__ float2 shup2(float2 v) {
  return make_float2(__shfl_up_sync(FULL, v.x, 1), __shfl_up_sync(FULL, v.y, 1));
}

// One CTA of the product: tile (bx, by) of gx tiles along x, z-chunk bz; blin / nblk are the
// CTA's linear index and the CTA count of this grid's launch (for the fused dot).
template <int MODE, bool DOT, bool NC = true, int TY = TYP>
__device__ __forceinline__ void march2_body(const March2Args& A, const March2Const& K, int bx,
                                            int by, int bz, int gx, unsigned blin,
                                            unsigned nblk, int l, int t) {
  constexpr bool CHEBY = MODE == M_CHEB;
  PDL_ENTER();
  // the stop flag is tested after the first planes' loads are issued, so that its latency
  // and theirs overlap (every CTA starts with them)
  const int stop = A.skip != nullptr ? *A.skip : 0;
  const Geom g = A.g;
  const int i = bx * 30 - 1 + l;
  const int j0 = by * (2 * TY - 2) - 1 + 2 * t;
  const int j1 = j0 + 1;
  const int kb = bz * A.kz;
  const int ke = min(kb + A.kz, g.nzn);
  const int nn = g.nn, plane = g.nxn * g.nyn, eplane = g.nx * g.ny;
  const bool col_i = i >= 0 && i < g.nxn;
  const bool c0 = col_i && j0 >= 0 && j0 < g.nyn;
  const bool c1 = col_i && j1 >= 0 && j1 < g.nyn;
  const bool el_i = i >= 0 && i < g.nx && l < 31;
  const bool e0 = el_i && j0 >= 0 && j0 < g.ny;
  const bool e1 = el_i && j1 >= 0 && j1 < g.ny && t < TY - 1;
  const bool lane_out = l >= 1 && l <= 30;
  const bool o0 = lane_out && c0 && t >= 1;
  const bool o1 = lane_out && c1 && t <= TY - 2;
  const int nb0 = c0 ? i + g.nxn * j0 : 0, nb1 = c1 ? i + g.nxn * j1 : 0;
  const int eb0 = e0 ? i + g.nx * j0 : 0, eb1 = e1 ? i + g.nx * j1 : 0;

  // sN: node row j0 of each thread row, plane k+1, and a zero row TY (the row above the
  // last thread row); sV: the sy = 1 half of each thread row's upper element in rows 1..TY,
  // for the thread row above, and a zero row 0 (below the first): no selects on the reads
  __shared__ float sN[3][TY + 1][32];
  __shared__ float sV[6][TY + 1][32];
  if (t == 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) sN[c][TY][l] = 0.0f;
#pragma unroll
    for (int q = 0; q < 6; ++q) sV[q][0][l] = 0.0f;
  }
  // lane 0 has no left neighbour: its shuffled-in value is weighted 0 (an FMA, not a select)
  const float2 wleft = bc2(l > 0 ? 1.0f : 0.0f), nwleft = bc2(l > 0 ? -1.0f : 0.0f);

  auto load_plane = [&](int k, float2 (&v)[3]) {
    const bool in = k >= 0 && k < g.nzn;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      v[c].x = (in && c0)
                   ? ldv<NC>(TOMO_AT(A.x, (size_t)c * nn + nb0 + plane * k, 3 * nn, 1))
                   : 0.0f;
      v[c].y = (in && c1)
                   ? ldv<NC>(TOMO_AT(A.x, (size_t)c * nn + nb1 + plane * k, 3 * nn, 1))
                   : 0.0f;
    }
  };
  auto load_s = [&](int k) -> float2 {
    const bool in = k >= 0 && k < g.nz;
    return make_float2((in && e0) ? ldv<NC>(TOMO_AT(A.s, eb0 + eplane * k, g.nel, 2)) : 0.0f,
                       (in && e1) ? ldv<NC>(TOMO_AT(A.s, eb1 + eplane * k, g.nel, 2)) : 0.0f);
  };

  // carried raw values at plane k: A0 own rows (j0, j1), N0 row j0+2, C0 = lane+1 of A0,
  // DN0 = lane+1 of N0
  float2 A0[3], C0[3];
  float N0[3], DN0[3];
  load_plane(kb - 1, A0);
  float2 A1n[3];
  load_plane(kb, A1n);
  float2 sen = load_s(kb - 1);
  const bool tile_fixed = A.tile_fixed == nullptr || A.tile_fixed[bx + gx * by] != 0;
  if (stop) return;
#pragma unroll
  for (int c = 0; c < 3; ++c) sN[c][t][l] = A0[c].x;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    N0[c] = sN[c][t + 1][l];
    C0[c] = shdn2(A0[c]);
    DN0[c] = __shfl_down_sync(FULL, N0[c], 1);
  }
  __syncthreads();

  float2 carry[3] = {bc2(0.0f), bc2(0.0f), bc2(0.0f)};
  // fused inner product: per step the three components are summed in FP32, then added to
  // the pair dhi + dlo with TwoSum (FP64 runs at 1/64 of the FP32 rate on this part)
  float2 dhi = bc2(0.0f), dlo = bc2(0.0f);

  auto step = [&](int k) {
    float2 A1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) A1[c] = A1n[c];
    const float2 se = sen;
    load_plane(k + 2, A1n);
    sen = load_s(k + 1);
    // epilogue operands of nodes (i, j0, k), (i, j1, k)
    const bool w0 = o0 && k >= kb, w1 = o1 && k >= kb;
    const int n0 = nb0 + plane * max(k, 0), n1 = nb1 + plane * max(k, 0);
    unsigned m0 = 0u, m1 = 0u;
    float2 bv[3], xp[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      bv[c] = bc2(0.0f);
      xp[c] = bc2(0.0f);
    }
    if (tile_fixed) {  // (CTA-uniform) only tiles that hold fixed nodes read the mask
      if (w0) m0 = A.mask[TOMO_CHK(n0, nn, 3)];
      if (w1) m1 = A.mask[TOMO_CHK(n1, nn, 3)];
    }
    if (MODE != M_APPLY) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (w0) bv[c].x = ldv<NC>(TOMO_AT(A.b, (size_t)c * nn + n0, 3 * nn, 3));
        if (w1) bv[c].y = ldv<NC>(TOMO_AT(A.b, (size_t)c * nn + n1, 3 * nn, 3));
      }
    }
    float2 inv = bc2(0.0f);  // CHEB: D^-1 of the two nodes (precomputed per level)
    if (CHEBY) {
      if (w0) inv.x = ldv<NC>(A.invd + TOMO_CHK(n0, nn, 3));
      if (w1) inv.y = ldv<NC>(A.invd + TOMO_CHK(n1, nn, 3));
    }
    if (CHEBY && A.c1 != 0.0f && !A.xprev_zero) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float* xpc = A.xprev + (size_t)c * nn;
        if (w0) xp[c].x = NC ? xpc[TOMO_CHK(n0, nn, 3)] : __ldcg(xpc + TOMO_CHK(n0, nn, 3));
        if (w1) xp[c].y = NC ? xpc[TOMO_CHK(n1, nn, 3)] : __ldcg(xpc + TOMO_CHK(n1, nn, 3));
      }
    }

    // ---- neighbour values at plane k+1 ----
#pragma unroll
    for (int c = 0; c < 3; ++c) sN[c][t][l] = A1[c].x;
    __syncthreads();
    float N1[3], DN1[3];
    float2 C1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      N1[c] = sN[c][t + 1][l];
      C1[c] = shdn2(A1[c]);
      DN1[c] = __shfl_down_sync(FULL, N1[c], 1);
    }

    // ---- forward: modes from edge differences, per component ----
    // element corners: A* (sx0, sy0), C* (sx1, sy0), B* (sx0, sy1), D* (sx1, sy1); *0 plane
    // k (sz0), *1 plane k+1 (sz1).  B = (A.y, N), D = (C.y, DN).
    float2 X[3][8];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 B0 = make_float2(A0[c].y, N0[c]), B1 = make_float2(A1[c].y, N1[c]);
      const float2 D0 = make_float2(C0[c].y, DN0[c]), D1 = make_float2(C1[c].y, DN1[c]);
      const float2 ex00 = sub2(A0[c], C0[c]), ex10 = sub2(B0, D0);
      const float2 ex01 = sub2(A1[c], C1[c]), ex11 = sub2(B1, D1);
      const float2 ey00 = sub2(A0[c], B0), ey10 = sub2(C0[c], D0);
      const float2 ey01 = sub2(A1[c], B1), ey11 = sub2(C1[c], D1);
      const float2 ez00 = sub2(A0[c], A1[c]), ez10 = sub2(C0[c], C1[c]);
      const float2 ez01 = sub2(B0, B1), ez11 = sub2(D0, D1);
      const float2 p0 = add2(ex00, ex10), m0v = sub2(ex00, ex10);
      const float2 p1 = add2(ex01, ex11), m1v = sub2(ex01, ex11);
      X[c][1] = add2(p0, p1);
      X[c][5] = sub2(p0, p1);
      X[c][3] = add2(m0v, m1v);
      X[c][7] = sub2(m0v, m1v);
      const float2 q0 = add2(ey00, ey10), q1 = add2(ey01, ey11);
      X[c][2] = add2(q0, q1);
      X[c][6] = sub2(q0, q1);
      X[c][4] = add2(add2(ez00, ez10), add2(ez01, ez11));
      X[c][0] = bc2(0.0f);
    }

    // ---- K0 in the mode basis, scaled by s_e ----
    float2 W[3][8];
    {
      const float2 a0s = mul2(se, bc2(K.a0)), b0s = mul2(se, bc2(K.b0));
      const float2 a7s = mul2(se, bc2(K.a7)), b7s = mul2(se, bc2(K.b7));
      const float2 tas = mul2(se, bc2(K.ta)), tbs = mul2(se, bc2(K.tb));
      const float2 uas = mul2(se, bc2(K.ua)), uds = mul2(se, bc2(K.ud));
#pragma unroll
      for (int c = 0; c < 3; ++c) W[c][0] = bc2(0.0f);
      {  // class 0: members (0,1) (1,2) (2,4)
        const float2 S = add2(add2(X[0][1], X[1][2]), X[2][4]);
        const float2 bS = mul2(b0s, S);
        W[0][1] = fma2(a0s, X[0][1], bS);
        W[1][2] = fma2(a0s, X[1][2], bS);
        W[2][4] = fma2(a0s, X[2][4], bS);
      }
      {  // class 7: members (0,6) (1,5) (2,3)
        const float2 S = add2(add2(X[0][6], X[1][5]), X[2][3]);
        const float2 bS = mul2(b7s, S);
        W[0][6] = fma2(a7s, X[0][6], bS);
        W[1][5] = fma2(a7s, X[1][5], bS);
        W[2][3] = fma2(a7s, X[2][3], bS);
      }
#pragma unroll
      for (int tt = 0; tt < 3; ++tt) {  // classes 1, 2, 4
        const int k2 = 1 << tt, ca = (tt + 1) % 3, cb = (tt + 2) % 3;
        const int ma = k2 ^ (1 << ca), mb = k2 ^ (1 << cb);
        const float2 xa = X[ca][ma], xb = X[cb][mb];
        W[ca][ma] = fma2(tbs, xb, mul2(tas, xa));
        W[cb][mb] = fma2(tbs, xa, mul2(tas, xb));
      }
#pragma unroll
      for (int tt = 0; tt < 3; ++tt) {  // classes 3, 5, 6 (decoupled member tt, m = 7)
        const int k2 = 7 ^ (1 << tt), ca = (tt + 1) % 3, cb = (tt + 2) % 3;
        const int ma = k2 ^ (1 << ca), mb = k2 ^ (1 << cb);
        const float2 u = mul2(uas, add2(X[ca][ma], X[cb][mb]));
        W[ca][ma] = u;
        W[cb][mb] = u;
        W[tt][7] = mul2(uds, X[tt][7]);
      }
    }

    // ---- staged inverse: x-stage, shuffle to lane+1, y-stage, shared memory, z-stage ----
    float2 T[3][2];
    float2 V1keep[3][2];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 G[4];
      // (my, mz) -> q = my + 2 mz; modes m0 = 2 my + 4 mz (mx = 0), m0 + 1 (mx = 1)
      {
        const float2 w1 = W[c][1];  // q = 0: W[0] = 0, so U0 = w1, U1 = -w1
        const float2 fromleft = shup2(w1);
        G[0] = fma2(fromleft, nwleft, w1);
      }
#pragma unroll
      for (int q = 1; q < 4; ++q) {
        const int m0i = 2 * (q & 1) + 4 * (q >> 1);
        const float2 u0 = add2(W[c][m0i], W[c][m0i + 1]);
        const float2 u1 = sub2(W[c][m0i], W[c][m0i + 1]);
        const float2 fromleft = shup2(u1);
        G[q] = fma2(fromleft, wleft, u0);
      }
#pragma unroll
      for (int mz = 0; mz < 2; ++mz) {
        const float2 v0 = add2(G[2 * mz], G[2 * mz + 1]);  // sy = 0
        const float2 v1 = sub2(G[2 * mz], G[2 * mz + 1]);  // sy = 1
        T[c][mz] = v0;
        V1keep[c][mz] = v1;
        sV[2 * c + mz][t + 1][l] = v1.y;  // upper element's sy = 1 half -> node row j0 + 2
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
#pragma unroll
      for (int mz = 0; mz < 2; ++mz) {
        const float prev = sV[2 * c + mz][t][l];
        // node row j0 gets the element row below (previous thread row); row j1 gets the
        // lower element of this pair
        T[c][mz] = add2(T[c][mz], make_float2(prev, V1keep[c][mz].x));
      }
    }
    // z-stage: plane k (output) and plane k+1 (carried)
    float2 out[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 y0 = add2(T[c][0], T[c][1]);
      const float2 y1 = sub2(T[c][0], T[c][1]);
      out[c] = add2(carry[c], y0);
      carry[c] = y1;
    }

    // ---- epilogue ----
    if (w0 || w1) {
      float2 pc = bc2(0.0f);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float2 v;
        if (MODE == M_APPLY) {
          v = out[c];
        } else if (MODE == M_RESID) {
          v = sub2(bv[c], out[c]);
        } else {
          const float2 w = mul2(sub2(bv[c], out[c]), inv);
          v = fma2(bc2(A.c2), w, A0[c]);
          if (A.c1 != 0.0f) v = fma2(bc2(A.c1), sub2(A0[c], xp[c]), v);
        }
        const bool f0 = (m0 >> c) & 1u, f1 = (m1 >> c) & 1u;
        if (f0) v.x = 0.0f;
        if (f1) v.y = 0.0f;
        float* dst = CHEBY ? A.xprev : A.y;
        if (w0) dst[TOMO_CHK((size_t)c * nn + n0, 3 * nn, 4)] = v.x;
        if (w1) dst[TOMO_CHK((size_t)c * nn + n1, 3 * nn, 4)] = v.y;
        if (DOT) {
          const float2 d2 = (MODE == M_APPLY) ? A0[c] : bv[c];
          pc = fma2(make_float2(w0 ? d2.x : 0.0f, w1 ? d2.y : 0.0f), v, pc);
        }
      }
      if (DOT) {
        const float2 s = add2(dhi, pc);
        const float2 bb = sub2(s, dhi);
        const float2 err = add2(sub2(dhi, sub2(s, bb)), sub2(pc, bb));
        dhi = s;
        dlo = add2(dlo, err);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      A0[c] = A1[c];
      C0[c] = C1[c];
      N0[c] = N1[c];
      DN0[c] = DN1[c];
    }
    };
  // The product and the residual run unrolled by two (the plane buffers swap roles without
  // register copies: 8 % on the product at the benchmark size, measured); the Chebyshev
  // step keeps one step per iteration unless TOMO_MARCH2_CHEB_UNROLL says otherwise
  // (unrolled it spills).
  if constexpr (CHEBY) {
#pragma unroll kChebUnroll
    for (int k = kb - 1; k < ke; ++k) step(k);
  } else {
#pragma unroll 2
    for (int k = kb - 1; k < ke; ++k) step(k);
  }
  if (DOT) {
    double v[1] = {((double)dhi.x + (double)dlo.x) + ((double)dhi.y + (double)dlo.y)};
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

}  // namespace

}  // namespace tomo
