// Host-side construction of the hex8 element constants used by the kernels.
//
// K0 is the stiffness of the unit cube with E = 1 (state equation of Eq. 4, Section III-D,
// discretised with trilinear hex8 elements, three displacement components per node).
// It is built from exact one-dimensional integrals of the linear shape functions
// N0 = 1 - t, N1 = t on [0, 1]:
//     M = int N_a N_b,  S = int N_a' N_b',  C = int N_a' N_b,
// with G^{ij}_{ab} = int d_i N_a d_j N_b = prod over axes of M, S, C or C^T, and
//     K0[(a,c),(b,d)] = lam G^{cd}_{ab} + mu G^{dc}_{ab} + mu delta_cd sum_k G^{kk}_{ab}
// (the isotropic bilinear form lam div u div v + 2 mu eps(u):eps(v)).
//
// The kernels use K0 in the per-component Walsh-Hadamard basis, where the cube's three
// reflection symmetries make it block diagonal (eight 3x3 blocks, see common.cuh).
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "host.h"

namespace tomo {

static int bit(int a, int q) { return (a >> q) & 1; }

void build_unit_stiffness(double nu, double K0[576]) {
  const double lam = nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  const double mu = 1.0 / (2.0 * (1.0 + nu));
  const double M[2][2] = {{1.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 1.0 / 3.0}};
  const double S[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
  const double C[2][2] = {{-0.5, -0.5}, {0.5, 0.5}};  // C[a][b] = int N_a' N_b
  // G[a][b][i][j]
  static double G[8][8][3][3];
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double g = 1.0;
          for (int q = 0; q < 3; ++q) {
            const int aq = bit(a, q), bq = bit(b, q);
            if (q == i && q == j) g *= S[aq][bq];
            else if (q == i) g *= C[aq][bq];
            else if (q == j) g *= C[bq][aq];
            else g *= M[aq][bq];
          }
          G[a][b][i][j] = g;
        }
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) {
      const double lap = G[a][b][0][0] + G[a][b][1][1] + G[a][b][2][2];
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d)
          K0[(3 * a + c) * 24 + 3 * b + d] =
              lam * G[a][b][c][d] + mu * G[a][b][d][c] + (c == d ? mu * lap : 0.0);
    }
}

static int popc(int v) { return __builtin_popcount((unsigned)v); }

// Returns false if K0 is not block diagonal in the Walsh-Hadamard basis (cannot happen
// for an isotropic cube; checked so that the kernels' sparsity assumptions are safe).
bool build_hadamard_blocks(const double K0[576], double blk[8][3][3], double* k0diag) {
  // B[(m,c),(m',c')] = 1/64 sum_{s,s'} chi_m(s) K0[(s,c),(s',c')] chi_m'(s')
  double B[24][24];
  double bmax = 0.0;
  for (int m = 0; m < 8; ++m)
    for (int c = 0; c < 3; ++c)
      for (int mp = 0; mp < 8; ++mp)
        for (int cp = 0; cp < 3; ++cp) {
          double v = 0.0;
          for (int s = 0; s < 8; ++s)
            for (int sp = 0; sp < 8; ++sp) {
              const double chi = ((popc(m & s) + popc(mp & sp)) & 1) ? -1.0 : 1.0;
              v += chi * K0[(3 * s + c) * 24 + 3 * sp + cp];
            }
          B[3 * m + c][3 * mp + cp] = v / 64.0;
          bmax = std::fmax(bmax, std::fabs(v / 64.0));
        }
  for (int i = 0; i < 24; ++i)
    for (int j = 0; j < 24; ++j) {
      const int ki = (i / 3) ^ (1 << (i % 3)), kj = (j / 3) ^ (1 << (j % 3));
      if (ki != kj && std::fabs(B[i][j]) > 1e-12 * bmax) return false;
    }
  for (int k = 0; k < 8; ++k)
    for (int c = 0; c < 3; ++c)
      for (int cp = 0; cp < 3; ++cp)
        blk[k][c][cp] = B[3 * (k ^ (1 << c)) + c][3 * (k ^ (1 << cp)) + cp];
  // Structural zeros the kernels rely on: the translation member of classes 1, 2, 4 and
  // the coupling of the m = 7 member to the others in classes 3, 5, 6.
  for (int k = 1; k < 7; ++k) {
    for (int c = 0; c < 3; ++c) {
      const int m = k ^ (1 << c);
      for (int cp = 0; cp < 3; ++cp) {
        const int mp = k ^ (1 << cp);
        bool zero = false;
        if (m == 0 || mp == 0) zero = true;
        if ((k == 3 || k == 5 || k == 6) && ((m == 7) != (mp == 7))) zero = true;
        if (zero) {
          if (std::fabs(blk[k][c][cp]) > 1e-12 * bmax) return false;
          blk[k][c][cp] = 0.0;
        }
      }
    }
  }
  *k0diag = K0[0];
  for (int i = 1; i < 24; ++i)
    if (std::fabs(K0[i * 25] - K0[0]) > 1e-14) return false;
  return true;
}

// The eight Hadamard-basis blocks of the isotropic cube come in four kinds (related by axis
// permutations): class 0 (normal strains) and class 7 are p I + q (11^T - I); classes 1, 2, 4
// couple two members with [[a, b], [b, a]] (the translation member is zero); classes 3, 5, 6
// couple two members with a (11^T) and leave the m = 7 member alone with d.  Returns false if
// blk does not have this form.
bool block_kinds(const double blk[8][3][3], BlockKinds* out) {
  const double p0 = blk[0][0][0], q0 = blk[0][0][1], p7 = blk[7][0][0], q7 = blk[7][0][1];
  const double ta = blk[1][1][1], tb = blk[1][1][2];
  const double ua = blk[3][0][0], ud = blk[3][2][2];
  const double tol = 1e-12 * std::fabs(p0);
  auto eq = [&](double a, double b) { return std::fabs(a - b) <= tol; };
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      if (!eq(blk[0][c][d], c == d ? p0 : q0)) return false;
      if (!eq(blk[7][c][d], c == d ? p7 : q7)) return false;
    }
  for (int t = 0; t < 3; ++t) {
    const int k = 1 << t, ca = (t + 1) % 3, cb = (t + 2) % 3;
    if (!eq(blk[k][ca][ca], ta) || !eq(blk[k][cb][cb], ta) || !eq(blk[k][ca][cb], tb) ||
        !eq(blk[k][cb][ca], tb))
      return false;
    const int k2 = 7 ^ (1 << t);
    if (!eq(blk[k2][ca][ca], ua) || !eq(blk[k2][cb][cb], ua) || !eq(blk[k2][ca][cb], ua) ||
        !eq(blk[k2][cb][ca], ua) || !eq(blk[k2][t][t], ud))
      return false;
  }
  out->a0 = p0 - q0;
  out->b0 = q0;
  out->a7 = p7 - q7;
  out->b7 = q7;
  out->ta = ta;
  out->tb = tb;
  out->ua = ua;
  out->ud = ud;
  return true;
}

std::vector<FilterTap> filter_taps(double rmin) {
  std::vector<FilterTap> taps;
  const int R = (int)std::ceil(rmin) - 1;
  for (int dk = -R; dk <= R; ++dk)
    for (int dj = -R; dj <= R; ++dj)
      for (int di = -R; di <= R; ++di) {
        const double w = rmin - std::sqrt((double)(di * di + dj * dj + dk * dk));
        if (w > 0.0) taps.push_back(FilterTap{di, dj, dk, w});
      }
  return taps;
}

}  // namespace tomo
