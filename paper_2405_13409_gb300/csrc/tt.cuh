// 2-bounce refraction (TT) chains: FP64 construction of the bivariate system
// of Sec. 3.4-3.5 in per-thread scratch, and the warp-cooperative Bezout
// determinant sign of Sec. 4.2 (k >= 2 branch).
//
// System (reading of the paper's TT row, Table tab_sum): with the scaled
// refracted direction D at x1 (Eq. eq_refr_rational, sqrt(beta) replaced by
// a rational piece) and the Moller-Trumbore mapping u2 = (u~, v~) / kappa
// (Eq. eq_rct), the segment x2 - x1 is parallel to D, so the constraints at
// x2 are written with D in place of x2 - x1 (kappa (x2 - x1) = t~ D would
// make t~ a common factor of both polynomials and the resultant vanish):
//   a = (D x (x3 - x1)) . M2                                   degree 16
//   b = eta1^2 |K2|^2 ((D x M2) . e)^2 - eta2^2 |D|^2 ((K2 x M2) . e)^2   46
// with M2 = kappa n2, K2 = kappa (x3 - x2), e the projection axis.  When T2
// has one normal, M2 is that normal (kappa would otherwise be a common
// factor).
#pragma once
#include "polys.cuh"

namespace spoly {

constexpr int kTTDa = 16;             // total degree of a
constexpr int kTTDb = 46;             // total degree of b
constexpr int kTTDmap = 8;            // u~, v~ (kappa: 7)
constexpr int kTTMaxN = 32;           // largest Bezout size of the warp kernels
constexpr int kSqrtPieces = 6;
constexpr double kTTRootTol = 1e-10;  // FP64 polish width in v1
constexpr int kTTPaperIters = 10;     // FP32 bisection iterations (Sec. 4.2)
constexpr int kTTNewtonIters = 8;
constexpr double kTTIllCond = 1e-7;

// Rational sqrt pieces: breaks[7], coeffs[6][3] = (c0, c1, d1) of
// (c0 + c1 x) / (1 + d1 x) on [breaks[k], breaks[k+1]).
struct SqrtTable {
  double breaks[kSqrtPieces + 1];
  double c[kSqrtPieces][3];
};

// Per-system record written by the build kernel.
struct TTSys {
  int32_t chain;   // index in the k = 2 chain list
  int32_t piece;   // sqrt piece
  int32_t da, db;  // trimmed u-degrees (-1: degenerate)
  int32_t n;       // Bezout size max(da, db)
  int32_t ks;      // u = 2^ks w balances the u-coefficients (FP32 copy)
  uint32_t flags;  // SPOLY_FLAG_SQRT_SPLIT
  int32_t first_item, n_items;  // bracket range in the queue (sign kernel)
  int32_t noisy;   // 1 + slot of the FP32 signs kept for the FP64 re-sampling pass (0: none)
};

// Arena of one system (FP64, element e at base[e * stride]): the final a, b
// and the mapping polynomials (the kept part, copied to the system's scratch
// row), then the intermediates of the construction.
constexpr int kOffA = 0;
constexpr int kOffB = kOffA + bsize(kTTDa);
constexpr int kOffUt = kOffB + bsize(kTTDb);
constexpr int kOffVt = kOffUt + bsize(kTTDmap);
constexpr int kOffKap = kOffVt + bsize(kTTDmap);
constexpr int kTTKeep = kOffKap + bsize(kTTDmap);  // kept for the polish and path phases
// intermediates, in the order tt_construct takes them: five linear vectors,
// three quadratics, four quartics, a cubic and two degree-7 vectors, three
// degree-8 vectors, four degree-16 and two degree-32 polynomials
constexpr int kTTWork = 5 * 3 * bsize(1) + 3 * bsize(2) + 4 * bsize(4) + 3 * bsize(3) + 2 * 3 * bsize(7) +
                        3 * 3 * bsize(8) + 4 * bsize(16) + 2 * bsize(32);
constexpr int kTTScratch = kTTKeep + kTTWork;
// FP32 copy for the sign kernel: a and b scaled and normalised.
constexpr int kTT32 = bsize(kTTDa) + bsize(kTTDb);

#ifndef SPOLY_HOST_BUILD
// A bivariate polynomial of total degree D (coefficient k at p[k * st]).
struct GP {
  double* p;
  int64_t st;
  int D;
  SPOLY_D double& at(int i, int j) const { return p[int64_t(bidx(D, i, j)) * st]; }
  SPOLY_D double& k(int idx) const { return p[int64_t(idx) * st]; }
};

struct Arena {
  double* base;
  int64_t st;
  int off;
  SPOLY_D GP take(int D) {
    GP g{base + int64_t(off) * st, st, D};
    off += bsize(D);
    return g;
  }
};

// The construction helpers below are warp-cooperative: all 32 lanes of a
// warp call them together with the same arguments (polynomials in the
// warp's shared-memory arena); each returns after a __syncwarp, so its
// results are visible to every lane.

// (i, j) of the graded index t of a degree-D polynomial: row offsets are
// off(i) = i (2D + 3 - i) / 2.
SPOLY_D void flat_to_ij(int D, int t, int& i, int& j) {
  const float B = float(2 * D + 3);
  int r = int((B - sqrtf(fmaxf(B * B - 8.0f * float(t), 0.0f))) * 0.5f);
  r = max(0, min(r, D));
  while (r > 0 && r * (2 * D + 3 - r) / 2 > t) --r;
  while (r < D && (r + 1) * (2 * D + 3 - (r + 1)) / 2 <= t) ++r;
  i = r;
  j = t - r * (2 * D + 3 - r) / 2;
}

SPOLY_D void gp_zero(const GP& c) {
  for (int t = threadIdx.x & 31; t < bsize(c.D); t += 32) c.k(t) = 0.0;
  __syncwarp();
}

// c(0, 0) += x
SPOLY_D void gp_add00(const GP& c, double x) {
  if ((threadIdx.x & 31) == 0) c.at(0, 0) += x;
  __syncwarp();
}

// c += s * a * b, keeping only the terms of total degree <= c.D (the others
// vanish when the factors' true degrees are below their slots').  Lanes take
// the terms of b; the terms of a run in step, one __syncwarp apart, so two
// lanes never update one coefficient at once.
SPOLY_D void gp_mac_trunc(const GP& c, const GP& a, const GP& b, double s) {
  const int lane = threadIdx.x & 31;
  const int nb = bsize(b.D);
  for (int t0 = 0; t0 < nb; t0 += 32) {
    const int t = t0 + lane;
    int i2 = 0, j2 = 0;
    double y = 0.0;
    if (t < nb) {
      flat_to_ij(b.D, t, i2, j2);
      y = s * b.k(t);
    }
    for (int i1 = 0; i1 <= a.D; ++i1)
      for (int j1 = 0; i1 + j1 <= a.D; ++j1) {
        const double x = a.at(i1, j1);
        if (x == 0.0) continue;  // the same for every lane
        if (y != 0.0 && i1 + j1 + i2 + j2 <= c.D)
          c.at(i1 + i2, j1 + j2) = fma(x, y, c.at(i1 + i2, j1 + j2));
        __syncwarp();
      }
  }
  __syncwarp();
}

// c += s * a * b  (c.D >= a.D + b.D)
SPOLY_D void gp_mac(const GP& c, const GP& a, const GP& b, double s) { gp_mac_trunc(c, a, b, s); }

// c += s * a  (c.D >= a.D)
SPOLY_D void gp_axpy(const GP& c, const GP& a, double s) {
  for (int t = threadIdx.x & 31; t < bsize(a.D); t += 32) {
    int i, j;
    flat_to_ij(a.D, t, i, j);
    c.at(i, j) = fma(s, a.k(t), c.at(i, j));
  }
  __syncwarp();
}

SPOLY_D double gp_eval(const GP& a, double u, double v) {
  double r = 0.0;
  for (int i = a.D; i >= 0; --i) {
    double row = 0.0;
    for (int j = a.D - i; j >= 0; --j) row = fma(row, v, a.at(i, j));
    r = fma(r, u, row);
  }
  return r;
}

struct GV {
  GP x, y, z;
};

SPOLY_D GV gv_take(Arena& A, int D) { return {A.take(D), A.take(D), A.take(D)}; }
SPOLY_D void gv_zero(const GV& v) {
  gp_zero(v.x);
  gp_zero(v.y);
  gp_zero(v.z);
}
// r += s * (a . b)
SPOLY_D void gv_dot_mac(const GP& r, const GV& a, const GV& b, double s) {
  gp_mac(r, a.x, b.x, s);
  gp_mac(r, a.y, b.y, s);
  gp_mac(r, a.z, b.z, s);
}
// r += s * ((a x b) . e) for an axis e (component ax: 0 x, 1 y, 2 z)
SPOLY_D void gv_cross_axis_mac(const GP& r, const GV& a, const GV& b, int ax, double s) {
  const GP* A[3] = {&a.x, &a.y, &a.z};
  const GP* B[3] = {&b.x, &b.y, &b.z};
  const int i = (ax + 1) % 3, j = (ax + 2) % 3;
  gp_mac(r, *A[i], *B[j], s);
  gp_mac(r, *A[j], *B[i], -s);
}
// r += s * ((a x k) . m) with constant vectors k, m  == s * a . (k x m)
SPOLY_D void gv_dot_const_mac(const GP& r, const GV& a, d3 w, double s) {
  gp_axpy(r, a.x, s * w.x);
  gp_axpy(r, a.y, s * w.y);
  gp_axpy(r, a.z, s * w.z);
}

// Affine vector polynomial c0 + u cu + v cv into a degree-D slot.
SPOLY_D void gv_set_lin(const GV& v, d3 c0, d3 cu, d3 cv) {
  gv_zero(v);
  if ((threadIdx.x & 31) == 0) {
    v.x.at(0, 0) = c0.x;
    v.x.at(1, 0) = cu.x;
    v.x.at(0, 1) = cv.x;
    v.y.at(0, 0) = c0.y;
    v.y.at(1, 0) = cu.y;
    v.y.at(0, 1) = cv.y;
    v.z.at(0, 0) = c0.z;
    v.z.at(1, 0) = cu.z;
    v.z.at(0, 1) = cv.z;
  }
  __syncwarp();
}
#endif

}  // namespace spoly
