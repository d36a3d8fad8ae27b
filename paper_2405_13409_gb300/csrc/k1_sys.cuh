// Per-candidate device code of the 1-bounce solve, shared by the isolation,
// side and finish kernels.
//
// Per candidate (query q, triangle t), following Sec. 4.3:
//   coefficient phase   a(u,v), b(u,v) in FP64 (Sec. 3.5 "R", "T")
//   elimination phase   Bezout entries in FP64 (Eq. eq_bezout), converted to
//                       T = float (mixed) or double (plain)
//   univariate phase    r(z) = det by memoised Laplace expansion and
//                       recursive-derivative isolation (Sec. 4.2) in T
//   polish              FP64: the same resultant in FP64, each bracket's root
//                       by Newton steps inside it (then bisection)
//   path phase          FP64: u from a(u, v*) = 0, Newton on (a, b),
//                       path-space check of Eq. eq_ch, in-triangle test.
#pragma once
#include "k1.cuh"
#include "polys.cuh"

namespace spoly {
template <int DB>
struct K1Sys {
  BPd<2> a;
  BPd<DB> b;
  int na, nb, n;
  Scaling sc;
};

// Coefficient phase for one candidate; false if the system is degenerate.
template <int DB>
SPOLY_D bool k1_system(const TriD& tr, const QueryD& q, K1Sys<DB>& s) {
  const Frame f = make_frame(tr, q);
  s.a = build_a(f);
  if constexpr (DB == 4) {
    s.b = build_b_R(f, tr, choose_edge(tr, q));
  } else {
    s.b = build_b_T(f, choose_b(tr, q), q.eta0, q.eta1);
  }
  s.na = deg_u<2>(s.a);
  s.nb = deg_u<DB>(s.b);
  s.n = max(s.na, s.nb);
  if (s.na < 0 || s.nb < 0 || s.n < 1) return false;
  s.sc = choose_scaling<DB>(s.b, s.nb);
  apply_scaling<2>(s.a, s.sc);
  apply_scaling<DB>(s.b, s.sc);
  return true;
}

// Largest resultant degree bound N (DA + DB - N) over the Bezout sizes N <= 6
// of T (DA + DB - 1 = 7): 16 at N = 4.
constexpr int kRD = 16;  // largest resultant degree bound over all Bezout sizes

// u-coefficients of a at a fixed z: A_m(z) for m <= 2 (zero beyond na).
template <typename T>
SPOLY_D void a_at(const BPd<2>& a, int na, T z, T (&am)[3]) {
#pragma unroll
  for (int m = 0; m <= 2; ++m) {
    T s = T(0);
#pragma unroll
    for (int j = 2 - m; j >= 0; --j) s = fma(s, z, T(a.c[bidx(2, m, j)]));
    am[m] = (m <= na) ? s : T(0);
  }
}

// Real roots of A2 w^2 + A1 w + A0 (stable formulas); flags tangent roots.
template <typename T>
SPOLY_D int quad_roots(T A0, T A1, T A2, T tang, T (&w)[2], uint32_t (&fl)[2]) {
  const T mag = fabs(A0) + fabs(A1) + fabs(A2);
  if (!(mag > T(0))) return 0;
  if (fabs(A2) <= T(kTrim) * mag) {
    if (fabs(A1) <= T(kTrim) * mag) return 0;
    w[0] = -A0 / A1;
    fl[0] = 0u;
    return 1;
  }
  const T disc = A1 * A1 - T(4) * A2 * A0;
  const T dmag = A1 * A1 + fabs(T(4) * A2 * A0);
  if (disc < T(0)) {
    if (-disc <= tang * dmag) {
      w[0] = -A1 / (T(2) * A2);
      fl[0] = SPOLY_FLAG_TANGENT | SPOLY_FLAG_ILL_COND;
      return 1;
    }
    return 0;
  }
  const T sq = sqrt(disc);
  const T qq = T(-0.5) * (A1 + (A1 >= T(0) ? sq : -sq));
  if (qq == T(0)) {
    w[0] = T(0);
    fl[0] = 0u;
    return 1;
  }
  w[0] = qq / A2;
  w[1] = A0 / qq;
  fl[0] = fl[1] = (disc <= tang * dmag) ? (SPOLY_FLAG_TANGENT | SPOLY_FLAG_ILL_COND) : 0u;
  return 2;
}

// Path-space check of the specular vertex (Eq. eq_ch) with the sidedness
// reading: reflection keeps x0 and x2 on one side of the tangent plane and
// needs |h| > 1e-9; refraction crosses it.  residual = |h x n| / (|h| |n|).
SPOLY_D bool vertex_check(d3 xprev, d3 x, d3 xnext, d3 n, int type, double eta_in, double eta_out,
                          double* residual, uint32_t* flags) {
  const d3 d0 = x - xprev, d1 = xnext - x;
  const double l0 = norm(d0), l1 = norm(d1), ln = norm(n);
  if (!(l0 > 0.0) || !(l1 > 0.0) || !(ln > 0.0)) return false;
  const d3 h = (type == SPOLY_R) ? ((1.0 / l1) * d1 - (1.0 / l0) * d0)
                                 : ((eta_out / l1) * d1 - (eta_in / l0) * d0);
  const double lh = norm(h);
  if (!(lh > 1e-9)) return false;
  *residual = norm(cross(h, n)) / (lh * ln);
  const double s0 = dot(d0, n), s1 = dot(d1, n);
  if (dot(xprev - x, n) < 0.0) *flags |= SPOLY_FLAG_BACKFACE;
  if (s0 == 0.0 || s1 == 0.0) return false;
  if (type == SPOLY_R) return (s0 < 0.0) != (s1 < 0.0);
  return (s0 < 0.0) == (s1 < 0.0);
}

// Newton on the scaled system (a, b)(w, z) = 0; accepted when the move in
// (u, v) stays within kNewtonMove.  A step below 1e-16 in (u, v) ends it
// (the next one would move the root by less than its last bit).
template <int DB>
SPOLY_D void newton_ab(const K1Sys<DB>& s, double& w, double& z) {
  double ww = w, zz = z;
  for (int it = 0; it < kNewtonIters; ++it) {
    double fa, a1, a2, fb, b1, b2;
    beval_grad<2>(s.a, ww, zz, &fa, &a1, &a2);
    beval_grad<DB>(s.b, ww, zz, &fb, &b1, &b2);
    const double det = a1 * b2 - a2 * b1;
    if (!(fabs(det) > 0.0)) break;
    const double dw = (fa * b2 - fb * a2) / det;
    const double dz = (a1 * fb - b1 * fa) / det;
    if (!isfinite(dw) || !isfinite(dz)) break;
    ww -= dw;
    zz -= dz;
    if (fabs(dw) * s.sc.s <= 1e-16 && fabs(dz) * s.sc.t <= 1e-16) break;
  }
  if (fabs(ww - w) * s.sc.s <= kNewtonMove && fabs(zz - z) * s.sc.t <= kNewtonMove) {
    w = ww;
    z = zz;
  }
}

}  // namespace spoly
