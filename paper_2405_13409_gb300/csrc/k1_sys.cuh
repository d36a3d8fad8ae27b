// Per-candidate device code of the 1-bounce solve, shared by the isolation,
// generic and polish kernels.
//
// Per candidate (query q, triangle t), following Sec. 5.3:
//   coefficient phase   a(u,v), b(u,v) in FP64 (Sec. 3.5 "R", "T")
//   elimination phase   Bezout entries in FP64 (Eq. eq_bezout), converted to
//                       T = float (mixed) or double (plain)
//   univariate phase    r(z) = det by memoised Laplace expansion and
//                       recursive-derivative isolation (Sec. 5.2) in T
//   path phase          FP64: bisection of the numeric determinant near the
//                       bracket, u from a(u, v*) = 0, Newton on (a, b),
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

// -------------------------------------------------------------- polish
// Numeric Bezout matrix from the u-coefficients of a and b at one z.
template <int NM, int DB>
SPOLY_D void numeric_bezout(const double (&av)[3], const double (&bv)[DB + 1], int n, double (&m)[NM][NM]) {
#pragma unroll
  for (int i = 0; i < NM; ++i)
#pragma unroll
    for (int j = 0; j < NM; ++j) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        if (k > i || k > NM - 1 - j) continue;
        if (k > n - 1 - j) continue;
        const int p = i - k, q = j + 1 + k;
        if (p <= 2 && q <= DB) s = fma(av[p], bv[q], s);
        if (q <= 2 && p <= DB) s = fma(-bv[p], av[q], s);
      }
      m[i][j] = (i < n && j < n) ? s : 0.0;
    }
}

template <int DB>
SPOLY_D double det_at(const K1Sys<DB>& s, double z) {
  double av[3], bv[DB + 1];
#pragma unroll
  for (int mm = 0; mm <= 2; ++mm) {
    double acc = 0.0;
#pragma unroll
    for (int j = 2 - mm; j >= 0; --j) acc = fma(acc, z, s.a.c[bidx(2, mm, j)]);
    av[mm] = (mm <= s.na) ? acc : 0.0;
  }
#pragma unroll
  for (int mm = 0; mm <= DB; ++mm) {
    double acc = 0.0;
#pragma unroll
    for (int j = DB - mm; j >= 0; --j) acc = fma(acc, z, s.b.c[bidx(DB, mm, j)]);
    bv[mm] = (mm <= s.nb) ? acc : 0.0;
  }
  constexpr int NM = (DB == 4) ? 4 : 6;
  double m[NM][NM];
  numeric_bezout<NM, DB>(av, bv, s.n, m);
  return det_ge<NM>(m, s.n);
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
// (u, v) stays within kNewtonMove.
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
  }
  if (fabs(ww - w) * s.sc.s <= kNewtonMove && fabs(zz - z) * s.sc.t <= kNewtonMove) {
    w = ww;
    z = zz;
  }
}

template <int DB>
SPOLY_D int k1_polish_one(const TriD& tr, const QueryD& qd, const RootItem& it, int q, int t,
                          spoly_path (&out)[6], unsigned& n_u, unsigned& lost) {
  K1Sys<DB> s;
  if (!k1_system<DB>(tr, qd, s)) return 0;
  const double zmin = -kDelta / s.sc.t, zmax = (1.0 + kDelta) / s.sc.t;
  double zlo = it.zlo, zhi = it.zhi;
  uint32_t vflags = it.flags;
  double zs;
  if (vflags & SPOLY_FLAG_TANGENT) {
    zs = 0.5 * (zlo + zhi);
  } else {
    double flo = det_at<DB>(s, zlo), fhi = det_at<DB>(s, zhi);
    double wdt = fmax(zhi - zlo, 1e-15 / s.sc.t);
    int grow = 0;
    while (!((flo < 0.0) != (fhi < 0.0)) && flo != 0.0 && fhi != 0.0 && grow < 20) {
      zlo = fmax(zmin - wdt, zlo - wdt);
      zhi = fmin(zmax + wdt, zhi + wdt);
      wdt *= 2.0;
      flo = det_at<DB>(s, zlo);
      fhi = det_at<DB>(s, zhi);
      ++grow;
    }
    if (flo == 0.0) {
      zs = zlo;
    } else if (fhi == 0.0) {
      zs = zhi;
    } else if ((flo < 0.0) != (fhi < 0.0)) {
      const double tol = kPolishTol / s.sc.t;
      while (zhi - zlo > tol) {
        const double zm = 0.5 * (zlo + zhi);
        if (!(zm > zlo && zm < zhi)) break;
        const double fm = det_at<DB>(s, zm);
        if (fm == 0.0) {
          zlo = zhi = zm;
          break;
        }
        if ((fm < 0.0) == (flo < 0.0)) {
          zlo = zm;
          flo = fm;
        } else {
          zhi = zm;
        }
      }
      zs = 0.5 * (zlo + zhi);
    } else {
      ++lost;
      return 0;
    }
    // Ill-conditioning: |r'(v*)| / sum|r_i| from a central difference of the
    // FP64 determinant (h = 1e-6 in v).
    const double h = 1e-6 / s.sc.t;
    const double slope = (det_at<DB>(s, zs + h) - det_at<DB>(s, zs - h)) / (2.0 * h);
    const double scale = ldexp(double(it.rscale), it.pad);
    if (fabs(slope) / s.sc.t < kIllCond * scale) vflags |= SPOLY_FLAG_ILL_COND;
  }
  if (zs < zmin || zs > zmax) return 0;
  const double v0 = zs * s.sc.t;
  // u from a(u, v*) = 0 (Sec. 5.3); fall back to b if a(., v*) vanishes.
  double am[3];
  a_at<double>(s.a, s.na, zs, am);
  double amag = 0.0;
#pragma unroll
  for (int k = 0; k < bsize(2); ++k) amag = fmax(amag, fabs(s.a.c[k]));
  double wr[DB + 1];
  uint32_t wf[DB + 1];
  int nw = 0;
  const double wlo = -kDelta / s.sc.s, whi = (1.0 - v0 + kDelta) / s.sc.s;
  if (fmax(fabs(am[0]), fmax(fabs(am[1]), fabs(am[2]))) > kTrim * amag) {
    double w2[2];
    uint32_t f2[2];
    const int n2 = quad_roots<double>(am[0], am[1], am[2], 1e-12, w2, f2);
    for (int i = 0; i < n2; ++i)
      if (w2[i] >= wlo && w2[i] <= whi) {
        wr[nw] = w2[i];
        wf[nw] = f2[i];
        ++nw;
      }
  } else {
    double bv[DB + 1];
    double bs = 0.0;
#pragma unroll
    for (int mm = 0; mm <= DB; ++mm) {
      double acc = 0.0;
#pragma unroll
      for (int j = DB - mm; j >= 0; --j) acc = fma(acc, zs, s.b.c[bidx(DB, mm, j)]);
      bv[mm] = (mm <= s.nb) ? acc : 0.0;
      bs += fabs(bv[mm]);
    }
    double blo[DB + 1], bhi[DB + 1];
    uint32_t bfl[DB + 1];
    const int n2 = isolate<double, DB>(bv, s.nb, wlo, whi, kIsoTol64 / s.sc.s * 1e-2, kTangent64, bs, blo, bhi, bfl);
    for (int i = 0; i < n2 && nw <= DB; ++i) {
      wr[nw] = 0.5 * (blo[i] + bhi[i]);
      wf[nw] = bfl[i];
      ++nw;
    }
  }
  int np = 0;
  for (int i = 0; i < nw; ++i) {
    ++n_u;
    double w = wr[i], z = zs;
    newton_ab<DB>(s, w, z);
    const double u = w * s.sc.s, v = z * s.sc.t;
    uint32_t flags = vflags | wf[i];
    const d3 x1 = tr.p0 + u * (tr.p1 - tr.p0) + v * (tr.p2 - tr.p0);
    const d3 nn = tr.n0 + u * (tr.n1 - tr.n0) + v * (tr.n2 - tr.n0);
    double res = 1.0;
    if (!vertex_check(qd.x0, x1, qd.x2, nn, qd.type, qd.eta0, qd.eta1, &res, &flags)) continue;
    if (!(res < kResidual)) continue;
    const double wmin = fmin(fmin(u, v), 1.0 - u - v);
    if (wmin < 0.0) continue;
    if (wmin < kEdgeEps) flags |= SPOLY_FLAG_EDGE;
    bool dup = false;
    for (int k = 0; k < np; ++k)
      if (fabs(out[k].uv[0][0] - u) <= 1e-9 && fabs(out[k].uv[0][1] - v) <= 1e-9) {
        out[k].flags |= flags;
        dup = true;
      }
    if (dup || np >= 6) continue;
    spoly_path& p = out[np++];
    p.query = q;
    p.tri[0] = t;
    p.tri[1] = -1;
    p.reserved = 0;
    p.uv[0][0] = u;
    p.uv[0][1] = v;
    p.uv[1][0] = 0.0;
    p.uv[1][1] = 0.0;
    p.x[0][0] = x1.x;
    p.x[0][1] = x1.y;
    p.x[0][2] = x1.z;
    p.x[1][0] = p.x[1][1] = p.x[1][2] = 0.0;
    p.residual = float(res);
    p.flags = flags;
  }
  return np;
}

}  // namespace spoly
