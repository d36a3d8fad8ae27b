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

// Bits of RootItem::flags after the v-polish: root 1 in zlo with public flags
// in bits 0-7, root 2 in zhi with public flags in bits 8-15.
constexpr uint32_t kRoot1Valid = 1u << 30;
constexpr uint32_t kRoot2Valid = 1u << 31;

// FP64 bisection of the numeric determinant on [zl, zh] (signs differ).
template <int DB>
SPOLY_D double bisect_det(const K1Sys<DB>& s, double zl, double zh, double fl) {
  const double tol = kPolishTol / s.sc.t;
  while (zh - zl > tol) {
    const double zm = 0.5 * (zl + zh);
    if (!(zm > zl && zm < zh)) break;
    const double fm = det_at<DB>(s, zm);
    if (fm == 0.0) return zm;
    if ((fm < 0.0) == (fl < 0.0)) {
      zl = zm;
      fl = fm;
    } else {
      zh = zm;
    }
  }
  return 0.5 * (zl + zh);
}

// Ill-conditioning of a polished root: |r'(v*)| / sum|r_i| from a central
// difference of the FP64 determinant (h = 1e-6 in v).
template <int DB>
SPOLY_D uint32_t ill_flag(const K1Sys<DB>& s, double z, const RootItem& it) {
  const double h = 1e-6 / s.sc.t;
  const double slope = (det_at<DB>(s, z + h) - det_at<DB>(s, z - h)) / (2.0 * h);
  const double scale = ldexp(double(it.rscale), it.pad);
  return (fabs(slope) / s.sc.t < kIllCond * scale) ? SPOLY_FLAG_ILL_COND : 0u;
}

// Root next to a point c on one side (dir = -1 or +1): step out from c by
// doubling until the FP64 determinant changes sign (within `reach` in v),
// then bisect.  Returns false when no sign change is found.
template <int DB>
SPOLY_D bool side_root(const K1Sys<DB>& s, double c, double fc, int dir, double zmin, double zmax, double* root,
                       double reach = 1e-3) {
  double p = c;
  double w = 1e-8 / s.sc.t;
  const double wmax = reach / s.sc.t;
  while (w <= wmax) {
    double x = c + dir * w;
    if (x < zmin || x > zmax) return false;
    const double fx = det_at<DB>(s, x);
    if (fx == 0.0) {
      *root = x;
      return true;
    }
    if ((fx < 0.0) != (fc < 0.0)) {
      *root = (dir < 0) ? bisect_det<DB>(s, x, p, fx) : bisect_det<DB>(s, p, x, fc);
      return true;
    }
    p = x;
    w *= 2.0;
  }
  return false;
}

// v-polish of one bracket in FP64 (root polishing by bisection near the
// final interval).  A sign-change bracket from the isolation is bisected on
// the numeric determinant to width 1e-12 in v.  A bracket whose FP64 signs
// agree (the FP32 root is displaced) and a tangent bracket (critical point of
// the isolated polynomial) are resolved into the nearest FP64 roots on either
// side.  Writes the roots back into `it`.
template <int DB>
SPOLY_D void k1_polish_v(const TriD& tr, const QueryD& qd, RootItem& it, unsigned& lost) {
  K1Sys<DB> s;
  const uint32_t in_flags = it.flags & 0xffu;
  it.flags = 0u;
  if (!k1_system<DB>(tr, qd, s)) {
    ++lost;
    return;
  }
  const double zmin = -kDelta / s.sc.t, zmax = (1.0 + kDelta) / s.sc.t;
  double r1 = 0.0, r2 = 0.0;
  bool v1 = false, v2 = false;
  uint32_t f1 = 0u, f2 = 0u;
  if (in_flags & SPOLY_FLAG_TANGENT) {
    const double c = 0.5 * (it.zlo + it.zhi);
    const double fc = det_at<DB>(s, c);
    if (fc == 0.0) {
      r1 = c;
      v1 = true;
      f1 = SPOLY_FLAG_TANGENT | SPOLY_FLAG_ILL_COND;
    } else {
      v1 = side_root<DB>(s, c, fc, -1, zmin, zmax, &r1, kSideReach);
      v2 = side_root<DB>(s, c, fc, +1, zmin, zmax, &r2, kSideReach);
    }
  } else {
    const double zlo = it.zlo, zhi = it.zhi;
    const double flo = det_at<DB>(s, zlo), fhi = det_at<DB>(s, zhi);
    if (flo == 0.0) {
      r1 = zlo;
      v1 = true;
    } else if (fhi == 0.0) {
      r1 = zhi;
      v1 = true;
    } else if ((flo < 0.0) != (fhi < 0.0)) {
      r1 = bisect_det<DB>(s, zlo, zhi, flo);
      v1 = true;
    } else {
      // The FP32 bracket has no FP64 sign change: the FP32 root is displaced.
      // Search outward on both sides for the nearest FP64 roots.
      v1 = side_root<DB>(s, zlo, flo, -1, zmin, zmax, &r1, kSideReach);
      v2 = side_root<DB>(s, zhi, fhi, +1, zmin, zmax, &r2, kSideReach);
    }
  }
  if (v1 && !(f1 & SPOLY_FLAG_TANGENT)) f1 |= ill_flag<DB>(s, r1, it);
  if (v2) f2 |= ill_flag<DB>(s, r2, it);
  v1 = v1 && r1 >= zmin && r1 <= zmax;
  v2 = v2 && r2 >= zmin && r2 <= zmax;
  if (!v1 && !v2) ++lost;
  it.zlo = r1;
  it.zhi = r2;
  it.flags = (v1 ? kRoot1Valid : 0u) | (v2 ? kRoot2Valid : 0u) | (f1 & 0xffu) | ((f2 & 0xffu) << 8);
}

// Path phase (Sec. 5.3) for one polished root z*: u from a(u, v*) = 0 (b if
// a(., v*) vanishes), Newton on (a, b), path-space check of Eq. eq_ch,
// sidedness and the in-triangle test.  Appends up to 6 paths to `out`.
template <int DB>
SPOLY_D int k1_path_root(const K1Sys<DB>& s, const TriD& tr, const QueryD& qd, double zs, uint32_t vflags, int q,
                         int t, spoly_path (&out)[6], int np, unsigned& n_u) {
  const double v0 = zs * s.sc.t;
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

// Path phase of queue item i.  Roots already produced by an earlier bracket
// of the same candidate (items of one candidate are contiguous in the queue)
// or equal to the item's other root within 1e-9 in v are skipped.
template <int DB>
SPOLY_D int k1_path_item(const TriD& tr, const QueryD& qd, const RootItem* queue, int64_t i, int q, int t,
                         spoly_path (&out)[6], unsigned& n_u) {
  const RootItem it = queue[i];
  K1Sys<DB> s;
  if (!k1_system<DB>(tr, qd, s)) return 0;
  const double dtol = 1e-9 / s.sc.t;
  int np = 0;
  for (int r = 0; r < 2; ++r) {
    const uint32_t valid = r == 0 ? kRoot1Valid : kRoot2Valid;
    if (!(it.flags & valid)) continue;
    const double z = r == 0 ? it.zlo : it.zhi;
    bool dup = (r == 1 && (it.flags & kRoot1Valid) && fabs(it.zlo - z) <= dtol);
    for (int64_t j = i - 1; j >= 0 && !dup; --j) {
      const RootItem o = queue[j];
      if (o.chain != it.chain) break;
      if (((o.flags & kRoot1Valid) && fabs(o.zlo - z) <= dtol) || ((o.flags & kRoot2Valid) && fabs(o.zhi - z) <= dtol))
        dup = true;
    }
    if (dup) continue;
    const uint32_t vflags = r == 0 ? (it.flags & 0xffu) : ((it.flags >> 8) & 0xffu);
    np = k1_path_root<DB>(s, tr, qd, z, vflags, q, t, out, np, n_u);
  }
  return np;
}

}  // namespace spoly
