// FP64 v-polish and path phase of the 1-bounce solve (Sec. 4.3).
#pragma once
#include <type_traits>

#include "k1_generic.cuh"

namespace spoly {

// Bits of RootItem::flags after the v-polish: root 1 in zlo with public flags
// in bits 0-7, root 2 in zhi with public flags in bits 8-15.
constexpr uint32_t kRoot1Valid = 1u << 30;
constexpr uint32_t kRoot2Valid = 1u << 31;
constexpr uint32_t kPolished = 1u << 29;  // the item's roots are final (a path re-run skips the polish)

// Generic-size FP64 resultant (runtime n), kept out of line so its large
// local arrays do not shape the register allocation of the common path.
#ifdef SPOLY_HOST_BUILD
#define SPOLY_NOINLINE
#else
#define SPOLY_NOINLINE __device__ __noinline__
#endif
template <int DB>
SPOLY_NOINLINE void k1_r64_generic(const K1Sys<DB>& s, double (&r)[kRD + 1]) {
  double E[6][6][DB + 2];
  for (int i = 0; i < s.n; ++i)
    for (int j = 0; j < s.n; ++j) bezout_entry_rt<DB>(s.a, s.b, s.na, s.nb, s.n, i, j, E[i][j]);
  laplace_rt<DB>(E, s.n, r);
}

// FP64 resultant r(z) of a candidate's scaled system (the same Bezout entries
// and Laplace expansion as the isolation, in FP64), normalised by a power of
// two and trimmed like the isolation's.  Returns its degree (< 1: none; -1
// when r vanishes).  Out of line: a kernel that calls it from several places
// holds one copy of the expansions.
template <int DB>
SPOLY_NOINLINE int k1_r64(const K1Sys<DB>& s, double (&r)[kRD + 1]) {
  constexpr int ED = DB + 1;
#pragma unroll
  for (int c = 0; c <= kRD; ++c) r[c] = 0.0;
  int rd = -1;
  auto sized = [&](auto nc, auto lap) {
    constexpr int N = decltype(nc)::value;
    constexpr int RDn = N * (ED - N + 1);
    double E[sym_size(N, ED)], rr[RDn + 1];
    bezout_sym<double, N, 2, DB>(s.a, s.b, s.na, s.nb, E);
    lap(E, rr);
#pragma unroll
    for (int c = 0; c <= RDn; ++c) r[c] = rr[c];
    rd = RDn;
  };
  using I2 = std::integral_constant<int, 2>;
  using I3 = std::integral_constant<int, 3>;
  using I4 = std::integral_constant<int, 4>;
  using I5 = std::integral_constant<int, 5>;
  using I6 = std::integral_constant<int, 6>;
  if constexpr (DB == 4) {
    if (s.n == 3) sized(I3{}, [](auto& E, auto& rr) { laplace_R3<double>(E, rr); });
    else if (s.n == 4) sized(I4{}, [](auto& E, auto& rr) { laplace_R4<double>(E, rr); });
    else if (s.n == 2) sized(I2{}, [](auto& E, auto& rr) { laplace_R2<double>(E, rr); });
  } else {
    if (s.n == 6) sized(I6{}, [](auto& E, auto& rr) { laplace_T6<double>(E, rr); });
    else if (s.n == 5) sized(I5{}, [](auto& E, auto& rr) { laplace_T5<double>(E, rr); });
    else if (s.n == 4) sized(I4{}, [](auto& E, auto& rr) { laplace_T4<double>(E, rr); });
    else if (s.n == 3) sized(I3{}, [](auto& E, auto& rr) { laplace_T3<double>(E, rr); });
    else if (s.n == 2) sized(I2{}, [](auto& E, auto& rr) { laplace_T2<double>(E, rr); });
  }
  if (rd < 0) {
    k1_r64_generic<DB>(s, r);
    rd = s.n * (ED - s.n + 1);
  }
  long long mb = 0;
#pragma unroll
  for (int c = 0; c <= kRD; ++c) mb = max(mb, absbits(r[c]));
  if (mb == 0) return -1;
  const int e2 = expo_bits(mb) + 1;
  const double Z = (1.0 + kDelta) * scale2(1.0, -s.sc.kt);
  double mxz = 0.0, zp = 1.0;
  double zpow[kRD + 1];
#pragma unroll
  for (int c = 0; c <= kRD; ++c) {
    r[c] = scale2(r[c], -e2);
    zpow[c] = zp;
    mxz = fmax(mxz, fabs(r[c]) * zp);
    zp *= Z;
  }
  int deg = rd;
#pragma unroll
  for (int c = kRD; c >= 1; --c)
    if (c == deg && fabs(r[c]) * zpow[c] <= kTrim * mxz) --deg;
  return deg;
}

SPOLY_D double horner64(const double (&r)[kRD + 1], int deg, double z) {
  double f = 0.0;
#pragma unroll
  for (int c = kRD; c >= 0; --c)
    if (c <= deg) f = fma(f, z, r[c]);
  return f;
}

SPOLY_D double dhorner64(const double (&r)[kRD + 1], int deg, double z) {
  double f = 0.0;
#pragma unroll
  for (int c = kRD; c >= 1; --c)
    if (c <= deg) f = fma(f, z, double(c) * r[c]);
  return f;
}

// r and r' at z by one Horner pass.
SPOLY_D void horner64_d(const double (&r)[kRD + 1], int deg, double z, double* f, double* df) {
  double a = 0.0, d = 0.0;
#pragma unroll
  for (int c = kRD; c >= 0; --c)
    if (c <= deg) {
      d = fma(d, z, a);
      a = fma(a, z, r[c]);
    }
  *f = a;
  *df = d;
}

// Root of r in [zl, zh] (signs differ) to width kPolishTol in v: Newton
// steps from the midpoint while they stay inside the shrinking bracket (a
// step below tol / 4 ends the search), then bisection.  Every FP64
// instruction costs about 64 cycles of an SM sub-partition on this part, so
// the few Newton steps replace the ~20 bisection steps from an FP32 bracket.
SPOLY_D double bisect64(const double (&r)[kRD + 1], int deg, double zl, double zh, double fl, double tol) {
  double x = 0.5 * (zl + zh);
  for (int it = 0; it < 6 && zh - zl > tol; ++it) {
    double f, df;
    horner64_d(r, deg, x, &f, &df);
    if (f == 0.0) return x;
    if ((f < 0.0) == (fl < 0.0)) {
      zl = x;
      fl = f;
    } else {
      zh = x;
    }
    const double st = f / df;
    const double xn = x - st;
    if (!(xn > zl && xn < zh)) break;
    if (fabs(st) <= 0.25 * tol) return xn;
    x = xn;
  }
  while (zh - zl > tol) {
    const double zm = 0.5 * (zl + zh);
    if (!(zm > zl && zm < zh)) break;
    const double fm = horner64(r, deg, zm);
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

// Root of r next to a point c on one side (dir = -1 or +1): step out from c
// by doubling until r changes sign (within `reach` in v), then bisect.
SPOLY_D bool side_root64(const double (&r)[kRD + 1], int deg, double t, double c, double fc, int dir, double zmin,
                         double zmax, double* root) {
  double p = c;
  double w = 1e-8 / t;
  const double wmax = kSideReach / t;
  const double tol = kPolishTol / t;
  while (w <= wmax) {
    const double x = c + dir * w;
    if (x < zmin || x > zmax) return false;
    const double fx = horner64(r, deg, x);
    if (fx == 0.0) {
      *root = x;
      return true;
    }
    if ((fx < 0.0) != (fc < 0.0)) {
      *root = (dir < 0) ? bisect64(r, deg, x, p, fx, tol) : bisect64(r, deg, p, x, fc, tol);
      return true;
    }
    p = x;
    w *= 2.0;
  }
  return false;
}

// Root next to c found by Newton from c (within `reach` of c and inside
// [zmin, zmax]), confirmed by a sign change of r across [x - tol, x + tol].
// A displaced FP32 root is a simple root a little outside its bracket, which
// this finds in a few steps.
SPOLY_D bool newton_root64(const double (&r)[kRD + 1], int deg, double c, double zmin, double zmax, double reach,
                           double tol, double* root) {
  double x = c;
  for (int it = 0; it < 10; ++it) {
    double f, df;
    horner64_d(r, deg, x, &f, &df);
    if (f == 0.0) {
      *root = x;
      return true;
    }
    if (!(fabs(df) > 0.0)) return false;
    const double st = f / df;
    x -= st;
    if (!(x >= zmin && x <= zmax) || !(fabs(x - c) <= reach)) return false;
    if (fabs(st) <= 0.25 * tol) {
      const double fl = horner64(r, deg, x - tol), fh = horner64(r, deg, x + tol);
      if (fl == 0.0 || fh == 0.0 || (fl < 0.0) != (fh < 0.0)) {
        *root = x;
        return true;
      }
      return false;
    }
  }
  return false;
}

// ILL_COND when |r'(v*)| / sum_i |r_i| < kIllCond (v-domain coefficients:
// r(v) = p(v / t), so r_i = p_i t^-i and r'(v) = p'(z) / t).
SPOLY_D uint32_t ill_flag64(const double (&r)[kRD + 1], int deg, double t, double z) {
  double S = 0.0, ti = 1.0;
  const double it = 1.0 / t;  // t is a power of two: exact
#pragma unroll
  for (int c = 0; c <= kRD; ++c) {
    if (c <= deg) S += fabs(r[c]) * ti;
    ti *= it;
  }
  return (fabs(dhorner64(r, deg, z)) / t < kIllCond * S) ? SPOLY_FLAG_ILL_COND : 0u;
}

// v-polish of one bracket in FP64 on the FP64 resultant of the candidate's
// system s (ok: k1_system succeeded).  A sign-change bracket from the
// isolation is refined to width 1e-12 in v.  A bracket whose FP64 signs agree
// (the FP32 root is displaced) takes the Newton root next to its centre;
// failing that, and for a tangent bracket (critical point of the isolated
// polynomial), the nearest FP64 roots on either side within kSideReach.
// Writes the roots back into `it`.
// r64 / deg64: the candidate's FP64 resultant when the caller has it
// (nullptr: formed here).
template <int DB>
SPOLY_D void k1_polish_v(const K1Sys<DB>& s, bool ok, RootItem& it, unsigned& lost, const double* r64 = nullptr,
                         int deg64 = -1) {
  const uint32_t in_flags = it.flags & 0xffu;
  it.flags = 0u;
  double r[kRD + 1];
  int deg = -1;
  if (ok && r64) {
#pragma unroll
    for (int c = 0; c <= kRD; ++c) r[c] = r64[c];
    deg = deg64;
  } else if (ok) {
    deg = k1_r64<DB>(s, r);
  }
  if (deg < 1) {
    ++lost;
    return;
  }
  const double t = s.sc.t, tol = kPolishTol / t;
  const double zmin = -kDelta / t, zmax = (1.0 + kDelta) / t;
  double r1 = 0.0, r2 = 0.0;
  bool v1 = false, v2 = false;
  uint32_t f1 = 0u, f2 = 0u;
  const double zlo = it.zlo, zhi = it.zhi;
  const double flo = horner64(r, deg, zlo), fhi = horner64(r, deg, zhi);
  if (in_flags & SPOLY_FLAG_TANGENT) {
    const double c = 0.5 * (zlo + zhi), fc = horner64(r, deg, c);
    if (fc == 0.0) {
      r1 = c;
      v1 = true;
      f1 = SPOLY_FLAG_TANGENT | SPOLY_FLAG_ILL_COND;
    } else {
      v1 = side_root64(r, deg, t, c, fc, -1, zmin, zmax, &r1);
      v2 = side_root64(r, deg, t, c, fc, +1, zmin, zmax, &r2);
    }
  } else if (flo == 0.0) {
    r1 = zlo;
    v1 = true;
  } else if (fhi == 0.0) {
    r1 = zhi;
    v1 = true;
  } else if ((flo < 0.0) != (fhi < 0.0)) {
    r1 = bisect64(r, deg, zlo, zhi, flo, tol);
    v1 = true;
  } else if (newton_root64(r, deg, 0.5 * (zlo + zhi), zmin, zmax, kSideReach / t, tol, &r1)) {
    v1 = true;
  } else {
    v1 = side_root64(r, deg, t, zlo, flo, -1, zmin, zmax, &r1);
    v2 = side_root64(r, deg, t, zhi, fhi, +1, zmin, zmax, &r2);
  }
  if (v1 && !(f1 & SPOLY_FLAG_TANGENT)) f1 |= ill_flag64(r, deg, t, r1);
  if (v2) f2 |= ill_flag64(r, deg, t, r2);
  v1 = v1 && r1 >= zmin && r1 <= zmax;
  v2 = v2 && r2 >= zmin && r2 <= zmax;
  if (!v1 && !v2) ++lost;
  it.zlo = r1;
  it.zhi = r2;
  it.flags = (v1 ? kRoot1Valid : 0u) | (v2 ? kRoot2Valid : 0u) | (f1 & 0xffu) | ((f2 & 0xffu) << 8);
}

// Path phase (Sec. 4.3) for one polished root z*: u from a(u, v*) = 0 (b if
// a(., v*) vanishes), Newton on (a, b), path-space check of Eq. eq_ch,
// sidedness and the in-triangle test.  Appends up to 6 paths to `out`.
template <int DB>
SPOLY_D int k1_path_root(const K1Sys<DB>& s, const TriD& tr, const QueryD& qd, double zs, uint32_t vflags, int q,
                         int t, int chain, spoly_path (&out)[6], int np, unsigned& n_u, const PixelFilter& pix) {
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
    int qout = q;
    if (pix.on) {
      int64_t pq;
      if (!project_pixel(pix, x1.x, x1.y, x1.z, &pq)) continue;
      if (pix.assign) qout = int(pq);
      else if (pq != q) continue;
    }
    bool dup = false;
    for (int k = 0; k < np; ++k)
      if (fabs(out[k].uv[0][0] - u) <= 1e-9 && fabs(out[k].uv[0][1] - v) <= 1e-9) {
        out[k].flags |= flags;
        dup = true;
      }
    if (dup || np >= 6) continue;
    spoly_path& p = out[np++];
    p.query = qout;
    p.tri[0] = t;
    p.tri[1] = -1;
    p.chain = chain;
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

// Paths of both polished roots of one queue item (roots within `dtol` of an
// earlier root of the item, or of `skip_z` roots, are skipped).
template <int DB>
SPOLY_D int k1_item_paths(const K1Sys<DB>& s, const TriD& tr, const QueryD& qd, const RootItem& it, int q, int t,
                          spoly_path (&out)[6], int np, unsigned& n_u, const PixelFilter& pix,
                          const RootItem* earlier, int64_t n_earlier) {
  const double dtol = 1e-9 / s.sc.t;
  for (int r = 0; r < 2; ++r) {
    const uint32_t valid = r == 0 ? kRoot1Valid : kRoot2Valid;
    if (!(it.flags & valid)) continue;
    const double z = r == 0 ? it.zlo : it.zhi;
    bool dup = (r == 1 && (it.flags & kRoot1Valid) && fabs(it.zlo - z) <= dtol);
    for (int64_t j = 0; j < n_earlier && !dup; ++j) {
      const RootItem o = earlier[j];
      if (((o.flags & kRoot1Valid) && fabs(o.zlo - z) <= dtol) || ((o.flags & kRoot2Valid) && fabs(o.zhi - z) <= dtol))
        dup = true;
    }
    if (dup) continue;
    const uint32_t vflags = r == 0 ? (it.flags & 0xffu) : ((it.flags >> 8) & 0xffu);
    np = k1_path_root<DB>(s, tr, qd, z, vflags, q, t, it.chain, out, np, n_u, pix);
  }
  return np;
}

// FP64 polish (once per item) and path phase of the n items of one
// candidate, in their isolation order.  A root equal within 1e-9 in v to a
// root of an earlier item, or to the item's other root, is skipped; so is a
// path within 1e-9 in (u, v) of a path of an earlier item (two brackets
// around a near-double root of r(v) whose Newton refinements meet), so that
// each candidate reports a solution once, like the oracle's merge rule.
// Every path goes to emit(path).
constexpr int kChainHist = 24;  // earlier-item paths kept for the duplicate test
template <int DB, typename Emit>
SPOLY_D void k1_chain_solve(const K1Sys<DB>& s, bool ok, const TriD& tr, const QueryD& qd, RootItem* items, int n,
                            int q, int t, const PixelFilter& pix, unsigned& lost, unsigned& n_u, Emit&& emit,
                            const double* r64 = nullptr, int deg64 = -1) {
  for (int k = 0; k < n; ++k) {
    RootItem it = items[k];
    if (!(it.flags & kPolished)) {
      k1_polish_v<DB>(s, ok, it, lost, r64, deg64);
      it.flags |= kPolished;
      items[k] = it;
    }
  }
  if (!ok) return;
  double hu[kChainHist], hv[kChainHist];
  int nh = 0;
  for (int k = 0; k < n; ++k) {
    spoly_path cur[6];
    const int np = k1_item_paths<DB>(s, tr, qd, items[k], q, t, cur, 0, n_u, pix, items, k);
    for (int m = 0; m < np; ++m) {
      bool dup = false;
      for (int h = 0; h < nh; ++h)
        if (fabs(hu[h] - cur[m].uv[0][0]) <= 1e-9 && fabs(hv[h] - cur[m].uv[0][1]) <= 1e-9) dup = true;
      if (!dup) emit(cur[m]);
    }
    for (int m = 0; m < np && nh < kChainHist; ++m) {
      hu[nh] = cur[m].uv[0][0];
      hv[nh] = cur[m].uv[0][1];
      ++nh;
    }
  }
}

#ifndef SPOLY_HOST_BUILD
// Appends one path outside the warp-aggregated append (a candidate with more
// paths than a lane keeps).
SPOLY_D void append_path(const K1Params& P, spoly_path p) {
  const unsigned long long idx = atomicAdd(P.counters + C_ADMISSIBLE, 1ull);
  if (p.flags & SPOLY_FLAG_ILL_COND) atomicAdd(P.counters + C_FLAGGED, 1ull);
  if (P.chain_ids) p.chain = __ldg(P.chain_ids + p.chain);
  if (idx < (unsigned long long)P.path_cap) P.paths[idx] = p;
}
#endif

}  // namespace spoly
