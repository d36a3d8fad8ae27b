// Device polynomial machinery for the 1-bounce solve.
//
// Bivariate polynomials are stored densely in graded order: the coefficient
// of u^i v^j (i + j <= D) sits at bidx(D, i, j).  All loops over degrees are
// compile-time so that fully unrolled code keeps the coefficients in
// registers.
#pragma once
#include "common.cuh"

namespace spoly {

SPOLY_HD constexpr int bsize(int D) { return (D + 1) * (D + 2) / 2; }
SPOLY_HD constexpr int bidx(int D, int i, int j) { return i * (D + 1) - (i * (i - 1)) / 2 + j; }

template <typename T, int D>
struct BP {
  T c[bsize(D)];
};

template <int D>
using BPd = BP<double, D>;

// Linear vector polynomial c0 + u cu + v cv (positions and normals, Eq. eq_xi
// and eq_ni with u_i = (1-u-v, u, v)).
struct L3 {
  d3 c0, cu, cv;
};

SPOLY_D L3 l3_cross_c(const L3& a, d3 k) { return {cross(a.c0, k), cross(a.cu, k), cross(a.cv, k)}; }

// Dot product of two linear vector polynomials: a degree-2 scalar polynomial.
SPOLY_D BPd<2> l3_dot(const L3& a, const L3& b) {
  BPd<2> r;
  r.c[bidx(2, 0, 0)] = dot(a.c0, b.c0);
  r.c[bidx(2, 1, 0)] = dot(a.c0, b.cu) + dot(a.cu, b.c0);
  r.c[bidx(2, 0, 1)] = dot(a.c0, b.cv) + dot(a.cv, b.c0);
  r.c[bidx(2, 2, 0)] = dot(a.cu, b.cu);
  r.c[bidx(2, 1, 1)] = dot(a.cu, b.cv) + dot(a.cv, b.cu);
  r.c[bidx(2, 0, 2)] = dot(a.cv, b.cv);
  return r;
}

template <int D1, int D2>
SPOLY_D BPd<D1 + D2> bmul(const BPd<D1>& a, const BPd<D2>& b) {
  constexpr int D = D1 + D2;
  BPd<D> r;
#pragma unroll
  for (int k = 0; k < bsize(D); ++k) r.c[k] = 0.0;
#pragma unroll
  for (int i = 0; i <= D1; ++i)
#pragma unroll
    for (int j = 0; i + j <= D1; ++j)
#pragma unroll
      for (int k = 0; k <= D2; ++k)
#pragma unroll
        for (int l = 0; k + l <= D2; ++l)
          r.c[bidx(D, i + k, j + l)] = fma(a.c[bidx(D1, i, j)], b.c[bidx(D2, k, l)], r.c[bidx(D, i + k, j + l)]);
  return r;
}

// x * a + y * b for equal degrees.
template <int D>
SPOLY_D BPd<D> blin(double x, const BPd<D>& a, double y, const BPd<D>& b) {
  BPd<D> r;
#pragma unroll
  for (int k = 0; k < bsize(D); ++k) r.c[k] = x * a.c[k] + y * b.c[k];
  return r;
}

// -------------------------------------------------- projection switches
// Reading of "switch if the equation degenerates" (Sec. 3.3): with
// m = (x2 - x0) x n_c (n_c the centroid normal), the square form uses the
// first of (1,0,0), (0,0,1), (0,1,0) with |m^ . b| >= kSwitch; the product
// form uses t = n x e1 unless |m^ . e1^| < kSwitch and |m^ . e2^| > |m^ . e1^|.
// The choice is a threshold heuristic (it moves spurious roots, never true
// ones), so it runs in FP32 off the FP64 pipe.
SPOLY_D void plane_normal32(const TriD& tr, const QueryD& q, float& mx, float& my, float& mz) {
  const float wx = float(q.x2.x - q.x0.x), wy = float(q.x2.y - q.x0.y), wz = float(q.x2.z - q.x0.z);
  const float nx = float(tr.n0.x) + float(tr.n1.x) + float(tr.n2.x);
  const float ny = float(tr.n0.y) + float(tr.n1.y) + float(tr.n2.y);
  const float nz = float(tr.n0.z) + float(tr.n1.z) + float(tr.n2.z);
  mx = wy * nz - wz * ny;
  my = wz * nx - wx * nz;
  mz = wx * ny - wy * nx;
}

SPOLY_D d3 choose_b(const TriD& tr, const QueryD& q) {
  float mx, my, mz;
  plane_normal32(tr, q, mx, my, mz);
  const float m2 = mx * mx + my * my + mz * mz;
  if (!(m2 > 0.f)) return mk(1, 0, 0);
  const float t2 = float(kSwitch * kSwitch) * m2;  // |m^ . b| >= kSwitch  <=>  (m . b)^2 >= kSwitch^2 |m|^2
  if (mx * mx >= t2) return mk(1, 0, 0);
  if (mz * mz >= t2) return mk(0, 0, 1);
  if (my * my >= t2) return mk(0, 1, 0);
  return mk(1, 0, 0);
}

SPOLY_D int choose_edge(const TriD& tr, const QueryD& q) {
  float mx, my, mz;
  plane_normal32(tr, q, mx, my, mz);
  const float m2 = mx * mx + my * my + mz * mz;
  if (!(m2 > 0.f)) return 1;
  const float e1x = float(tr.p1.x - tr.p0.x), e1y = float(tr.p1.y - tr.p0.y), e1z = float(tr.p1.z - tr.p0.z);
  const float e2x = float(tr.p2.x - tr.p0.x), e2y = float(tr.p2.y - tr.p0.y), e2z = float(tr.p2.z - tr.p0.z);
  const float d1 = mx * e1x + my * e1y + mz * e1z, d2 = mx * e2x + my * e2y + mz * e2z;
  const float c1 = d1 * d1 / (e1x * e1x + e1y * e1y + e1z * e1z);  // (m . e^)^2, times |m|^2
  const float c2 = d2 * d2 / (e2x * e2x + e2y * e2y + e2z * e2z);
  return (c1 < float(kSwitch * kSwitch) * m2 && c2 > c1) ? 2 : 1;
}

// ------------------------------------------------------ coefficient phase
// Local frame with origin p0: x1 = u e1 + v e2, n = n0 + u (n1-n0) + v (n2-n0).
// The polynomials are translation invariant, so only differences appear.
struct Frame {
  L3 d0, d1, N;  // d0 = x1 - x0, d1 = x2 - x1, N = n(u, v)
  d3 w;          // x2 - x0
};

SPOLY_D Frame make_frame(const TriD& tr, const QueryD& q) {
  Frame f;
  const d3 e1 = tr.p1 - tr.p0, e2 = tr.p2 - tr.p0;
  const d3 x0 = q.x0 - tr.p0, x2 = q.x2 - tr.p0;
  f.d0 = {mk(-x0.x, -x0.y, -x0.z), e1, e2};
  f.d1 = {x2, mk(-e1.x, -e1.y, -e1.z), mk(-e2.x, -e2.y, -e2.z)};
  f.N = {tr.n0, tr.n1 - tr.n0, tr.n2 - tr.n0};
  f.w = q.x2 - q.x0;
  return f;
}

// a = ((P u - x0) x (x2 - x0)) . N u   (Eq. eq_coplane, Sec. 3.5 "R"/"T")
SPOLY_D BPd<2> build_a(const Frame& f) { return l3_dot(l3_cross_c(f.d0, f.w), f.N); }

// R: b = (d0.n)(d1.t) + (d1.n)(d0.t), t = n x e   (Eq. eq_pf_result)
SPOLY_D BPd<4> build_b_R(const Frame& f, const TriD& tr, int edge) {
  const d3 e = (edge == 2) ? (tr.p2 - tr.p0) : (tr.p1 - tr.p0);
  const L3 t = l3_cross_c(f.N, e);
  BPd<4> x = bmul<2, 2>(l3_dot(f.d0, f.N), l3_dot(f.d1, t));
  BPd<4> y = bmul<2, 2>(l3_dot(f.d1, f.N), l3_dot(f.d0, t));
  return blin<4>(1.0, x, 1.0, y);
}

// T: b = eta0^2 |d1|^2 ((d0 x n).b)^2 - eta1^2 |d0|^2 ((d1 x n).b)^2
// (Eq. eq_cpf_result), using (d x n).b = d . (n x b).
SPOLY_D BPd<6> build_b_T(const Frame& f, d3 bvec, double eta0, double eta1) {
  const L3 nb = l3_cross_c(f.N, bvec);
  const BPd<2> p0 = l3_dot(f.d0, nb);
  const BPd<2> p1 = l3_dot(f.d1, nb);
  const BPd<6> x = bmul<2, 4>(l3_dot(f.d1, f.d1), bmul<2, 2>(p0, p0));
  const BPd<6> y = bmul<2, 4>(l3_dot(f.d0, f.d0), bmul<2, 2>(p1, p1));
  return blin<6>(eta0 * eta0, x, -eta1 * eta1, y);
}

// Highest u-power with a non-negligible coefficient polynomial (Bezout size
// rule "n is the degree", Sec. 4.1; negligible = max-abs <= kTrim * max-abs).
template <int D>
SPOLY_D int deg_u(const BPd<D>& p) {
  long long m = 0;
#pragma unroll
  for (int k = 0; k < bsize(D); ++k) m = max(m, absbits(p.c[k]));
  if (m == 0) return -1;
  const long long thr = absbits(kTrim * __longlong_as_double(m));
  int d = -1;
#pragma unroll
  for (int i = 0; i <= D; ++i) {
    long long mi = 0;
#pragma unroll
    for (int j = 0; i + j <= D; ++j) mi = max(mi, absbits(p.c[bidx(D, i, j)]));
    if (mi > thr) d = i;
  }
  return d;
}

// Exact power-of-two change of variables u = 2^ks w, v = 2^kt z that
// balances b's coefficient magnitudes across u- and v-powers, followed by a
// power-of-two normalisation of a and b.  Roots are unchanged (z = v / 2^kt);
// the FP32 Laplace expansion then stays inside FP32's exponent range.  The
// magnitudes are compared by their binary exponents (integer arithmetic).
struct Scaling {
  int ks, kt;   // u = 2^ks w, v = 2^kt z
  double s, t;  // 2^ks, 2^kt
};

template <int D>
SPOLY_D Scaling choose_scaling(const BPd<D>& b, int nu) {
  long long mall = 0;
  long long mu[D + 1], mv[D + 1];
#pragma unroll
  for (int i = 0; i <= D; ++i) mu[i] = mv[i] = 0;
#pragma unroll
  for (int i = 0; i <= D; ++i)
#pragma unroll
    for (int j = 0; i + j <= D; ++j) {
      const long long a = absbits(b.c[bidx(D, i, j)]);
      mu[i] = max(mu[i], a);
      mv[j] = max(mv[j], a);
      mall = max(mall, a);
    }
  const long long thr = absbits(kTrim * __longlong_as_double(mall));
  int nv = -1;
#pragma unroll
  for (int j = 0; j <= D; ++j)
    if (mv[j] > thr) nv = j;
  long long m0u = mu[0], mnu = 0, m0v = mv[0], mnv = 0;
#pragma unroll
  for (int i = 0; i <= D; ++i) {
    if (i == nu) mnu = mu[i];
    if (i == nv) mnv = mv[i];
  }
  Scaling sc{0, 0, 1.0, 1.0};
  if (nu > 0 && m0u > 0 && mnu > 0) sc.ks = __float2int_rn(float(expo_bits(m0u) - expo_bits(mnu)) / float(nu));
  if (nv > 0 && m0v > 0 && mnv > 0) sc.kt = __float2int_rn(float(expo_bits(m0v) - expo_bits(mnv)) / float(nv));
  sc.ks = max(-30, min(60, sc.ks));
  sc.kt = max(-30, min(60, sc.kt));
  sc.s = scale2(1.0, sc.ks);
  sc.t = scale2(1.0, sc.kt);
  return sc;
}

template <int D>
SPOLY_D void apply_scaling(BPd<D>& p, const Scaling& sc) {
  int emax = -100000;
#pragma unroll
  for (int i = 0; i <= D; ++i)
#pragma unroll
    for (int j = 0; i + j <= D; ++j) {
      const long long a = absbits(p.c[bidx(D, i, j)]);
      if (a) emax = max(emax, expo_bits(a) + sc.ks * i + sc.kt * j);
    }
  if (emax == -100000) return;
  const int shift0 = -(emax + 1);  // largest coefficient lands in [0.5, 1)
#pragma unroll
  for (int i = 0; i <= D; ++i)
#pragma unroll
    for (int j = 0; i + j <= D; ++j) p.c[bidx(D, i, j)] = scale2(p.c[bidx(D, i, j)], shift0 + sc.ks * i + sc.kt * j);
}

// ------------------------------------------------------ elimination phase
// Bezout matrix entries (Eq. eq_bezout), u eliminated, z hidden:
//   E_ij(z) = sum_{k=0}^{min(i, n-1-j)} A_{i-k} B_{j+1+k} - B_{i-k} A_{j+1+k}
// where A_m(z) / B_m(z) are the u^m coefficients (zero beyond the trimmed
// degrees na / nb).  Entry (i, j) has z-degree <= DA + DB - 1 - i - j.
template <int N, int DA, int DB>
struct BezoutPoly {
  static constexpr int ED = DA + DB - 1;
  double e[N][N][ED + 1];
};

template <int DA, int DB>
SPOLY_D double coefA(const BPd<DA>& a, int na, int m, int j) {
  return (m <= DA && m <= na && j <= DA - m) ? a.c[bidx(DA, m, j)] : 0.0;
}

template <int N, int DA, int DB>
SPOLY_D void bezout_entry(const BPd<DA>& a, const BPd<DB>& b, int na, int nb, int i, int j,
                          double (&out)[DA + DB]) {
  constexpr int ED = DA + DB - 1;
#pragma unroll
  for (int c = 0; c <= ED; ++c) out[c] = 0.0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (k > i || k > N - 1 - j) continue;
    const int p = i - k, q = j + 1 + k;
    // + A_p B_q
    if (p <= DA && q <= DB) {
      const bool on = (p <= na) && (q <= nb);
#pragma unroll
      for (int x = 0; x <= DA - p; ++x)
#pragma unroll
        for (int y = 0; y <= DB - q; ++y)
          out[x + y] = fma(on ? a.c[bidx(DA, p, x)] : 0.0, b.c[bidx(DB, q, y)], out[x + y]);
    }
    // - B_p A_q
    if (q <= DA && p <= DB) {
      const bool on = (q <= na) && (p <= nb);
#pragma unroll
      for (int x = 0; x <= DB - p; ++x)
#pragma unroll
        for (int y = 0; y <= DA - q; ++y)
          out[x + y] = fma(on ? -b.c[bidx(DB, p, x)] : 0.0, a.c[bidx(DA, q, y)], out[x + y]);
    }
  }
}

// ------------------------------------------------------ univariate phase
// Degree bound of the minor of rows [row, N) and column set `mask` when entry
// (i, j) has degree <= ED - i - j.
SPOLY_HD constexpr int minor_deg(int N, int ED, int row, unsigned mask) {
  int d = 0;
  for (int i = row; i < N; ++i) d += ED - i;
  for (int j = 0; j < N; ++j)
    if (mask & (1u << j)) d -= j;
  return d;
}

SPOLY_HD constexpr int popc_c(unsigned x) { return x == 0 ? 0 : int(x & 1u) + popc_c(x >> 1); }

// The Bezout matrix is symmetric; entries (i <= j) are packed row by row,
// entry (i, j) holding ED - i - j + 1 coefficients (none if negative).
SPOLY_HD constexpr int sym_off(int N, int ED, int i, int j) {
  int o = 0;
  for (int a = 0; a < N; ++a)
    for (int b = a; b < N; ++b) {
      if (a == i && b == j) return o;
      if (ED - a - b >= 0) o += ED - a - b + 1;
    }
  return o;
}
SPOLY_HD constexpr int sym_size(int N, int ED) { return sym_off(N, ED, N, N); }

// All Bezout entries in FP64 from the scaled a and b, converted to T and
// packed as above (the order the generated Laplace expansions read).
template <typename T, int N, int DA, int DB>
SPOLY_D void bezout_sym(const BPd<DA>& a, const BPd<DB>& b, int na, int nb,
                        T (&E)[sym_size(N, DA + DB - 1)]) {
  constexpr int ED = DA + DB - 1;
  int o = 0;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      if (ED - i - j < 0) continue;
      double e[ED + 1];
      bezout_entry<N, DA, DB>(a, b, na, nb, i, j, e);
#pragma unroll
      for (int c = 0; c <= ED; ++c)
        if (c <= ED - i - j) E[o + c] = T(e[c]);
      o += ED - i - j + 1;
    }
}

// Binomial coefficients C(i, j), i, j <= 16.
static __constant__ double c_binom[17][17] = {
    {1},
    {1, 1},
    {1, 2, 1},
    {1, 3, 3, 1},
    {1, 4, 6, 4, 1},
    {1, 5, 10, 10, 5, 1},
    {1, 6, 15, 20, 15, 6, 1},
    {1, 7, 21, 35, 35, 21, 7, 1},
    {1, 8, 28, 56, 70, 56, 28, 8, 1},
    {1, 9, 36, 84, 126, 126, 84, 36, 9, 1},
    {1, 10, 45, 120, 210, 252, 210, 120, 45, 10, 1},
    {1, 11, 55, 165, 330, 462, 462, 330, 165, 55, 11, 1},
    {1, 12, 66, 220, 495, 792, 924, 792, 495, 220, 66, 12, 1},
    {1, 13, 78, 286, 715, 1287, 1716, 1716, 1287, 715, 286, 78, 13, 1},
    {1, 14, 91, 364, 1001, 2002, 3003, 3432, 3003, 2002, 1001, 364, 91, 14, 1},
    {1, 15, 105, 455, 1365, 3003, 5005, 6435, 6435, 5005, 3003, 1365, 455, 105, 15, 1},
    {1, 16, 120, 560, 1820, 4368, 8008, 11440, 12870, 11440, 8008, 4368, 1820, 560, 120, 16, 1}};

// Weights of the order-j derivative divided by j!: w_i = C(i, j) p_i for
// j <= i <= deg, so that p^(j)(x) / j! = sum_{i >= j} w_i x^(i - j).
template <typename T, int DM>
SPOLY_D void deriv_weights(const T (&p)[DM + 1], int deg, int j, T (&w)[DM + 1]) {
#pragma unroll
  for (int i = 0; i <= DM; ++i) w[i] = (i >= j && i <= deg) ? p[i] * T(c_binom[i][j]) : T(0);
}

// Horner evaluation of sum_{i >= j} w_i x^(i - j).
template <typename T, int DM>
SPOLY_D T horner_from(const T (&w)[DM + 1], int j, T x) {
  T s = T(0);
#pragma unroll
  for (int i = DM; i >= 0; --i)
    if (i >= j) s = fma(s, x, w[i]);
  return s;
}

// sum_{i >= j} w_i x^(i - j) and its derivative by one Horner pass.
template <typename T, int DM>
SPOLY_D void horner_from_d(const T (&w)[DM + 1], int j, T x, T* f, T* df) {
  T a = T(0), d = T(0);
#pragma unroll
  for (int i = DM; i >= 0; --i)
    if (i >= j) {
      d = fma(d, x, a);
      a = fma(a, x, w[i]);
    }
  *f = a;
  *df = d;
}

// The root of sum_{i >= j} w_i x^(i - j) on a monotone piece [a, b] whose end
// values differ in sign (fa: the value at a), to a bracket of width <= tol.
// FP32: bisection.  FP64: safeguarded Newton (Numerical Recipes' rtsafe
// rule): each evaluation moves the bracket end of its sign; the next point is
// the Newton step from it unless that leaves the bracket or the step is not
// shrinking fast enough (|2 f| > |previous step * f'|), then the midpoint.
// A Newton step below tol / 4 ends the search once a bracket of width tol
// around it shows a sign change.  Each FP64 instruction costs about 64 cycles
// of an SM sub-partition on this part, and the ~40 bisection steps from a
// monotone piece to 1e-12 become ~6 Newton steps.
template <typename T, int DM>
SPOLY_D void refine_root(const T (&w)[DM + 1], int j, T& a, T& b, T fa, T tol) {
  if constexpr (sizeof(T) == 4) {
    while (b - a > tol) {
      const T m = T(0.5) * (a + b);
      if (!(m > a && m < b)) return;
      const T fm = horner_from<T, DM>(w, j, m);
      if (fm == T(0)) {
        a = b = m;
        return;
      }
      if ((fm < T(0)) == (fa < T(0))) {
        a = m;
        fa = fm;
      } else {
        b = m;
      }
    }
  } else {
    // FP32 first: safeguarded Newton on the FP32-rounded coefficients to
    // FP32 accuracy, then at most three FP64 Newton steps from there and the
    // FP64 sign test of a bracket of width tol around the result.  Each FP32
    // instruction costs a fraction of an FP64 one on this part; any failure
    // falls through to the FP64 search below, from the original bracket.
    {
      float wf[DM + 1];
#pragma unroll
      for (int i = 0; i <= DM; ++i) wf[i] = (i >= j) ? float(w[i]) : 0.0f;
      float af = float(a), bf = float(b), faf = float(fa);
      float x = 0.5f * (af + bf);
      float dxo = bf - af;
      for (int it = 0; it < 40; ++it) {
        float f, df;
        horner_from_d<float, DM>(wf, j, x, &f, &df);
        if (f == 0.0f) break;
        if ((f < 0.0f) == (faf < 0.0f)) {
          af = x;
          faf = f;
        } else {
          bf = x;
        }
        const float xn = x - f / df;
        float xs;
        if (!(xn > af && xn < bf) || fabsf(2.0f * f) > fabsf(dxo * df)) {
          xs = 0.5f * (af + bf);
        } else {
          xs = xn;
        }
        dxo = fabsf(xs - x);
        if (!(xs > af && xs < bf) || xs == x) break;
        x = xs;
      }
      double xd = double(x);
      bool conv = false;
      for (int it = 0; it < 3 && xd > a && xd < b; ++it) {
        double f, df;
        horner_from_d<double, DM>(w, j, xd, &f, &df);
        if (f == 0.0) {
          a = b = xd;
          return;
        }
        const double st = f / df;
        xd -= st;
        if (fabs(st) <= 0.25 * tol) {
          conv = true;
          break;
        }
      }
      if (conv && xd > a && xd < b) {
        const double l = fmax(a, xd - 0.5 * tol), h = fmin(b, xd + 0.5 * tol);
        const double fl = horner_from<double, DM>(w, j, l), fh = horner_from<double, DM>(w, j, h);
        if (fl == 0.0 || fh == 0.0) {
          a = b = (fl == 0.0) ? l : h;
          return;
        }
        if ((fl < 0.0) == (fa < 0.0) && (fh < 0.0) != (fa < 0.0)) {
          a = l;
          b = h;
          return;
        }
      }
    }
    T x = T(0.5) * (a + b), dx = b - a, dxold = b - a;
    for (int it = 0; it < 96; ++it) {
      T f, df;
      horner_from_d<T, DM>(w, j, x, &f, &df);
      if (f == T(0)) {
        a = b = x;
        return;
      }
      if ((f < T(0)) == (fa < T(0))) {
        a = x;
        fa = f;
      } else {
        b = x;
      }
      if (!(b - a > tol)) return;
      const T xn = x - f / df;
      if (!(xn > a && xn < b) || fabs(T(2) * f) > fabs(dxold * df)) {
        dxold = dx;
        dx = T(0.5) * (b - a);
        x = a + dx;
        if (!(x > a && x < b)) return;  // no representable point inside
        continue;
      }
      dxold = dx;
      dx = x - xn;
      x = xn;
      if (fabs(dx) <= T(0.25) * tol) {
        const T l = fmax(a, x - T(0.5) * tol), h = fmin(b, x + T(0.5) * tol);
        const T fl = horner_from<T, DM>(w, j, l), fh = horner_from<T, DM>(w, j, h);
        if (fl == T(0) || fh == T(0)) {
          a = b = (fl == T(0)) ? l : h;
          return;
        }
        if ((fl < T(0)) == (fa < T(0)) && (fh < T(0)) != (fa < T(0))) {
          a = l;
          b = h;
          return;
        }
      }
    }
  }
}

// Real roots of p on [lo, hi] by recursive-derivative isolation (Sec. 4.2):
// the roots of the derivative of order j split [lo, hi] into monotone pieces
// of the derivative of order j-1; each piece with a sign change holds one
// root, refined to width `tol` (refine_root).  A root exactly at a piece end
// belongs to the piece on its left.  At order 0, critical points c with
// |p(c)| <= tang * rscale are reported as tangent roots.  Derivatives are
// taken as p^(j) / j! (binomial weights), which has the same roots.
// Returns the number of brackets written to (blo, bhi, bfl), or -3 when
// dip > 0 and a critical point c has |p(c)| <= dip * rscale (the caller
// treats the isolation as uncertified).

template <typename T, int DM>
SPOLY_D int isolate(const T (&p)[DM + 1], int deg, T lo, T hi, T tol, T tang, T rscale, T (&blo)[DM + 1],
                    T (&bhi)[DM + 1], uint32_t (&bfl)[DM + 1], T dip = T(0)) {
  T crit[DM + 1];
  int nc = 0;
  int nout = 0;
  T w[DM + 1];
  for (int j = deg - 1; j >= 0; --j) {
    deriv_weights<T, DM>(p, deg, j, w);
    T nlo[DM + 1], nhi[DM + 1];
    int nn = 0;
    T s = lo;
    T fs = horner_from<T, DM>(w, j, s);
    // Arrays hold DM + 1 roots; evaluation noise could in principle report
    // more sign changes than the degree allows, so every write is guarded.
    if (fs == T(0)) {
      nlo[nn] = s;
      nhi[nn] = s;
      ++nn;
    }
    for (int k = 0; k <= nc && nn <= DM; ++k) {
      const T e = (k < nc) ? crit[k] : hi;
      if (!(e > s)) continue;
      const T fe = horner_from<T, DM>(w, j, e);
      if (fe == T(0)) {
        nlo[nn] = e;
        nhi[nn] = e;
        ++nn;
      } else if (fs != T(0) && ((fs < T(0)) != (fe < T(0)))) {
        T a = s, b = e;
        refine_root<T, DM>(w, j, a, b, fs, tol);
        nlo[nn] = a;
        nhi[nn] = b;
        ++nn;
      }
      s = e;
      fs = fe;
    }
    if (j == 0) {
      for (int k = 0; k < nn && nout <= DM; ++k) {
        blo[nout] = nlo[k];
        bhi[nout] = nhi[k];
        bfl[nout] = 0u;
        ++nout;
      }
      const int nsimple = nout;
      for (int k = 0; k < nc; ++k) {
        const T c = crit[k];
        if (!(c > lo && c < hi)) continue;
        const T f = horner_from<T, DM>(w, 0, c);
        if (fabs(f) <= dip * rscale) return -3;
        if (fabs(f) <= tang * rscale) {
          bool dup = false;
          for (int m = 0; m < nsimple; ++m)
            if (c >= blo[m] - tol && c <= bhi[m] + tol) dup = true;
          if (!dup && nout <= DM) {
            blo[nout] = c;
            bhi[nout] = c;
            bfl[nout] = SPOLY_FLAG_TANGENT | SPOLY_FLAG_ILL_COND;
            ++nout;
          }
        }
      }
    } else {
      nc = nn < DM ? nn : DM;
      for (int k = 0; k < nc; ++k) crit[k] = T(0.5) * (nlo[k] + nhi[k]);
    }
  }
  return nout;
}

// --------------------------------------------------------- FP64 numeric det
// det of an n x n FP64 matrix by Gaussian elimination with partial pivoting.
template <int N>
SPOLY_D double det_ge(double (&m)[N][N], int n) {
  double det = 1.0;
#pragma unroll
  for (int c = 0; c < N; ++c) {
    if (c >= n) break;
    int piv = c;
    double best = fabs(m[c][c]);
#pragma unroll
    for (int r = c + 1; r < N; ++r)
      if (r < n && fabs(m[r][c]) > best) {
        best = fabs(m[r][c]);
        piv = r;
      }
    if (best == 0.0) return 0.0;
    if (piv != c) {
      det = -det;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        // swap rows c and piv (piv is dynamic: select-based swap)
#pragma unroll
        for (int r = 0; r < N; ++r)
          if (r == piv) {
            const double tmp = m[c][k];
            m[c][k] = m[r][k];
            m[r][k] = tmp;
          }
      }
    }
    det *= m[c][c];
    const double inv = 1.0 / m[c][c];
#pragma unroll
    for (int r = c + 1; r < N; ++r) {
      if (r >= n) continue;
      const double f = m[r][c] * inv;
#pragma unroll
      for (int k = c + 1; k < N; ++k) m[r][k] = fma(-f, m[c][k], m[r][k]);
    }
  }
  return det;
}

// Evaluation of a graded bivariate polynomial and its partial derivatives.
template <int D>
SPOLY_D void beval_grad(const BPd<D>& p, double u, double v, double* f, double* fu, double* fv) {
  double s = 0.0, su = 0.0, sv = 0.0;
#pragma unroll
  for (int i = D; i >= 0; --i) {
    double row = 0.0, drow = 0.0;
#pragma unroll
    for (int j = D - i; j >= 0; --j) {
      drow = fma(drow, v, row);
      row = fma(row, v, p.c[bidx(D, i, j)]);
    }
    su = fma(su, u, s);
    s = fma(s, u, row);
    sv = fma(sv, u, drow);
  }
  *f = s;
  *fu = su;
  *fv = sv;
}

}  // namespace spoly
