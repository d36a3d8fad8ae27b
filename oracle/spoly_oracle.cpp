// FP64 CPU oracle for the specular-polynomial solve (TEST INFRASTRUCTURE).
//
// This file is test infrastructure, not product code.  Only the tests, the
// package's smoke() check and bench.py's CPU baseline / reference legs load
// it.  It shares no code, header, table or generator with the CUDA path.
//
// It follows the paper's pipeline step by step, in plain FP64, with generic
// dense polynomial arithmetic and no fusion or reordering:
//   1. coefficient phase (Sec. 4.3): build the bivariate specular polynomials
//      a(u,v), b(u,v) of one candidate from its vertex positions P and
//      normals N (Eq. eq_xi, eq_ni); R uses the endpoint-difference
//      coplanarity (Eq. eq_coplane) and the product form (Eq. eq_pf_result),
//      T uses the coplanarity and the square form (Eq. eq_cpf_result);
//      Sec. 3.5 paragraphs "R" and "T".
//   2. elimination phase (Sec. 4.1): the Bezout matrix of a and b in u with v
//      hidden, entries by the explicit sum of Eq. eq_bezout.
//   3. univariate phase (Sec. 4.2): r(v) = det R(v) by cofactor (Laplace)
//      expansion with polynomial entries, then recursive-derivative root
//      isolation with bisection (roots of r^(j) split [lo,hi] into monotone
//      pieces of r^(j-1)).
//   4. path phase (Sec. 4.3): put v back into a(u,v), solve for u, build the
//      path and check the specular constraint h x n = 0 (Eq. eq_ch) in path
//      space, sidedness and the in-triangle test.
// Readings of points the paper leaves open are listed with each constant.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------- constants
// Search domain for v (and u): [-kDelta, 1 + kDelta]; membership is decided
// by the in-triangle test afterwards.
constexpr double kDelta = 1e-6;
// A u-power of a bivariate polynomial counts for the Bezout size n only if
// its coefficient polynomial has max-abs > kTrim * (max-abs of the whole
// polynomial) (Eq. eq_bezout: "n is the degree").
constexpr double kTrim = 1e-13;
// Bisection stops at this interval length (the paper stops at 1e-9, Sec. 4.2;
// the oracle continues to the FP64 limit).
constexpr double kRootTol = 1e-14;
// A critical point c of r with |r(c)| <= kTangent * sum|r_i| * max(1,|c|)^d is
// a tangent (even-multiplicity) root and is flagged ill-conditioned.
constexpr double kTangent = 1e-12;
// A simple root is ill-conditioned if |r'(v*)| / sum|r_i| < kIllCond.
constexpr double kIllCond = 1e-8;
// Admissible if the path-space residual sin(angle(h, n)) < kResidual.
constexpr double kResidual = 1e-9;
// EDGE flag if min(u, v, 1-u-v) is within kEdge of 0.
constexpr double kEdge = 1e-7;
// Duplicate paths of one candidate within this max-norm distance are merged.
constexpr double kDedupe = 1e-9;

enum : uint32_t {
  F_ILL_COND = 1u,
  F_EDGE = 2u,
  F_BACKFACE = 4u,
  F_NEWTON_REFINED = 8u,
  F_SQRT_SPLIT = 16u,
  F_TANGENT = 32u,
};

// --------------------------------------------------------- univariate (v)
using UPoly = std::vector<double>;  // coefficient of v^i at index i

void utrim(UPoly& p) {
  while (!p.empty() && p.back() == 0.0) p.pop_back();
}

UPoly uadd(const UPoly& a, const UPoly& b) {
  UPoly r(std::max(a.size(), b.size()), 0.0);
  for (size_t i = 0; i < a.size(); ++i) r[i] += a[i];
  for (size_t i = 0; i < b.size(); ++i) r[i] += b[i];
  return r;
}

UPoly usub(const UPoly& a, const UPoly& b) {
  UPoly r(std::max(a.size(), b.size()), 0.0);
  for (size_t i = 0; i < a.size(); ++i) r[i] += a[i];
  for (size_t i = 0; i < b.size(); ++i) r[i] -= b[i];
  return r;
}

UPoly umul(const UPoly& a, const UPoly& b) {
  if (a.empty() || b.empty()) return {};
  UPoly r(a.size() + b.size() - 1, 0.0);
  for (size_t i = 0; i < a.size(); ++i)
    for (size_t j = 0; j < b.size(); ++j) r[i + j] += a[i] * b[j];
  return r;
}

double ueval(const UPoly& p, double x) {
  double s = 0.0;
  for (size_t i = p.size(); i-- > 0;) s = s * x + p[i];
  return s;
}

UPoly uderiv(const UPoly& p) {
  if (p.size() <= 1) return {};
  UPoly d(p.size() - 1);
  for (size_t i = 1; i < p.size(); ++i) d[i - 1] = p[i] * double(i);
  return d;
}

double uabssum(const UPoly& p) {
  double s = 0.0;
  for (double c : p) s += std::fabs(c);
  return s;
}

double umaxabs(const UPoly& p) {
  double s = 0.0;
  for (double c : p) s = std::max(s, std::fabs(c));
  return s;
}

// ------------------------------------------------------- bivariate (u, v)
// Dense sum_{i,j} c[i][j] u^i v^j with i + j <= deg, stored on a square grid.
struct BPoly {
  int deg = 0;
  std::vector<double> c;  // (deg+1)^2 entries, c[i*(deg+1)+j]
  BPoly() : deg(0), c(1, 0.0) {}
  explicit BPoly(int d) : deg(d), c(size_t(d + 1) * (d + 1), 0.0) {}
  double& at(int i, int j) { return c[size_t(i) * (deg + 1) + j]; }
  double at(int i, int j) const { return c[size_t(i) * (deg + 1) + j]; }
};

BPoly bconst(double k) {
  BPoly p(0);
  p.at(0, 0) = k;
  return p;
}

// k0 + ku*u + kv*v
BPoly blinear(double k0, double ku, double kv) {
  BPoly p(1);
  p.at(0, 0) = k0;
  p.at(1, 0) = ku;
  p.at(0, 1) = kv;
  return p;
}

BPoly badd(const BPoly& a, const BPoly& b, double sb = 1.0) {
  BPoly r(std::max(a.deg, b.deg));
  for (int i = 0; i <= a.deg; ++i)
    for (int j = 0; i + j <= a.deg; ++j) r.at(i, j) += a.at(i, j);
  for (int i = 0; i <= b.deg; ++i)
    for (int j = 0; i + j <= b.deg; ++j) r.at(i, j) += sb * b.at(i, j);
  return r;
}

BPoly bsub(const BPoly& a, const BPoly& b) { return badd(a, b, -1.0); }

BPoly bscale(const BPoly& a, double k) {
  BPoly r = a;
  for (double& x : r.c) x *= k;
  return r;
}

BPoly bmul(const BPoly& a, const BPoly& b) {
  BPoly r(a.deg + b.deg);
  for (int i = 0; i <= a.deg; ++i)
    for (int j = 0; i + j <= a.deg; ++j) {
      const double x = a.at(i, j);
      if (x == 0.0) continue;
      for (int k = 0; k <= b.deg; ++k)
        for (int l = 0; k + l <= b.deg; ++l) r.at(i + k, j + l) += x * b.at(k, l);
    }
  return r;
}

double bmaxabs(const BPoly& p) {
  double s = 0.0;
  for (double x : p.c) s = std::max(s, std::fabs(x));
  return s;
}

double beval(const BPoly& p, double u, double v) {
  double s = 0.0;
  for (int i = p.deg; i >= 0; --i) {
    double row = 0.0;
    for (int j = p.deg - i; j >= 0; --j) row = row * v + p.at(i, j);
    s = s * u + row;
  }
  return s;
}

// Partial derivatives of a bivariate polynomial.
BPoly bderiv_u(const BPoly& p) {
  BPoly r(std::max(0, p.deg - 1));
  for (int i = 1; i <= p.deg; ++i)
    for (int j = 0; i + j <= p.deg; ++j) r.at(i - 1, j) = double(i) * p.at(i, j);
  return r;
}

BPoly bderiv_v(const BPoly& p) {
  BPoly r(std::max(0, p.deg - 1));
  for (int i = 0; i <= p.deg; ++i)
    for (int j = 1; i + j <= p.deg; ++j) r.at(i, j - 1) = double(j) * p.at(i, j);
  return r;
}

// Reading: the recovered (u, v*) is refined by at most kNewtonIters Newton
// steps on the bivariate system a = b = 0 itself (Sec. 3.5), accepted only if
// the total move stays within kNewtonMove.  Where a(u, v) = 0 is nearly
// parallel to the u axis, u = u(v*) amplifies the error of the hidden
// variable; the refinement removes it so that the path-space residual test
// measures the method's root rather than that amplification.
constexpr int kNewtonIters = 3;
constexpr double kNewtonMove = 1e-5;

void newton_ab(const BPoly& a, const BPoly& b, double* u, double* v) {
  const BPoly au = bderiv_u(a), av = bderiv_v(a), bu = bderiv_u(b), bv = bderiv_v(b);
  double uu = *u, vv = *v;
  for (int it = 0; it < kNewtonIters; ++it) {
    const double fa = beval(a, uu, vv), fb = beval(b, uu, vv);
    const double a1 = beval(au, uu, vv), a2 = beval(av, uu, vv);
    const double b1 = beval(bu, uu, vv), b2 = beval(bv, uu, vv);
    const double det = a1 * b2 - a2 * b1;
    if (!(std::fabs(det) > 0.0)) break;
    const double du = (fa * b2 - fb * a2) / det;
    const double dv = (a1 * fb - b1 * fa) / det;
    if (!std::isfinite(du) || !std::isfinite(dv)) break;
    uu -= du;
    vv -= dv;
  }
  if (std::fabs(uu - *u) <= kNewtonMove && std::fabs(vv - *v) <= kNewtonMove) {
    *u = uu;
    *v = vv;
  }
}

// Coefficient of u^i as a polynomial in v (a_i(v) of Eq. eq_bezout's context).
UPoly bcoef_u(const BPoly& p, int i) {
  UPoly r;
  if (i > p.deg) return r;
  r.assign(size_t(p.deg - i + 1), 0.0);
  for (int j = 0; i + j <= p.deg; ++j) r[j] = p.at(i, j);
  return r;
}

// Highest power of u whose coefficient polynomial is not negligible.
int bdeg_u(const BPoly& p) {
  const double m = bmaxabs(p);
  if (m == 0.0) return -1;
  for (int i = p.deg; i >= 0; --i) {
    double mi = 0.0;
    for (int j = 0; i + j <= p.deg; ++j) mi = std::max(mi, std::fabs(p.at(i, j)));
    if (mi > kTrim * m) return i;
  }
  return -1;
}

// Exact total degree (highest i+j with a nonzero coefficient).
int btotal_deg(const BPoly& p, double rel = 0.0) {
  const double m = bmaxabs(p);
  for (int s = p.deg; s >= 0; --s)
    for (int i = 0; i <= s; ++i)
      if (std::fabs(p.at(i, s - i)) > rel * m && p.at(i, s - i) != 0.0) return s;
  return -1;
}

struct V3 {
  BPoly x, y, z;
};

V3 vconst(const double* k) { return {bconst(k[0]), bconst(k[1]), bconst(k[2])}; }

V3 vsub(const V3& a, const V3& b) { return {bsub(a.x, b.x), bsub(a.y, b.y), bsub(a.z, b.z)}; }

BPoly vdot(const V3& a, const V3& b) {
  return badd(badd(bmul(a.x, b.x), bmul(a.y, b.y)), bmul(a.z, b.z));
}

V3 vcross(const V3& a, const V3& b) {
  return {bsub(bmul(a.y, b.z), bmul(a.z, b.y)), bsub(bmul(a.z, b.x), bmul(a.x, b.z)),
          bsub(bmul(a.x, b.y), bmul(a.y, b.x))};
}

// Barycentric interpolation M u with u = (1-u-v, u, v): column m0 + u (m1 - m0)
// + v (m2 - m0), which is Eq. eq_xi for positions and Eq. eq_ni for normals.
V3 vbary(const double* m0, const double* m1, const double* m2) {
  V3 r;
  r.x = blinear(m0[0], m1[0] - m0[0], m2[0] - m0[0]);
  r.y = blinear(m0[1], m1[1] - m0[1], m2[1] - m0[1]);
  r.z = blinear(m0[2], m1[2] - m0[2], m2[2] - m0[2]);
  return r;
}

// ------------------------------------------------------------- 3-vectors
struct D3 {
  double x, y, z;
};
D3 d3(const double* p) { return {p[0], p[1], p[2]}; }
D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
D3 operator*(double k, D3 a) { return {k * a.x, k * a.y, k * a.z}; }
double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
D3 cross(D3 a, D3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double norm(D3 a) { return std::sqrt(dot(a, a)); }

// One triangle: positions p[3] and vertex normals n[3].
struct Tri {
  double p[3][3];
  double n[3][3];
};

Tri load_tri(const double* soa, int64_t n_tris, int64_t t) {
  Tri tr;
  for (int v = 0; v < 3; ++v)
    for (int c = 0; c < 3; ++c) {
      tr.p[v][c] = soa[int64_t(3 * v + c) * n_tris + t];
      tr.n[v][c] = soa[int64_t(9 + 3 * v + c) * n_tris + t];
    }
  return tr;
}

// ------------------------------------------------------ coefficient phase
// Reading of "switch if the equation degenerates" (Sec. 3.3, square form and
// product form): the projection basis b (square form) and the tangent edge
// (product form) are chosen from the geometry.  With m = (x2 - x0) x n_c
// (n_c = unnormalised centroid normal) the normal of the plane of incidence,
// the square form's spurious factor is (m . b) and the product form's is
// (m . e).  b: first of (1,0,0) [paper default], (0,0,1) [paper switch],
// (0,1,0) [extension] with |m^ . b| >= kSwitch.  t = n x e1 [paper default]
// unless |m^ . e1^| < kSwitch and |m^ . e2^| > |m^ . e1^|, then n x e2.
constexpr double kSwitch = 0.25;

void choose_projection(const Tri& tr, D3 x0, D3 x2, int type, D3* bvec, int* edge) {
  D3 nc = (1.0 / 3.0) * (d3(tr.n[0]) + d3(tr.n[1]) + d3(tr.n[2]));
  D3 m = cross(x2 - x0, nc);
  const double mn = norm(m);
  *bvec = {1.0, 0.0, 0.0};
  *edge = 1;
  if (!(mn > 0.0)) return;
  m = (1.0 / mn) * m;
  if (type == 1) {
    const D3 cand[3] = {{1, 0, 0}, {0, 0, 1}, {0, 1, 0}};
    for (int i = 0; i < 3; ++i)
      if (std::fabs(dot(m, cand[i])) >= kSwitch) {
        *bvec = cand[i];
        return;
      }
  } else {
    D3 e1 = d3(tr.p[1]) - d3(tr.p[0]);
    D3 e2 = d3(tr.p[2]) - d3(tr.p[0]);
    const double c1 = std::fabs(dot(m, e1)) / norm(e1);
    const double c2 = std::fabs(dot(m, e2)) / norm(e2);
    if (c1 < kSwitch && c2 > c1) *edge = 2;
  }
}

// Builds a(u,v) and b(u,v) for a 1-bounce candidate (Sec. 3.5, "R" and "T").
//   a = ((P u - x0) x (x2 - x0)) . N u                                [eq_coplane]
//   R: b = ((Pu - x0).Nu)((x2 - Pu).t) + ((x2 - Pu).Nu)((Pu - x0).t), t = Nu x e
//                                                                      [eq_pf_result]
//   T: b = eta0^2 |x2 - Pu|^2 (((Pu - x0) x Nu).b)^2
//        - eta1^2 |Pu - x0|^2 (((x2 - Pu) x Nu).b)^2                   [eq_cpf_result]
void build_k1(const Tri& tr, D3 x0v, D3 x2v, int type, double eta0, double eta1, BPoly* a, BPoly* b) {
  const double x0[3] = {x0v.x, x0v.y, x0v.z};
  const double x2[3] = {x2v.x, x2v.y, x2v.z};
  V3 X = vbary(tr.p[0], tr.p[1], tr.p[2]);  // x1 = P u
  V3 N = vbary(tr.n[0], tr.n[1], tr.n[2]);  // n1 = N u (unnormalised)
  V3 X0 = vconst(x0), X2 = vconst(x2);
  V3 d0 = vsub(X, X0);   // d_0 = x1 - x0
  V3 d1 = vsub(X2, X);   // d_1 = x2 - x1
  V3 w = vsub(X2, X0);   // x2 - x0
  *a = vdot(vcross(d0, w), N);
  D3 bvec;
  int edge;
  choose_projection(tr, x0v, x2v, type, &bvec, &edge);
  if (type == 0) {
    const int e = edge;  // e_{1,e} = p_e - p_0
    const double ev[3] = {tr.p[e][0] - tr.p[0][0], tr.p[e][1] - tr.p[0][1], tr.p[e][2] - tr.p[0][2]};
    V3 t = vcross(N, vconst(ev));
    *b = badd(bmul(vdot(d0, N), vdot(d1, t)), bmul(vdot(d1, N), vdot(d0, t)));
  } else {
    const double bv[3] = {bvec.x, bvec.y, bvec.z};
    V3 B = vconst(bv);
    BPoly p0 = vdot(vcross(d0, N), B);
    BPoly p1 = vdot(vcross(d1, N), B);
    BPoly lhs = bscale(bmul(vdot(d1, d1), bmul(p0, p0)), eta0 * eta0);
    BPoly rhs = bscale(bmul(vdot(d0, d0), bmul(p1, p1)), eta1 * eta1);
    *b = bsub(lhs, rhs);
  }
}

// ------------------------------------------------------ elimination phase
// Bezout matrix of a and b with respect to u, v hidden (Eq. eq_bezout):
//   R_ij(v) = sum_{k=0}^{min(i, n-1-j)} a_{i-k} b_{j+1+k} - b_{i-k} a_{j+1+k}
// with n = max(deg_u a, deg_u b) and a_m = b_m = 0 beyond their degrees.
std::vector<UPoly> bezout_matrix(const std::vector<UPoly>& ac, const std::vector<UPoly>& bc, int n) {
  auto A = [&](int m) -> const UPoly& {
    static const UPoly zero;
    return (m >= 0 && m < int(ac.size())) ? ac[m] : zero;
  };
  auto B = [&](int m) -> const UPoly& {
    static const UPoly zero;
    return (m >= 0 && m < int(bc.size())) ? bc[m] : zero;
  };
  std::vector<UPoly> R(size_t(n) * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      UPoly s;
      for (int k = 0; k <= std::min(i, n - 1 - j); ++k) {
        s = uadd(s, umul(A(i - k), B(j + 1 + k)));
        s = usub(s, umul(B(i - k), A(j + 1 + k)));
      }
      R[size_t(i) * n + j] = s;
    }
  return R;
}

// det of the submatrix of rows [row, n) and the given columns, by cofactor
// expansion along its first row (Sec. 4.2, "Laplacian expansion").
UPoly laplace_det(const std::vector<UPoly>& R, int n, int row, std::vector<int>& cols) {
  if (row == n - 1) return R[size_t(row) * n + cols[0]];
  UPoly det;
  const int m = int(cols.size());
  for (int jj = 0; jj < m; ++jj) {
    const int j = cols[jj];
    const UPoly& e = R[size_t(row) * n + j];
    if (e.empty()) continue;
    std::vector<int> sub;
    sub.reserve(m - 1);
    for (int kk = 0; kk < m; ++kk)
      if (kk != jj) sub.push_back(cols[kk]);
    UPoly minor = laplace_det(R, n, row + 1, sub);
    UPoly term = umul(e, minor);
    det = (jj % 2 == 0) ? uadd(det, term) : usub(det, term);
  }
  return det;
}

// ------------------------------------------------------ univariate phase
struct Root {
  double x;
  uint32_t flags;
};

// Bisection on [s, e] where p(s) and p(e) have opposite signs.
double bisect(const UPoly& p, double s, double e, double fs) {
  while (e - s > kRootTol) {
    const double m = 0.5 * (s + e);
    if (m <= s || m >= e) break;
    const double fm = ueval(p, m);
    if (fm == 0.0) return m;
    if ((fm < 0.0) == (fs < 0.0)) {
      s = m;
      fs = fm;
    } else {
      e = m;
    }
  }
  return 0.5 * (s + e);
}

// Real roots of p on [lo, hi] by recursive-derivative isolation (Sec. 4.2):
// the roots of p' split [lo, hi] into monotone pieces of p; each piece with a
// sign change holds one root, found by bisection.  A root exactly at a piece
// end belongs to the piece on its left.  With top_level, critical points where
// |p| is negligible are reported as tangent roots (no sign change).
std::vector<Root> isolate(UPoly p, double lo, double hi, bool top_level) {
  utrim(p);
  std::vector<Root> out;
  const int d = int(p.size()) - 1;
  if (d <= 0) return out;
  if (d == 1) {
    const double x = -p[0] / p[1];
    if (x >= lo && x <= hi) out.push_back({x, 0u});
    return out;
  }
  std::vector<Root> crit = isolate(uderiv(p), lo, hi, false);
  std::vector<double> pts;
  pts.push_back(lo);
  for (const Root& c : crit)
    if (c.x > lo && c.x < hi) pts.push_back(c.x);
  pts.push_back(hi);
  std::sort(pts.begin(), pts.end());
  double fs = ueval(p, pts[0]);
  if (fs == 0.0) out.push_back({pts[0], 0u});
  for (size_t i = 1; i < pts.size(); ++i) {
    const double s = pts[i - 1], e = pts[i];
    const double fe = ueval(p, e);
    if (fe == 0.0) {
      out.push_back({e, 0u});
    } else if (fs != 0.0 && ((fs < 0.0) != (fe < 0.0))) {
      out.push_back({bisect(p, s, e, fs), 0u});
    }
    fs = fe;
  }
  if (top_level) {
    const double sabs = uabssum(p);
    for (size_t i = 1; i + 1 < pts.size(); ++i) {
      const double c = pts[i];
      const double f = ueval(p, c);
      const double scale = sabs * std::pow(std::max(1.0, std::fabs(c)), d);
      if (std::fabs(f) <= kTangent * scale) out.push_back({c, F_TANGENT | F_ILL_COND});
    }
    std::sort(out.begin(), out.end(), [](const Root& x, const Root& y) { return x.x < y.x; });
    std::vector<Root> dedup;
    for (const Root& r : out) {
      if (!dedup.empty() && std::fabs(r.x - dedup.back().x) <= 1e-12) {
        dedup.back().flags |= r.flags;
        continue;
      }
      dedup.push_back(r);
    }
    out.swap(dedup);
  }
  return out;
}

// -------------------------------------------------------------- path phase
struct Path {
  int64_t chain;
  int32_t query, tri0, tri1;
  double uv[4];
  double x[6];
  double residual;
  uint32_t flags;
};

// Path-space check of one vertex (Eq. eq_ch): h = eta1 d1^ - eta0 d0^ must be
// parallel to n.  residual = |h x n| / (|h| |n|), the sine of their angle.
// Sidedness (reading of "check the specular constraints in path space",
// Sec. 4.3): reflection keeps x0 and x2 on the same side of the tangent plane
// (d0.n and d1.n of opposite signs) and needs |h| > 1e-9; refraction crosses
// it (d0.n and d1.n of equal signs).
bool vertex_check(D3 xprev, D3 x, D3 xnext, D3 n, int type, double eta_in, double eta_out,
                  double* residual, uint32_t* flags) {
  D3 d0 = x - xprev, d1 = xnext - x;
  const double l0 = norm(d0), l1 = norm(d1), ln = norm(n);
  if (!(l0 > 0.0) || !(l1 > 0.0) || !(ln > 0.0)) return false;
  D3 h = (type == 0) ? ((1.0 / l1) * d1 - (1.0 / l0) * d0) : ((eta_out / l1) * d1 - (eta_in / l0) * d0);
  const double lh = norm(h);
  if (!(lh > 1e-9)) return false;
  *residual = norm(cross(h, n)) / (lh * ln);
  const double s0 = dot(d0, n), s1 = dot(d1, n);
  if (dot(xprev - x, n) < 0.0) *flags |= F_BACKFACE;
  if (type == 0) return (s0 < 0.0) != (s1 < 0.0) && s0 != 0.0 && s1 != 0.0;
  return (s0 < 0.0) == (s1 < 0.0) && s0 != 0.0 && s1 != 0.0;
}

struct Counters {
  int64_t candidates = 0, degenerate = 0, v_roots = 0, u_roots = 0, admissible = 0, flagged = 0;
};

// Full 1-bounce solve of one candidate.  Appends admissible paths.
void solve_k1(const Tri& tr, D3 x0, D3 x2, int type, double eta0, double eta1, int64_t chain, int32_t q,
              int32_t t, std::vector<Path>& out, Counters& cnt) {
  cnt.candidates++;
  BPoly a, b;
  build_k1(tr, x0, x2, type, eta0, eta1, &a, &b);
  const int da = bdeg_u(a), db = bdeg_u(b);
  const int n = std::max(da, db);
  if (da < 0 || db < 0 || n < 1) {
    cnt.degenerate++;
    return;
  }
  std::vector<UPoly> ac, bc;
  for (int i = 0; i <= da; ++i) ac.push_back(bcoef_u(a, i));
  for (int i = 0; i <= db; ++i) bc.push_back(bcoef_u(b, i));
  std::vector<UPoly> R = bezout_matrix(ac, bc, n);
  std::vector<int> cols(n);
  for (int j = 0; j < n; ++j) cols[j] = j;
  UPoly r = laplace_det(R, n, 0, cols);
  // Drop negligible leading terms of r (they only move roots at infinity).
  const double rmax = umaxabs(r);
  while (!r.empty() && std::fabs(r.back()) <= kTrim * rmax) r.pop_back();
  if (r.empty()) {
    cnt.degenerate++;
    return;
  }
  std::vector<Root> vroots = isolate(r, -kDelta, 1.0 + kDelta, true);
  const UPoly dr = uderiv(r);
  const double rabs = uabssum(r);
  std::vector<Path> local;
  for (const Root& vr : vroots) {
    cnt.v_roots++;
    const double v0 = vr.x;
    const double v = v0;
    uint32_t vflags = vr.flags;
    if (std::fabs(ueval(dr, v)) < kIllCond * rabs) vflags |= F_ILL_COND;
    // Path phase: a(u, v*) = 0 for u (fall back to b if a(., v*) vanishes).
    UPoly au(size_t(da) + 1);
    double amag = 0.0;
    for (int i = 0; i <= da; ++i) {
      au[i] = ueval(ac[i], v);
      amag = std::max(amag, umaxabs(ac[i]));
    }
    if (umaxabs(au) <= kTrim * amag) {
      au.assign(size_t(db) + 1, 0.0);
      for (int i = 0; i <= db; ++i) au[i] = ueval(bc[i], v);
    }
    std::vector<Root> uroots = isolate(au, -kDelta, 1.0 - v + kDelta, true);
    for (const Root& ur : uroots) {
      cnt.u_roots++;
      double u = ur.x, v = v0;
      newton_ab(a, b, &u, &v);
      uint32_t flags = vflags | ur.flags;
      D3 p0 = d3(tr.p[0]), p1 = d3(tr.p[1]), p2 = d3(tr.p[2]);
      D3 n0 = d3(tr.n[0]), n1 = d3(tr.n[1]), n2 = d3(tr.n[2]);
      D3 x1 = p0 + u * (p1 - p0) + v * (p2 - p0);
      D3 nn = n0 + u * (n1 - n0) + v * (n2 - n0);
      double res = 1.0;
      if (!vertex_check(x0, x1, x2, nn, type, eta0, eta1, &res, &flags)) continue;
      if (!(res < kResidual)) continue;
      const double w = std::min(std::min(u, v), 1.0 - u - v);
      if (w < 0.0) continue;
      if (w < kEdge) flags |= F_EDGE;
      bool dup = false;
      for (Path& pp : local)
        if (std::fabs(pp.uv[0] - u) <= kDedupe && std::fabs(pp.uv[1] - v) <= kDedupe) {
          pp.flags |= flags;
          dup = true;
        }
      if (dup) continue;
      Path pth{};
      pth.chain = chain;
      pth.query = q;
      pth.tri0 = t;
      pth.tri1 = -1;
      pth.uv[0] = u;
      pth.uv[1] = v;
      pth.x[0] = x1.x;
      pth.x[1] = x1.y;
      pth.x[2] = x1.z;
      pth.residual = res;
      pth.flags = flags;
      local.push_back(pth);
    }
  }
  for (const Path& pth : local) {
    cnt.admissible++;
    if (pth.flags & F_ILL_COND) cnt.flagged++;
    out.push_back(pth);
  }
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

struct oracle_path {
  int64_t chain;
  int32_t query, tri0, tri1, pad;
  double uv[4];
  double x[6];
  double residual;
  uint32_t flags, pad2;
};

struct oracle_counters {
  int64_t candidates, degenerate, v_roots, u_roots, admissible, flagged;
};

// Solves every chain (query, tri0, tri1) of a 1-bounce workload.
//   tri      [18][n_tris] FP64 SoA (p0,p1,p2,n0,n1,n2 rows)
//   x_first, x_last [Q][3]; eta [Q][3]; types [Q][2] (0 = R, 1 = T); k [Q]
//   chains [n_chains][3] int32 (query, tri0, tri1)
// Writes at most `capacity` paths in chain order; *n_out receives the total.
// Returns 0, or -1 on a capacity overflow, -2 for an unsupported bounce count.
int oracle_solve(const double* tri, int64_t n_tris, const double* x_first, const double* x_last,
                 const double* eta, const int32_t* types, const int32_t* kb, const int32_t* chains,
                 int64_t n_chains, oracle_path* out, int64_t capacity, int64_t* n_out,
                 oracle_counters* counters, int n_threads) {
  if (n_threads <= 0) n_threads = int(std::max(1u, std::thread::hardware_concurrency()));
  for (int64_t c = 0; c < n_chains; ++c)
    if (kb[chains[3 * c]] != 1) return -2;
  std::atomic<int64_t> next{0};
  const int64_t block = 256;
  std::vector<std::vector<Path>> per_thread(n_threads);
  std::vector<Counters> cnts(n_threads);
  auto work = [&](int tid) {
    for (;;) {
      const int64_t s = next.fetch_add(block);
      if (s >= n_chains) break;
      const int64_t e = std::min(n_chains, s + block);
      for (int64_t c = s; c < e; ++c) {
        const int32_t q = chains[3 * c], t = chains[3 * c + 1];
        Tri tr = load_tri(tri, n_tris, t);
        solve_k1(tr, d3(x_first + 3 * q), d3(x_last + 3 * q), types[2 * q], eta[3 * q], eta[3 * q + 1], c, q, t,
                 per_thread[tid], cnts[tid]);
      }
    }
  };
  std::vector<std::thread> th;
  for (int i = 1; i < n_threads; ++i) th.emplace_back(work, i);
  work(0);
  for (auto& x : th) x.join();
  std::vector<Path> all;
  Counters tot;
  for (int i = 0; i < n_threads; ++i) {
    all.insert(all.end(), per_thread[i].begin(), per_thread[i].end());
    tot.candidates += cnts[i].candidates;
    tot.degenerate += cnts[i].degenerate;
    tot.v_roots += cnts[i].v_roots;
    tot.u_roots += cnts[i].u_roots;
    tot.admissible += cnts[i].admissible;
    tot.flagged += cnts[i].flagged;
  }
  std::stable_sort(all.begin(), all.end(), [](const Path& x, const Path& y) {
    if (x.chain != y.chain) return x.chain < y.chain;
    return x.uv[1] < y.uv[1] || (x.uv[1] == y.uv[1] && x.uv[0] < y.uv[0]);
  });
  *n_out = int64_t(all.size());
  if (counters) {
    counters->candidates = tot.candidates;
    counters->degenerate = tot.degenerate;
    counters->v_roots = tot.v_roots;
    counters->u_roots = tot.u_roots;
    counters->admissible = tot.admissible;
    counters->flagged = tot.flagged;
  }
  const int64_t m = std::min<int64_t>(capacity, int64_t(all.size()));
  for (int64_t i = 0; i < m; ++i) {
    const Path& p = all[i];
    oracle_path& o = out[i];
    std::memset(&o, 0, sizeof(o));
    o.chain = p.chain;
    o.query = p.query;
    o.tri0 = p.tri0;
    o.tri1 = p.tri1;
    std::memcpy(o.uv, p.uv, sizeof(o.uv));
    std::memcpy(o.x, p.x, sizeof(o.x));
    o.residual = p.residual;
    o.flags = p.flags;
  }
  return int64_t(all.size()) > capacity ? -1 : 0;
}

// Debug entry: the bivariate system of one 1-bounce candidate.  Writes a and b
// on square grids a_out[(i)*(7)+j], b_out[i*7+j] (degree <= 6) and their exact
// total degrees, u-degrees and the projection choice.
int oracle_system_k1(const double* tri18, const double* x0, const double* x2, int type, double eta0,
                     double eta1, double* a_out, double* b_out, int* info) {
  Tri tr = load_tri(tri18, 1, 0);
  BPoly a, b;
  build_k1(tr, d3(x0), d3(x2), type, eta0, eta1, &a, &b);
  std::memset(a_out, 0, sizeof(double) * 49);
  std::memset(b_out, 0, sizeof(double) * 49);
  for (int i = 0; i <= a.deg; ++i)
    for (int j = 0; i + j <= a.deg; ++j) a_out[i * 7 + j] = a.at(i, j);
  for (int i = 0; i <= b.deg; ++i)
    for (int j = 0; i + j <= b.deg; ++j) b_out[i * 7 + j] = b.at(i, j);
  D3 bvec;
  int edge;
  choose_projection(tr, d3(x0), d3(x2), type, &bvec, &edge);
  info[0] = btotal_deg(a, 1e-12);
  info[1] = btotal_deg(b, 1e-12);
  info[2] = bdeg_u(a);
  info[3] = bdeg_u(b);
  info[4] = edge;
  info[5] = bvec.x != 0.0 ? 0 : (bvec.z != 0.0 ? 2 : 1);
  return 0;
}

// Debug entry: r(v) = det of the Bezout matrix of two bivariate polynomials
// given on square grids (coefficient of u^i v^j at [i*(dmax+1)+j]), with the
// u-degree trimming of the solver.  Writes r's coefficients (low to high) and
// returns its length (0 if r vanishes), or -1 if r_cap is too small.
int oracle_resultant(const double* a_grid, const double* b_grid, int dmax, double* r_out, int r_cap) {
  BPoly a(dmax), b(dmax);
  for (int i = 0; i <= dmax; ++i)
    for (int j = 0; i + j <= dmax; ++j) {
      a.at(i, j) = a_grid[i * (dmax + 1) + j];
      b.at(i, j) = b_grid[i * (dmax + 1) + j];
    }
  const int da = bdeg_u(a), db = bdeg_u(b);
  const int n = std::max(da, db);
  if (da < 0 || db < 0 || n < 1) return 0;
  std::vector<UPoly> ac, bc;
  for (int i = 0; i <= da; ++i) ac.push_back(bcoef_u(a, i));
  for (int i = 0; i <= db; ++i) bc.push_back(bcoef_u(b, i));
  std::vector<UPoly> R = bezout_matrix(ac, bc, n);
  std::vector<int> cols(n);
  for (int j = 0; j < n; ++j) cols[j] = j;
  UPoly r = laplace_det(R, n, 0, cols);
  utrim(r);
  if (int(r.size()) > r_cap) return -1;
  for (size_t i = 0; i < r.size(); ++i) r_out[i] = r[i];
  return int(r.size());
}

// Debug entry: real roots of a univariate polynomial on [lo, hi] by the
// recursive-derivative isolation.  Returns the root count (or -1 if the
// buffer is too small); flags receive F_TANGENT | F_ILL_COND for tangent roots.
int oracle_isolate(const double* p, int len, double lo, double hi, double* roots, uint32_t* flags, int cap) {
  UPoly q(p, p + len);
  std::vector<Root> rs = isolate(q, lo, hi, true);
  if (int(rs.size()) > cap) return -1;
  for (size_t i = 0; i < rs.size(); ++i) {
    roots[i] = rs[i].x;
    flags[i] = rs[i].flags;
  }
  return int(rs.size());
}

}  // extern "C"
