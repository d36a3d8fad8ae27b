// TT chains, FP64 phase 1: piece enumeration and construction of the
// bivariate system (Sec. 3.4-3.5) per (chain, sqrt piece), one warp per
// system with its polynomials in shared memory.
#include "scan.cuh"
#include "tt_kernels.cuh"

namespace spoly {

// Argument of the sqrt approximant at a point p with normal n: x = beta / s,
// beta = |n|^2 |d|^2 - eta'^2 (|n|^2 |d|^2 - (d.n)^2), d = p - x0.
SPOLY_D double sqrt_arg(d3 p, d3 n, d3 x0, double er, double s) {
  const d3 d = p - x0;
  const double nd = dot(n, n) * dot(d, d), dn = dot(d, n);
  return (nd - er * er * (nd - dn * dn)) / s;
}

SPOLY_D int piece_of(const SqrtTable& tb, double x) {
  x = fmin(fmax(x, 0.0), 1.0);
  int k = 0;
  while (k < kSqrtPieces - 1 && x >= tb.breaks[k + 1]) ++k;
  return k;
}

// Pieces of the approximant spanned by x over the triangle (centroid and
// vertices), as a bit mask.
SPOLY_D unsigned tt_pieces(const TriD& t1, d3 x0, double e0, double e1, const SqrtTable& tb, double* s_out) {
  const d3 c = (1.0 / 3.0) * (t1.p0 + t1.p1 + t1.p2);
  const d3 nc = (1.0 / 3.0) * (t1.n0 + t1.n1 + t1.n2);
  const double s = dot(nc, nc) * dot(c - x0, c - x0);
  const double er = e0 / e1;
  unsigned m = 1u << piece_of(tb, sqrt_arg(c, nc, x0, er, s));
  m |= 1u << piece_of(tb, sqrt_arg(t1.p0, t1.n0, x0, er, s));
  m |= 1u << piece_of(tb, sqrt_arg(t1.p1, t1.n1, x0, er, s));
  m |= 1u << piece_of(tb, sqrt_arg(t1.p2, t1.n2, x0, er, s));
  *s_out = s;
  return m;
}

// Pieces spanned by each chain: count into chain_sys[2c + 1], mask kept.
__global__ void tt_count_kernel(TTParams P, uint8_t* masks) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < P.n_chains; c += stride) {
    const int q = P.chains[3 * c], t1 = P.chains[3 * c + 1];
    const QueryD qd = load_query(P.qv.x_first, P.qv.x_last, P.qv.eta, P.qv.types, q);
    const TriD a = load_tri(P.mesh.tri, P.mesh.n_tris, t1);
    double s;
    // an RR chain (exact reflected direction) is one system
    const unsigned mask = chain_kind(P.qv.types, q) == kChainRR ? 1u : tt_pieces(a, qd.x0, qd.eta0, qd.eta1, P.sqrt_tab, &s);
    masks[c] = uint8_t(mask);
    P.chain_sys[2 * c + 1] = __popc(mask);
  }
}

// One system per spanned piece at chain_sys[2c] + k: a chain's systems are
// contiguous and ordered by chain.
__global__ void tt_fill_kernel(TTParams P, const uint8_t* masks) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < P.n_chains; c += stride) {
    const unsigned mask = masks[c];
    const int cnt = __popc(mask);
    int k = 0;
    for (int pc = 0; pc < kSqrtPieces; ++pc)
      if (mask & (1u << pc)) {
        const int64_t i = int64_t(P.chain_sys[2 * c]) + k++;
        if (i < P.sys_cap) {
          TTSys sy{};
          sy.chain = int32_t(c);
          sy.piece = pc;
          sy.da = sy.db = sy.n = -1;
          sy.flags = cnt > 1 ? SPOLY_FLAG_SQRT_SPLIT : 0u;
          P.sys[i] = sy;
        }
      }
  }
}

// Projection axis of the square form at x2 (the switch of Sec. 3.3 read as for one bounce, at the second
// vertex): m = (x3 - c1) x n2c; first of x, z, y with |m_hat . e| >= 0.25.
SPOLY_D int tt_axis(const TriD& t1, const TriD& t2, d3 x3) {
  const d3 c1 = (1.0 / 3.0) * (t1.p0 + t1.p1 + t1.p2);
  const d3 n2 = (1.0 / 3.0) * (t2.n0 + t2.n1 + t2.n2);
  d3 m = cross(x3 - c1, n2);
  const double mn = norm(m);
  if (mn > 0.0) m = (1.0 / mn) * m;
  if (fabs(m.x) >= kSwitch) return 0;
  if (fabs(m.z) >= kSwitch) return 2;
  if (fabs(m.y) >= kSwitch) return 1;
  return 0;
}

SPOLY_D bool constant_normal(const TriD& t) {
  const d3 a = (1.0 / norm(t.n0)) * t.n0, b = (1.0 / norm(t.n1)) * t.n1, c = (1.0 / norm(t.n2)) * t.n2;
  const double e = fmax(fmax(fmax(fabs(b.x - a.x), fabs(b.y - a.y)), fmax(fabs(b.z - a.z), fabs(c.x - a.x))),
                        fmax(fabs(c.y - a.y), fabs(c.z - a.z)));
  return e < 1e-12;
}

// Builds a, b, u~, v~, kappa of one system (and the intermediates) in the
// warp's arena `base` (stride st); all 32 lanes of the warp call it.
SPOLY_D void tt_construct(const TriD& t1, const TriD& t2, const QueryD& qd, d3 x3, double eta2, int piece,
                          const SqrtTable& tb, double* base, int64_t st) {
  Arena A{base, st, 0};
  const GP a = A.take(kTTDa), b = A.take(kTTDb), ut = A.take(kTTDmap), vt = A.take(kTTDmap), kap = A.take(kTTDmap);
  const d3 x0 = qd.x0;
  const double er = qd.eta0 / qd.eta1;
  // x1, n1 (normal turned to the incident side, reading of Eq. eq_refr_rational)
  const d3 c1 = (1.0 / 3.0) * (t1.p0 + t1.p1 + t1.p2);
  const d3 nc = (1.0 / 3.0) * (t1.n0 + t1.n1 + t1.n2);
  const double sg = dot(c1 - x0, nc) > 0.0 ? -1.0 : 1.0;
  const double s = dot(nc, nc) * dot(c1 - x0, c1 - x0);
  const GV d0 = gv_take(A, 1), n1 = gv_take(A, 1), s2 = gv_take(A, 1), se1 = gv_take(A, 1), x31 = gv_take(A, 1);
  gv_set_lin(d0, t1.p0 - x0, t1.p1 - t1.p0, t1.p2 - t1.p0);
  gv_set_lin(n1, sg * t1.n0, sg * (t1.n1 - t1.n0), sg * (t1.n2 - t1.n0));
  gv_set_lin(s2, t1.p0 - t2.p0, t1.p1 - t1.p0, t1.p2 - t1.p0);
  gv_set_lin(x31, x3 - t1.p0, -1.0 * (t1.p1 - t1.p0), -1.0 * (t1.p2 - t1.p0));
  const d3 e21 = t2.p1 - t2.p0, e22 = t2.p2 - t2.p0;
  // se1 = s2 x e21 (linear)
  {
    const d3 c0 = mk(s2.x.at(0, 0), s2.y.at(0, 0), s2.z.at(0, 0));
    const d3 cu = mk(s2.x.at(1, 0), s2.y.at(1, 0), s2.z.at(1, 0));
    const d3 cv = mk(s2.x.at(0, 1), s2.y.at(0, 1), s2.z.at(0, 1));
    gv_set_lin(se1, cross(c0, e21), cross(cu, e21), cross(cv, e21));
  }
  const GP n1sq = A.take(2), dd = A.take(2), dn = A.take(2);
  gp_zero(n1sq);
  gp_zero(dd);
  gp_zero(dn);
  gv_dot_mac(n1sq, n1, n1, 1.0);
  gv_dot_mac(dd, d0, d0, 1.0);
  gv_dot_mac(dn, d0, n1, 1.0);
  const GP nd = A.take(4), beta = A.take(4), Q = A.take(4), num = A.take(4);
  gp_zero(nd);
  gp_mac(nd, n1sq, dd, 1.0);
  gp_zero(beta);
  gp_axpy(beta, nd, 1.0 - er * er);
  gp_mac(beta, dn, dn, er * er);
  const double c0 = tb.c[piece][0], cc1 = tb.c[piece][1], d1 = tb.c[piece][2];
  gp_zero(Q);
  gp_axpy(Q, beta, d1);
  gp_add00(Q, s);
  gp_zero(num);
  gp_axpy(num, beta, cc1);
  gp_add00(num, c0 * s);
  // tang = d0 |n1|^2 - n1 (d0 . n1): degree 3
  const GV tang = gv_take(A, 3);
  gv_zero(tang);
  gp_mac(tang.x, d0.x, n1sq, 1.0);
  gp_mac(tang.y, d0.y, n1sq, 1.0);
  gp_mac(tang.z, d0.z, n1sq, 1.0);
  gp_mac(tang.x, n1.x, dn, -1.0);
  gp_mac(tang.y, n1.y, dn, -1.0);
  gp_mac(tang.z, n1.z, dn, -1.0);
  // D = eta' Q tang - sqrt(s) num n1: degree 7
  const GV D = gv_take(A, 7);
  gv_zero(D);
  const double rs = sqrt(s);
  gp_mac(D.x, Q, tang.x, er);
  gp_mac(D.y, Q, tang.y, er);
  gp_mac(D.z, Q, tang.z, er);
  gp_mac(D.x, num, n1.x, -rs);
  gp_mac(D.y, num, n1.y, -rs);
  gp_mac(D.z, num, n1.z, -rs);
  // de2 = D x e22; u~ = de2 . s2; kappa = de2 . e21; v~ = se1 . D
  const GV de2 = gv_take(A, 7);
  gv_zero(de2);
  gp_axpy(de2.x, D.y, e22.z);
  gp_axpy(de2.x, D.z, -e22.y);
  gp_axpy(de2.y, D.z, e22.x);
  gp_axpy(de2.y, D.x, -e22.z);
  gp_axpy(de2.z, D.x, e22.y);
  gp_axpy(de2.z, D.y, -e22.x);
  gp_zero(ut);
  gv_dot_mac(ut, de2, s2, 1.0);
  gp_zero(kap);
  gv_dot_const_mac(kap, de2, e21, 1.0);
  gp_zero(vt);
  gv_dot_mac(vt, se1, D, 1.0);
  // M2 = kappa n20 + u~ (n21 - n20) + v~ (n22 - n20), or the constant normal
  const GV M2 = gv_take(A, 8);
  gv_zero(M2);
  if (constant_normal(t2)) {
    gp_add00(M2.x, t2.n0.x);
    gp_add00(M2.y, t2.n0.y);
    gp_add00(M2.z, t2.n0.z);
  } else {
    const d3 g1 = t2.n1 - t2.n0, g2 = t2.n2 - t2.n0;
    gp_axpy(M2.x, kap, t2.n0.x);
    gp_axpy(M2.y, kap, t2.n0.y);
    gp_axpy(M2.z, kap, t2.n0.z);
    gp_axpy(M2.x, ut, g1.x);
    gp_axpy(M2.y, ut, g1.y);
    gp_axpy(M2.z, ut, g1.z);
    gp_axpy(M2.x, vt, g2.x);
    gp_axpy(M2.y, vt, g2.y);
    gp_axpy(M2.z, vt, g2.z);
  }
  // K2 = kappa (x3 - p20) - u~ e21 - v~ e22
  const GV K2 = gv_take(A, 8);
  gv_zero(K2);
  const d3 w3 = x3 - t2.p0;
  gp_axpy(K2.x, kap, w3.x);
  gp_axpy(K2.y, kap, w3.y);
  gp_axpy(K2.z, kap, w3.z);
  gp_axpy(K2.x, ut, -e21.x);
  gp_axpy(K2.y, ut, -e21.y);
  gp_axpy(K2.z, ut, -e21.z);
  gp_axpy(K2.x, vt, -e22.x);
  gp_axpy(K2.y, vt, -e22.y);
  gp_axpy(K2.z, vt, -e22.z);
  // a = (D x (x3 - x1)) . M2
  const GV C = gv_take(A, 8);
  gv_zero(C);
  gp_mac(C.x, D.y, x31.z, 1.0);
  gp_mac(C.x, D.z, x31.y, -1.0);
  gp_mac(C.y, D.z, x31.x, 1.0);
  gp_mac(C.y, D.x, x31.z, -1.0);
  gp_mac(C.z, D.x, x31.y, 1.0);
  gp_mac(C.z, D.y, x31.x, -1.0);
  gp_zero(a);
  gv_dot_mac(a, C, M2, 1.0);
  // b = eta1^2 |K2|^2 p1^2 - eta2^2 |D|^2 p2^2
  const int ax = tt_axis(t1, t2, x3);
  const GP p1 = A.take(16), p2 = A.take(16), k2sq = A.take(16), dsq = A.take(16);
  gp_zero(p1);
  gp_zero(p2);
  gp_zero(k2sq);
  gp_zero(dsq);
  gv_cross_axis_mac(p1, D, M2, ax, 1.0);
  gv_cross_axis_mac(p2, K2, M2, ax, 1.0);
  gv_dot_mac(k2sq, K2, K2, 1.0);
  gv_dot_mac(dsq, D, D, 1.0);
  const GP p1sq = A.take(32), p2sq = A.take(32);
  gp_zero(p1sq);
  gp_zero(p2sq);
  gp_mac(p1sq, p1, p1, 1.0);
  gp_mac(p2sq, p2, p2, 1.0);
  gp_zero(b);
  // the factors' true degrees (|K2|^2 16, p1^2 30; |D|^2 14, p2^2 32) keep
  // the products within degree 46; their slots are larger
  gp_mac_trunc(b, k2sq, p1sq, qd.eta1 * qd.eta1);
  gp_mac_trunc(b, dsq, p2sq, -eta2 * eta2);
}

// Edge e of T2 in the tangent t2 = n2 x e of the RR product form at x2
// (reading of the switch "if the equation degenerates", Sec. 3.3, as for one
// bounce): with m = (x3 - c1) x n2c, e21 unless |m^ . e21^| < kSwitch and
// |m^ . e22^| > |m^ . e21^|, then e22.  FP64, as in the oracle.
SPOLY_D d3 rr_edge(const TriD& t1, const TriD& t2, d3 x3) {
  const d3 c1 = (1.0 / 3.0) * (t1.p0 + t1.p1 + t1.p2);
  const d3 n2 = (1.0 / 3.0) * (t2.n0 + t2.n1 + t2.n2);
  const d3 m = cross(x3 - c1, n2);
  const d3 e1 = t2.p1 - t2.p0, e2 = t2.p2 - t2.p0;
  const double mn = norm(m);
  if (!(mn > 0.0)) return e1;
  const double c1v = fabs(dot(m, e1)) / (mn * norm(e1)), c2v = fabs(dot(m, e2)) / (mn * norm(e2));
  return (c1v < kSwitch && c2v > c1v) ? e2 : e1;
}

// Builds a, b, u~, v~, kappa of an RR system (Sec. 3.5, Eq. eq_rr1) in the
// warp's arena: the scaled reflected direction D = d0 |n1|^2 - 2 (d0.n1) n1
// (Eq. eq_431_di) is a polynomial, so the mapping (Eq. eq_rct) is exact and
// a chain is one system.  a = (D x (x3 - x1)) . M2 (degree 8) and
// b = (D.M2)(K2.T2) + (D.T2)(K2.M2) (degree 15) with M2 = kappa n2,
// K2 = kappa d2, T2 = M2 x e.  All 32 lanes call it.
constexpr int kRRWork = 5 * 3 * bsize(1) + 2 * bsize(2) + 2 * 3 * bsize(3) + 3 * 3 * bsize(kTTDmap) + 3 * bsize(4) +
                        2 * bsize(7) + 2 * bsize(8);
static_assert(kRRWork <= kTTWork, "the RR temporaries fit the TT arena");

SPOLY_D void rr_construct(const TriD& t1, const TriD& t2, d3 x0, d3 x3, double* base, int64_t st) {
  Arena A{base, st, 0};
  const GP a = A.take(kTTDa), b = A.take(kTTDb), ut = A.take(kTTDmap), vt = A.take(kTTDmap), kap = A.take(kTTDmap);
  const GV d0 = gv_take(A, 1), n1 = gv_take(A, 1), s2 = gv_take(A, 1), se1 = gv_take(A, 1), x31 = gv_take(A, 1);
  gv_set_lin(d0, t1.p0 - x0, t1.p1 - t1.p0, t1.p2 - t1.p0);
  gv_set_lin(n1, t1.n0, t1.n1 - t1.n0, t1.n2 - t1.n0);
  gv_set_lin(s2, t1.p0 - t2.p0, t1.p1 - t1.p0, t1.p2 - t1.p0);
  gv_set_lin(x31, x3 - t1.p0, -1.0 * (t1.p1 - t1.p0), -1.0 * (t1.p2 - t1.p0));
  const d3 e21 = t2.p1 - t2.p0, e22 = t2.p2 - t2.p0;
  {
    const d3 c0 = mk(s2.x.at(0, 0), s2.y.at(0, 0), s2.z.at(0, 0));
    const d3 cu = mk(s2.x.at(1, 0), s2.y.at(1, 0), s2.z.at(1, 0));
    const d3 cv = mk(s2.x.at(0, 1), s2.y.at(0, 1), s2.z.at(0, 1));
    gv_set_lin(se1, cross(c0, e21), cross(cu, e21), cross(cv, e21));
  }
  const GP n1sq = A.take(2), dn = A.take(2);
  gp_zero(n1sq);
  gp_zero(dn);
  gv_dot_mac(n1sq, n1, n1, 1.0);
  gv_dot_mac(dn, d0, n1, 1.0);
  // D = d0 |n1|^2 - 2 (d0 . n1) n1: degree 3
  const GV D = gv_take(A, 3);
  gv_zero(D);
  gp_mac(D.x, d0.x, n1sq, 1.0);
  gp_mac(D.y, d0.y, n1sq, 1.0);
  gp_mac(D.z, d0.z, n1sq, 1.0);
  gp_mac(D.x, n1.x, dn, -2.0);
  gp_mac(D.y, n1.y, dn, -2.0);
  gp_mac(D.z, n1.z, dn, -2.0);
  // de2 = D x e22; u~ = de2 . s2 (4); kappa = de2 . e21 (3); v~ = se1 . D (4)
  const GV de2 = gv_take(A, 3);
  gv_zero(de2);
  gp_axpy(de2.x, D.y, e22.z);
  gp_axpy(de2.x, D.z, -e22.y);
  gp_axpy(de2.y, D.z, e22.x);
  gp_axpy(de2.y, D.x, -e22.z);
  gp_axpy(de2.z, D.x, e22.y);
  gp_axpy(de2.z, D.y, -e22.x);
  gp_zero(ut);
  gv_dot_mac(ut, de2, s2, 1.0);
  gp_zero(kap);
  gv_dot_const_mac(kap, de2, e21, 1.0);
  gp_zero(vt);
  gv_dot_mac(vt, se1, D, 1.0);
  // M2 = kappa n20 + u~ (n21 - n20) + v~ (n22 - n20) (degree 4), or the
  // constant normal; slots of the mapping's size
  const GV M2 = gv_take(A, kTTDmap);
  gv_zero(M2);
  if (constant_normal(t2)) {
    gp_add00(M2.x, t2.n0.x);
    gp_add00(M2.y, t2.n0.y);
    gp_add00(M2.z, t2.n0.z);
  } else {
    const d3 g1 = t2.n1 - t2.n0, g2 = t2.n2 - t2.n0;
    gp_axpy(M2.x, kap, t2.n0.x);
    gp_axpy(M2.y, kap, t2.n0.y);
    gp_axpy(M2.z, kap, t2.n0.z);
    gp_axpy(M2.x, ut, g1.x);
    gp_axpy(M2.y, ut, g1.y);
    gp_axpy(M2.z, ut, g1.z);
    gp_axpy(M2.x, vt, g2.x);
    gp_axpy(M2.y, vt, g2.y);
    gp_axpy(M2.z, vt, g2.z);
  }
  // K2 = kappa (x3 - p20) - u~ e21 - v~ e22 (degree 4)
  const GV K2 = gv_take(A, kTTDmap);
  gv_zero(K2);
  const d3 w3 = x3 - t2.p0;
  gp_axpy(K2.x, kap, w3.x);
  gp_axpy(K2.y, kap, w3.y);
  gp_axpy(K2.z, kap, w3.z);
  gp_axpy(K2.x, ut, -e21.x);
  gp_axpy(K2.y, ut, -e21.y);
  gp_axpy(K2.z, ut, -e21.z);
  gp_axpy(K2.x, vt, -e22.x);
  gp_axpy(K2.y, vt, -e22.y);
  gp_axpy(K2.z, vt, -e22.z);
  // T2 = M2 x e (degree 4)
  const d3 e = rr_edge(t1, t2, x3);
  const GV T2 = gv_take(A, kTTDmap);
  gv_zero(T2);
  gp_axpy(T2.x, M2.y, e.z);
  gp_axpy(T2.x, M2.z, -e.y);
  gp_axpy(T2.y, M2.z, e.x);
  gp_axpy(T2.y, M2.x, -e.z);
  gp_axpy(T2.z, M2.x, e.y);
  gp_axpy(T2.z, M2.y, -e.x);
  // a = (D x (x3 - x1)) . M2
  const GV C = gv_take(A, 4);
  gv_zero(C);
  gp_mac(C.x, D.y, x31.z, 1.0);
  gp_mac(C.x, D.z, x31.y, -1.0);
  gp_mac(C.y, D.z, x31.x, 1.0);
  gp_mac(C.y, D.x, x31.z, -1.0);
  gp_mac(C.z, D.x, x31.y, 1.0);
  gp_mac(C.z, D.y, x31.x, -1.0);
  gp_zero(a);
  gv_dot_mac(a, C, M2, 1.0);
  // b = (D.M2)(K2.T2) + (D.T2)(K2.M2); the factors' true degrees (7, 8) sit
  // below their slots' sums, which the products truncate to
  const GP dm = A.take(7), kt = A.take(8), dt = A.take(7), km = A.take(8);
  gp_zero(dm);
  gp_zero(kt);
  gp_zero(dt);
  gp_zero(km);
  gv_dot_mac(dm, D, M2, 1.0);
  gv_dot_mac(kt, K2, T2, 1.0);
  gv_dot_mac(dt, D, T2, 1.0);
  gv_dot_mac(km, K2, M2, 1.0);
  gp_zero(b);
  gp_mac(b, dm, kt, 1.0);
  gp_mac(b, dt, km, 1.0);
}

// log2 x for x > 0 (frexp keeps tiny and huge values exact in the exponent).
SPOLY_D double log2_pos(double x) {
  int e;
  const double m = frexp(x, &e);
  return double(e) + double(log2f(float(m)));
}

// Trimmed u-degrees (a u-power counts above 1e-13 of the polynomial's max-abs), the u scaling u = 2^ks w and the scaled,
// normalised FP32 copy `c32` ([kTT32], a then b) of the system in the warp's
// arena; `rowmax` holds kTTDa + kTTDb + 2 doubles of shared memory.  All 32
// lanes call it.
SPOLY_D void tt_finish(TTSys& sy, double* base, float* c32, double* rowmax) {
  const int lane = threadIdx.x & 31;
  const GP a{base + kOffA, 1, kTTDa}, b{base + kOffB, 1, kTTDb};
  constexpr int kRows = kTTDa + 1 + kTTDb + 1;
  double* ra = rowmax;
  double* rb = rowmax + kTTDa + 1;
  for (int r = lane; r < kRows; r += 32) {
    const bool in_a = r <= kTTDa;
    const GP& p = in_a ? a : b;
    const int i = in_a ? r : r - kTTDa - 1;
    double m = 0.0;
    for (int j = 0; i + j <= p.D; ++j) m = fmax(m, fabs(p.at(i, j)));
    rowmax[r] = m;
  }
  __syncwarp();
  double am = 0.0, bm = 0.0;
  for (int i = 0; i <= kTTDa; ++i) am = fmax(am, ra[i]);
  for (int i = 0; i <= kTTDb; ++i) bm = fmax(bm, rb[i]);
  int da = -1, db = -1;
  for (int i = 0; i <= kTTDa; ++i)
    if (ra[i] > kTrim * am) da = i;
  for (int i = 0; i <= kTTDb; ++i)
    if (rb[i] > kTrim * bm) db = i;
  sy.da = da;
  sy.db = db;
  sy.n = (da < 0 || db < 0) ? -1 : max(da, db);
  if (sy.n < 1) {
    sy.n = -1;
    return;
  }
  // least-squares slope of log2(row max) over the kept rows of both
  double sx = 0, sy2 = 0, sxx = 0, sxy = 0, cnt = 0;
  for (int r = lane; r < kRows; r += 32) {
    const bool in_a = r <= kTTDa;
    const int i = in_a ? r : r - kTTDa - 1;
    const double m = rowmax[r];
    if (m > 0.0 && i <= (in_a ? da : db)) {
      const double l = log2_pos(m / (in_a ? am : bm));
      sx += i;
      sy2 += l;
      sxx += double(i) * i;
      sxy += i * l;
      cnt += 1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy2 += __shfl_xor_sync(0xffffffffu, sy2, o);
    sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
    sxy += __shfl_xor_sync(0xffffffffu, sxy, o);
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  const double den = cnt * sxx - sx * sx;
  const double g = den > 0.0 ? (cnt * sxy - sx * sy2) / den : 0.0;
  int ks = int(rint(-g));
  ks = max(-20, min(20, ks));
  sy.ks = ks;
  // scaled, normalised FP32 copy
  double am2 = 0.0, bm2 = 0.0;
  for (int i = 0; i <= da; ++i) am2 = fmax(am2, ldexp(ra[i], ks * i));
  for (int i = 0; i <= db; ++i) bm2 = fmax(bm2, ldexp(rb[i], ks * i));
  const double ia = 1.0 / am2, ib = 1.0 / bm2;
  for (int t = lane; t < kTT32; t += 32) {
    const bool in_a = t < bsize(kTTDa);
    const int idx = in_a ? t : t - bsize(kTTDa);
    int i, j;
    flat_to_ij(in_a ? kTTDa : kTTDb, idx, i, j);
    const double c = in_a ? a.k(idx) : b.k(idx);
    c32[t] = i <= (in_a ? da : db) ? float(ldexp(c, ks * i) * (in_a ? ia : ib)) : 0.0f;
  }
}

// One warp per system: construction in the warp's shared-memory arena, then
// the kept polynomials to the system's scratch row and the FP32 copy.
constexpr int kBuildWarps = 6;
constexpr int kArena = kTTScratch + kTTDa + kTTDb + 2;  // doubles per warp

__global__ void __launch_bounds__(kBuildWarps * 32) tt_build_kernel(TTParams P) {
  extern __shared__ double build_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double* arena = build_smem + int64_t(warp) * kArena;
  const int64_t nw = int64_t(gridDim.x) * kBuildWarps;
  const int64_t n_sys = tt_n_sys(P);
  for (int64_t i = int64_t(blockIdx.x) * kBuildWarps + warp; i < n_sys; i += nw) {
    TTSys sy = P.sys[P.sys_offset + i];
    const int64_t c = sy.chain;
    const int q = P.chains[3 * c], t1 = P.chains[3 * c + 1], t2 = P.chains[3 * c + 2];
    const QueryD qd = load_query(P.qv.x_first, P.qv.x_last, P.qv.eta, P.qv.types, q);
    const double eta2 = P.qv.eta[3 * q + 2];
    const TriD ta = load_tri(P.mesh.tri, P.mesh.n_tris, t1);
    const TriD tb = load_tri(P.mesh.tri, P.mesh.n_tris, t2);
    const int kind = chain_kind(P.qv.types, q);
    if (kind == kChainRR) {
      rr_construct(ta, tb, qd.x0, qd.x2, arena, 1);
    } else if (kind == kChainTT) {
      tt_construct(ta, tb, qd, qd.x2, eta2, sy.piece, P.sqrt_tab, arena, 1);
    } else {
      // mixed bounce types are not built: a zero system has no roots
      Arena A{arena, 1, 0};
      const GP a = A.take(kTTDa), b = A.take(kTTDb);
      gp_zero(a);
      gp_zero(b);
    }
    double* keep = P.scratch + i * kTTKeep;
    for (int t = lane; t < kTTKeep; t += 32) keep[t] = arena[t];
    tt_finish(sy, arena, P.coef32 + i * kTT32, arena + kTTScratch);
    if (lane == 0) P.sys[P.sys_offset + i] = sy;
    __syncwarp();
  }
}

cudaError_t launch_tt_count(const TTParams& P, uint8_t* masks, int num_sms, cudaStream_t st) {
  if (P.n_chains <= 0) return cudaSuccess;
  const int64_t g = std::min<int64_t>((P.n_chains + 127) / 128, int64_t(num_sms) * 8);
  tt_count_kernel<<<int(g), 128, 0, st>>>(P, masks);
  return cudaGetLastError();
}

cudaError_t launch_tt_fill(const TTParams& P, const uint8_t* masks, int num_sms, cudaStream_t st) {
  if (P.n_chains <= 0) return cudaSuccess;
  const int64_t g = std::min<int64_t>((P.n_chains + 127) / 128, int64_t(num_sms) * 8);
  tt_fill_kernel<<<int(g), 128, 0, st>>>(P, masks);
  return cudaGetLastError();
}

__global__ void tt_counts_kernel(const int32_t* chain_sys, int64_t n, int32_t* cnt) {
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n; c += int64_t(gridDim.x) * blockDim.x)
    cnt[c] = chain_sys[2 * c + 1];
}

__global__ void tt_offsets_kernel(int32_t* chain_sys, int64_t n, const int32_t* cnt, const int64_t* off,
                                  unsigned long long* n_sys) {
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n; c += int64_t(gridDim.x) * blockDim.x) {
    chain_sys[2 * c] = int32_t(off[c]);
    if (c == n - 1) *n_sys = (unsigned long long)(off[c] + cnt[c]);
  }
}

size_t tt_offsets_scratch_bytes(int64_t n_chains) {
  const int64_t nb = n_chains / scan::kScanBlock + 2;
  return size_t(n_chains) * 12 + 256 + size_t(2 * nb + 3 * scan::kScanBlock) * 8;
}

cudaError_t launch_tt_offsets(const TTParams& P, void* tmp, int num_sms, cudaStream_t st) {
  const int64_t n = P.n_chains;
  if (n <= 0) return cudaSuccess;
  char* b = static_cast<char*>(tmp);
  int32_t* cnt = reinterpret_cast<int32_t*>(b);
  int64_t* off = reinterpret_cast<int64_t*>(b + ((size_t(n) * 4 + 255) & ~size_t(255)));
  int64_t* sums = off + n;
  const int64_t nb = n / scan::kScanBlock + 2;
  const int64_t g = std::min<int64_t>((n + 255) / 256, int64_t(num_sms) * 8);
  tt_counts_kernel<<<int(g), 256, 0, st>>>(P.chain_sys, n, cnt);
  cudaError_t e = scan::exclusive_scan<int32_t>(cnt, off, n, sums, sums + nb, sums + 2 * nb, st);
  if (e != cudaSuccess) return e;
  tt_offsets_kernel<<<int(g), 256, 0, st>>>(P.chain_sys, n, cnt, off, P.counters + TT_SYSTEMS);
  return cudaGetLastError();
}

cudaError_t launch_tt_build(const TTParams& P, int num_sms, cudaStream_t st) {
  if (P.n_sys <= 0) return cudaSuccess;
  const size_t smem = size_t(kBuildWarps) * kArena * sizeof(double);
  static bool attr = false;
  if (!attr) {
    const cudaError_t e = cudaFuncSetAttribute(tt_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t g = std::min<int64_t>((P.n_sys + kBuildWarps - 1) / kBuildWarps, int64_t(num_sms));
  tt_build_kernel<<<int(g), kBuildWarps * 32, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace spoly
