// Generic-size (runtime n) FP64 path of the 1-bounce univariate phase, used
// for Bezout sizes without an unrolled expansion.
#pragma once
#include "k1_iso.cuh"

namespace spoly {

// Bezout entry (i, j) for a runtime size n (Eq. eq_bezout).
template <int DB>
SPOLY_D void bezout_entry_rt(const BPd<2>& a, const BPd<DB>& b, int na, int nb, int n, int i, int j,
                             double (&out)[DB + 2]) {
  constexpr int ED = DB + 1;
  for (int c = 0; c <= ED; ++c) out[c] = 0.0;
  const int kmax = min(i, n - 1 - j);
  for (int k = 0; k <= kmax; ++k) {
    const int p = i - k, q = j + 1 + k;
    if (p <= 2 && p <= na && q <= DB && q <= nb)
      for (int x = 0; x <= 2 - p; ++x)
        for (int y = 0; y <= DB - q; ++y) out[x + y] += a.c[bidx(2, p, x)] * b.c[bidx(DB, q, y)];
    if (q <= 2 && q <= na && p <= DB && p <= nb)
      for (int x = 0; x <= DB - p; ++x)
        for (int y = 0; y <= 2 - q; ++y) out[x + y] -= b.c[bidx(DB, p, x)] * a.c[bidx(2, q, y)];
  }
}

// Memoised Laplace expansion with a runtime size n <= 6 (Sec. 4.2).
template <int DB>
SPOLY_D void laplace_rt(const double (&E)[6][6][DB + 2], int n, double (&r)[kRD + 1]) {
  constexpr int ED = DB + 1;
  double M[64][kRD + 1];
  for (int j = 0; j < n; ++j)
    for (int c = 0; c <= kRD; ++c) M[1 << j][c] = (c <= ED - (n - 1) - j) ? E[n - 1][j][c] : 0.0;
  for (int row = n - 2; row >= 0; --row) {
    for (unsigned mask = 1; mask < (1u << n); ++mask) {
      if (__popc(mask) != n - row) continue;
      double acc[kRD + 1];
      for (int c = 0; c <= kRD; ++c) acc[c] = 0.0;
      int pos = 0;
      for (int j = 0; j < n; ++j) {
        if (!(mask & (1u << j))) continue;
        const unsigned sub = mask & ~(1u << j);
        const int de = ED - row - j;
        const int ds = minor_deg(n, ED, row + 1, sub);
        if (de >= 0 && ds >= 0)
          for (int x = 0; x <= de; ++x) {
            const double ex = (pos & 1) ? -E[row][j][x] : E[row][j][x];
            for (int y = 0; y <= ds && x + y <= kRD; ++y) acc[x + y] = fma(ex, M[sub][y], acc[x + y]);
          }
        ++pos;
      }
      for (int c = 0; c <= kRD; ++c) M[mask][c] = acc[c];
    }
  }
  for (int c = 0; c <= kRD; ++c) r[c] = M[(1u << n) - 1u][c];
}

template <int DB>
SPOLY_D int k1_generic_one(const K1Sys<DB>& s, RootItem (&items)[kRD + 1], int chain, unsigned& n_v,
                           unsigned& n_pref) {
  double E[6][6][DB + 2];
  for (int i = 0; i < s.n; ++i)
    for (int j = 0; j < s.n; ++j) bezout_entry_rt<DB>(s.a, s.b, s.na, s.nb, s.n, i, j, E[i][j]);
  double r[kRD + 1];
  laplace_rt<DB>(E, s.n, r);
  return k1_finish<double, kRD, DB>(s, r, r, items, chain, n_v, n_pref);
}

}  // namespace spoly
