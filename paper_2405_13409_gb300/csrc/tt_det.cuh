// Warp-cooperative sign of the Bezout determinant of a TT system at one value
// of the hidden variable v1 (Sec. 5.2, k >= 2): lane r holds row r of the
// n x n matrix (n <= 31); Gaussian elimination with partial pivoting picks
// the pivot by a warp arg-max and broadcasts the pivot row by shuffles.  The
// determinant's sign is the product of the pivots' signs and the parity of
// the pivot order; its log2 magnitude is the sum of the pivots' log2.
#pragma once
#include "tt_kernels.cuh"

namespace spoly {

constexpr unsigned kFull = 0xffffffffu;

// Coefficients in w (u = 2^ks w) of a and b at v: lane i writes a_i(v) and
// b_i(v) to sa[i], sb[i] (zero above the trimmed degrees, up to index n).
// `ca(i, j)`, `cb(i, j)` read the scaled coefficient of w^i v^j.
template <typename T, typename CA, typename CB>
SPOLY_D void tt_coeffs_at(T v, int da, int db, int n, int lane, CA ca, CB cb, T* sa, T* sb) {
  T av = T(0), bv = T(0);
  if (lane <= da) {
    for (int j = kTTDa - lane; j >= 0; --j) av = fma(av, v, ca(lane, j));
  }
  if (lane <= db) {
    for (int j = kTTDb - lane; j >= 0; --j) bv = fma(bv, v, cb(lane, j));
  }
  if (lane <= n) {
    sa[lane] = av;
    sb[lane] = bv;
  }
  __syncwarp();
}

// Row r of the Bezout matrix of Eq. eq_bezout from the coefficients at v.
template <typename T, int N>
SPOLY_D void tt_bezout_row(const T* sa, const T* sb, int n, int r, T (&row)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T s = T(0);
    if (r < n && j < n) {
      const int kmax = min(r, n - 1 - j);
      for (int k = 0; k <= kmax; ++k) s = fma(sa[r - k], sb[j + 1 + k], fma(-sb[r - k], sa[j + 1 + k], s));
    }
    row[j] = s;
  }
}

template <typename T, int N>
SPOLY_D int tt_warp_det_sign(T (&row)[N], int n, int lane, float* log2abs) {
  unsigned used = 0u;
  const unsigned nmask = n >= 32 ? kFull : ((1u << n) - 1u);
  int sg = 1, par = 0;
  float l2 = 0.0f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    if (k >= n) break;
    const bool mine = lane < n && !((used >> lane) & 1u);
    T key = mine ? fabs(row[k]) : T(-1);
    int idx = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ok = __shfl_xor_sync(kFull, key, o);
      const int oi = __shfl_xor_sync(kFull, idx, o);
      if (ok > key || (ok == key && oi < idx)) {
        key = ok;
        idx = oi;
      }
    }
    if (!(key > T(0))) {
      *log2abs = -1e30f;
      return 0;
    }
    const int p = idx;
    const T pv = __shfl_sync(kFull, row[k], p);
    if (pv < T(0)) sg = -sg;
    par += __popc(~used & ((1u << p) - 1u) & nmask);
    used |= 1u << p;
    l2 += log2f(float(fabs(pv)));
    const bool act = lane < n && !((used >> lane) & 1u);
    const T f = act ? row[k] / pv : T(0);
#pragma unroll
    for (int j = k + 1; j < N; ++j) {
      if (j >= n) break;
      const T pj = __shfl_sync(kFull, row[j], p);
      if (act) row[j] = fma(-f, pj, row[j]);
    }
  }
  *log2abs = l2;
  return (par & 1) ? -sg : sg;
}

// Sign (and log2 |det|) of the system at v, for one warp.
template <typename T, int N, typename CA, typename CB>
SPOLY_D int tt_sign_at(T v, int da, int db, int n, int lane, CA ca, CB cb, T* sa, T* sb, float* l2) {
  tt_coeffs_at<T>(v, da, db, n, lane, ca, cb, sa, sb);
  T row[N];
  tt_bezout_row<T, N>(sa, sb, n, lane, row);
  __syncwarp();
  return tt_warp_det_sign<T, N>(row, n, lane, l2);
}

}  // namespace spoly
