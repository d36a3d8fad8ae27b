// Group-cooperative sign of the Bezout determinant of a TT system at one
// value of the hidden variable v1 (Sec. 4.2, k >= 2 branch).
//
// A group of G aligned lanes evaluates one sample.  The matrix is padded to
// a compile-time size N >= n with an identity block (the determinant is
// unchanged) and distributed cyclically: lane g of the group holds the rows
// g, g + G, ..., g + G (R - 1), R = N / G, as R x N registers.
//
//  * Coefficients: lane g evaluates a_i(v), b_i(v) for i = g + G s by Horner.
//  * Bezout matrix (Eq. eq_bezout): B[r][j] = sum_{k <= min(r, n-1-j)}
//    (a_{r-k} b_{j+1+k} - b_{r-k} a_{j+1+k}) obeys the recurrence
//    B[r][j] = B[r-1][j+1] + a_r b_{j+1} - b_r a_{j+1}.  Row r is formed
//    from row r - 1 shifted by one column; lane g forms the columns
//    g + G t of every row, which by the symmetry of B are its own rows.
//    The shift is one shuffle per column slot.
//  * Gaussian elimination with partial pivoting: the pivot is the group's
//    arg-max (ties to the lower row) over rows not yet used, the pivot row
//    is broadcast one column at a time; rows are never moved, and the
//    determinant's sign is the product of the pivots' signs and the parity
//    of the pivot order.
//
// Control flow is uniform across the warp (no early exits; a singular
// column marks the determinant zero and the elimination runs on), so every
// shuffle uses the full warp mask.
#pragma once
#include "tt_kernels.cuh"

namespace spoly {

constexpr unsigned kGroupFull = 0xffffffffu;

// a_i(v), b_i(v) for i = g + G s, s = 0..R (zero above the trimmed degrees).
// `ca`, `cb`: the graded coefficient arrays of a and b (bidx layout).  ks
// (FP64 only): the rows are scaled by 2^(ks i) after Horner, which equals
// scaling every coefficient (an exact power of two).
template <typename T, int N, int G>
SPOLY_D void tt_group_coeffs(const T* __restrict__ ca, const T* __restrict__ cb, T v, int da, int db, int g,
                             T (&av)[N / G + 1], T (&bv)[N / G + 1], int ks = 0) {
  constexpr int R = N / G;
#pragma unroll
  for (int s = 0; s <= R; ++s) {
    const int i = g + G * s;
    T a = T(0), b = T(0);
    if (i <= da) {
      const T* row = ca + bidx(kTTDa, i, 0);
      for (int j = kTTDa - i; j >= 0; --j) a = fma(a, v, row[j]);
    }
    if (i <= db) {
      const T* row = cb + bidx(kTTDb, i, 0);
      for (int j = kTTDb - i; j >= 0; --j) b = fma(b, v, row[j]);
    }
    if (sizeof(T) == 8 && ks != 0) {
      const T sc = T(ldexp(1.0, ks * i));
      a *= sc;
      b *= sc;
    }
    av[s] = a;
    bv[s] = b;
  }
}

// The lane's R rows of the padded Bezout matrix: A[t][c] = B[g + G t][c].
template <typename T, int N, int G>
SPOLY_D void tt_group_bezout(const T (&av)[N / G + 1], const T (&bv)[N / G + 1], int n, int g, T (&A)[N / G][N]) {
  constexpr int R = N / G;
  const int nxt = (g + 1) & (G - 1);
  // a_q, b_q for q = g + G t + 1 live on lane g + 1, slot t (lane 0, slot
  // t + 1, for the group's last lane)
  T aq[R], bq[R];
#pragma unroll
  for (int t = 0; t < R; ++t) {
    aq[t] = __shfl_sync(kGroupFull, g == 0 ? av[t + 1] : av[t], nxt, G);
    bq[t] = __shfl_sync(kGroupFull, g == 0 ? bv[t + 1] : bv[t], nxt, G);
  }
#pragma unroll
  for (int r = 0; r < N; ++r) {
    const T ar = __shfl_sync(kGroupFull, av[r / G], r % G, G);
    const T br = __shfl_sync(kGroupFull, bv[r / G], r % G, G);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      // B[r-1][g + G t + 1], by the same neighbour rule; zero past column N - 1
      T sh = T(0);
      if (r > 0) {
        const T snd = (g == 0) ? (t + 1 < R ? A[t + 1][r - 1] : T(0)) : A[t][r - 1];
        sh = __shfl_sync(kGroupFull, snd, nxt, G);
      }
      A[t][r] = fma(ar, bq[t], fma(-br, aq[t], sh));
    }
  }
  // identity block beyond the Bezout size
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const int id = g + G * t;
#pragma unroll
    for (int c = 0; c < N; ++c)
      if (id >= n || c >= n) A[t][c] = (id == c) ? T(1) : T(0);
  }
}

// log2 |x| for x != 0 without overflow or underflow in either precision.
template <typename T>
SPOLY_D float tt_log2_abs(T x) {
  int e;
  const T m = frexp(fabs(x), &e);
  return float(e) + log2f(float(m));
}

// Sign of det A (0 if singular) and log2 |det A| (-1e30 if singular).
template <typename T, int N, int G>
SPOLY_D int tt_group_eliminate(T (&A)[N / G][N], int g, float* log2abs) {
  constexpr int R = N / G;
  unsigned used = 0u;
  int sg = 1, par = 0;
  bool zero = false;
  float l2 = 0.0f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    T best = T(-1);
    int bi = N;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int id = g + G * t;
      const T x = fabs(A[t][k]);
      if (!((used >> id) & 1u) && x > best) {
        best = x;
        bi = id;
      }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(kGroupFull, best, o, G);
      const int oi = __shfl_xor_sync(kGroupFull, bi, o, G);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    const bool sing = !(best > T(0));
    zero |= sing;
    // a singular column (or NaN entries) still takes an unused row, so the
    // bookkeeping stays consistent while the remaining steps run
    const int p = (bi < N) ? bi : __ffs(~used) - 1;
    const int owner = p & (G - 1), slot = p / G;
    auto pick = [&](int c) {
      T x = A[0][c];
#pragma unroll
      for (int t = 1; t < R; ++t) x = (slot == t) ? A[t][c] : x;
      return x;
    };
    const T pv = __shfl_sync(kGroupFull, pick(k), owner, G);
    if (!sing) {
      if (pv < T(0)) sg = -sg;
      l2 += tt_log2_abs(pv);
    }
    par += __popc(~used & ((1u << p) - 1u));
    used |= 1u << p;
    const T rcp = sing ? T(0) : T(1) / pv;
    T f[R];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int id = g + G * t;
      f[t] = ((used >> id) & 1u) ? T(0) : A[t][k] * rcp;
    }
    // constant trip count, so that the loop unrolls and A stays in registers
#pragma unroll
    for (int c = 0; c < N; ++c) {
      if (c <= k) continue;
      const T pc = __shfl_sync(kGroupFull, pick(c), owner, G);
#pragma unroll
      for (int t = 0; t < R; ++t) A[t][c] = fma(-f[t], pc, A[t][c]);
    }
  }
  *log2abs = zero ? -1e30f : l2;
  return zero ? 0 : ((par & 1) ? -sg : sg);
}

struct GroupSign {
  int sign;    // -1, 0, 1
  float log2;  // log2 |det| (-1e30 when zero)
};

// Sign and log2 |det| of the system at v for the calling group; every lane
// of the warp calls it (possibly with different v per group).  Kept out of
// line: each (T, N, G) body is compiled once however often it is called.
template <typename T, int N, int G>
__device__ __noinline__ GroupSign tt_group_sign(const T* ca, const T* cb, T v, int da, int db, int n, int g,
                                                int ks = 0) {
  T av[N / G + 1], bv[N / G + 1];
  tt_group_coeffs<T, N, G>(ca, cb, v, da, db, g, av, bv, ks);
  T A[N / G][N];
  tt_group_bezout<T, N, G>(av, bv, n, g, A);
  GroupSign r;
  r.sign = tt_group_eliminate<T, N, G>(A, g, &r.log2);
  return r;
}

}  // namespace spoly
