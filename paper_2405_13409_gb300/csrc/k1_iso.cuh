// Isolation kernel of the 1-bounce solve for the common Bezout sizes
// (R: n = 3 or 4, T: n = 5 or 6), templated on the arithmetic type of the
// univariate phase.  Candidates whose trimmed size differs go to a side
// queue handled in FP64 by the side kernel.
#pragma once
#include "k1_sys.cuh"
#include "laplace_gen.cuh"

namespace spoly {

// Post-Laplace steps shared by the sized and generic kernels: power-of-two
// normalisation and trimming of r, recursive-derivative isolation and the
// u-range pre-filter.  Returns the number of brackets written to `items`,
// -1 if r vanishes identically, or (T = float) -2 when the FP32 isolation is
// not certified (kCert32*): the candidate is then re-isolated in FP64.  `ra`
// (T = float) holds the expansion over |E| of the same entries; FP64 callers
// pass r again.
template <typename T, int RD, int DB>
SPOLY_D int k1_finish(const K1Sys<DB>& s, T (&r)[RD + 1], const T (&ra)[RD + 1], RootItem (&items)[kRD + 1],
                      int chain, unsigned& n_vroots, unsigned& n_pref) {
  constexpr bool fp32 = sizeof(T) == 4;
  // Power-of-two normalisation of r and trimming of negligible leading terms
  // (their contribution over the domain is below kTrim of the largest term).
  const double inv_t = scale2(1.0, -s.sc.kt);  // 1 / t, exact
  const T Z = T((1.0 + kDelta) * inv_t);
  T mx = T(0);
#pragma unroll
  for (int c = 0; c <= RD; ++c) mx = fmax(mx, fabs(r[c]));
  if (!(mx > T(0))) return fp32 ? -2 : -1;
  if (fp32 && mx < T(kCert32Tiny)) return -2;
  int e2;
  frexp(mx, &e2);
#pragma unroll
  for (int c = 0; c <= RD; ++c) r[c] = ldexp(r[c], -e2);
  T zpow[RD + 1];
  zpow[0] = T(1);
#pragma unroll
  for (int c = 1; c <= RD; ++c) zpow[c] = zpow[c - 1] * Z;
  T mxz = T(0);
#pragma unroll
  for (int c = 0; c <= RD; ++c) mxz = fmax(mxz, fabs(r[c]) * zpow[c]);
  int deg = RD;
#pragma unroll
  for (int c = RD; c >= 1; --c)
    if (c == deg && fabs(r[c]) * zpow[c] <= T(kTrim) * mxz) --deg;
  if (deg < 1) return 0;
  // sum_i |p_i| t^-i: the magnitude scale of r over v in [0, 1].
  T rscale = T(0);
  {
    const T it = T(inv_t);
    T zz = T(1);
#pragma unroll
    for (int c = 0; c <= RD; ++c) {
      if (c <= deg) rscale += fabs(r[c]) * zz;
      zz *= it;
    }
  }
  const T lo = T(-kDelta * inv_t), hi = Z;
  const T tol = fp32 ? T(kIsoTol32 * inv_t) : T(kIsoTol64 * inv_t);
  const T tang = fp32 ? T(kTangent32) : T(kTangent64);
  if constexpr (fp32) {
    // cancellation ratio of the expansion, then both ends of the domain
    const T it = T(inv_t);
    T Rs = T(0), zz = T(1);
#pragma unroll
    for (int c = 0; c <= RD; ++c) {
      if (c <= deg) Rs += ldexp(ra[c], -e2) * zz;
      zz *= it;
    }
    if (!(Rs <= T(kCert32Cancel) * rscale)) return -2;
    T flo = T(0), fhi = T(0);
#pragma unroll
    for (int c = RD; c >= 0; --c)
      if (c <= deg) {
        flo = fma(flo, lo, r[c]);
        fhi = fma(fhi, hi, r[c]);
      }
    if (fabs(flo) <= T(kCert32Dip) * rscale || fabs(fhi) <= T(kCert32Dip) * rscale) return -2;
  }
  T blo[RD + 1], bhi[RD + 1];
  uint32_t bfl[RD + 1];
  const int nb = isolate<T, RD>(r, deg, lo, hi, tol, tang, rscale, blo, bhi, bfl, fp32 ? T(kCert32Dip) : T(0));
  if (nb < 0) return -2;
  n_vroots += nb;
  // Pre-polish filter: keep a bracket only if a(u, v) = 0 has a real u within
  // kPrefilterMargin of [0, 1 - v] (or a(., v) is degenerate), at the bracket
  // or kPrefilterDv away from it on either side in v: where the curve a = 0
  // runs nearly parallel to the u axis, u(v) amplifies the error of the FP32
  // root, and the side samples catch it.
  int nq = 0;
  for (int k = 0; k < nb; ++k) {
    const T zm = T(0.5) * (blo[k] + bhi[k]);
    const T m = T(kPrefilterMargin);
    bool keep = (s.na == 0);
    for (int side = 0; side < 3 && !keep; ++side) {
      const T z = zm + T(side == 0 ? 0.0 : (side == 1 ? -kPrefilterDv : kPrefilterDv) / s.sc.t);
      const T v = z * T(s.sc.t);
      T am[3];
      a_at<T>(s.a, s.na, z, am);
      T w[2];
      uint32_t wf[2];
      const int nw = quad_roots<T>(am[0], am[1], am[2], T(1e-3), w, wf);
      if (nw == 0 && fabs(am[0]) + fabs(am[1]) + fabs(am[2]) == T(0)) keep = true;
      for (int i = 0; i < nw; ++i) {
        const T u = w[i] * T(s.sc.s);
        if (u >= -m && u <= T(1) - v + m) keep = true;
      }
    }
    if (!keep) {
      ++n_pref;
      continue;
    }
    RootItem itm;
    itm.zlo = double(blo[k]);
    itm.zhi = double(bhi[k]);
    itm.chain = chain;
    itm.flags = bfl[k];
    itm.rscale = float(rscale);
    itm.pad = e2;
    items[nq++] = itm;
  }
  return nq;
}

// Resultant of the generic size N by the unrolled Laplace expansion, then
// the shared post-processing.
template <typename T, int N, int DB>
SPOLY_D int k1_isolate_sized(const K1Sys<DB>& s, RootItem (&items)[kRD + 1], int chain, unsigned& n_vroots,
                             unsigned& n_pref) {
  constexpr int ED = 2 + DB - 1;
  constexpr int RD = N * (ED - N + 1);
  T r[RD + 1];
  T ra[RD + 1];  // FP32: the expansion over |E| (certification); unused in FP64
  {
    T E[sym_size(N, ED)];
    bezout_sym<T, N, 2, DB>(s.a, s.b, s.na, s.nb, E);
    if constexpr (N == 2 && DB == 4) laplace_R2<T>(E, r);
    if constexpr (N == 3 && DB == 4) laplace_R3<T>(E, r);
    if constexpr (N == 4 && DB == 4) laplace_R4<T>(E, r);
    if constexpr (N == 2 && DB == 6) laplace_T2<T>(E, r);
    if constexpr (N == 3 && DB == 6) laplace_T3<T>(E, r);
    if constexpr (N == 4 && DB == 6) laplace_T4<T>(E, r);
    if constexpr (N == 5 && DB == 6) laplace_T5<T>(E, r);
    if constexpr (N == 6 && DB == 6) laplace_T6<T>(E, r);
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int i = 0; i < sym_size(N, ED); ++i) E[i] = fabs(E[i]);
      if constexpr (N == 2 && DB == 4) laplace_abs_R2<T>(E, ra);
      if constexpr (N == 3 && DB == 4) laplace_abs_R3<T>(E, ra);
      if constexpr (N == 4 && DB == 4) laplace_abs_R4<T>(E, ra);
      if constexpr (N == 2 && DB == 6) laplace_abs_T2<T>(E, ra);
      if constexpr (N == 3 && DB == 6) laplace_abs_T3<T>(E, ra);
      if constexpr (N == 4 && DB == 6) laplace_abs_T4<T>(E, ra);
      if constexpr (N == 5 && DB == 6) laplace_abs_T5<T>(E, ra);
      if constexpr (N == 6 && DB == 6) laplace_abs_T6<T>(E, ra);
    } else {
#pragma unroll
      for (int c = 0; c <= RD; ++c) ra[c] = T(0);
    }
  }
  return k1_finish<T, RD, DB>(s, r, ra, items, chain, n_vroots, n_pref);
}

// Isolation with the unrolled expansion of the candidate's Bezout size;
// -2 when the size has none (handled by the generic runtime-size path).
template <typename T, int DB>
SPOLY_D int k1_isolate_dispatch(const K1Sys<DB>& s, RootItem (&items)[kRD + 1], int chain, unsigned& n_v,
                                unsigned& n_pref) {
  if constexpr (DB == 4) {
    if (s.n == 3) return k1_isolate_sized<T, 3, 4>(s, items, chain, n_v, n_pref);
    if (s.n == 4) return k1_isolate_sized<T, 4, 4>(s, items, chain, n_v, n_pref);
    if (s.n == 2) return k1_isolate_sized<T, 2, 4>(s, items, chain, n_v, n_pref);
  } else {
    if (s.n == 6) return k1_isolate_sized<T, 6, 6>(s, items, chain, n_v, n_pref);
    if (s.n == 5) return k1_isolate_sized<T, 5, 6>(s, items, chain, n_v, n_pref);
    if (s.n == 4) return k1_isolate_sized<T, 4, 6>(s, items, chain, n_v, n_pref);
    if (s.n == 3) return k1_isolate_sized<T, 3, 6>(s, items, chain, n_v, n_pref);
    if (s.n == 2) return k1_isolate_sized<T, 2, 6>(s, items, chain, n_v, n_pref);
  }
  return -2;
}

// Flat-shaded triangles (bit-identical vertex normals) degenerate the system:
// a loses u-degree, det = lc(b)^(n-m) Res gains a high-multiplicity spurious
// root, and FP32 isolation can lose true roots beside it.  They take the FP64
// isolation in mixed mode (integer compares: no FP64 pipe work).
SPOLY_D bool flat_shaded(const TriD& tr) {
  auto eq = [](d3 a, d3 b) {
    return __double_as_longlong(a.x) == __double_as_longlong(b.x) &&
           __double_as_longlong(a.y) == __double_as_longlong(b.y) &&
           __double_as_longlong(a.z) == __double_as_longlong(b.z);
  };
  return eq(tr.n0, tr.n1) && eq(tr.n0, tr.n2);
}

#ifndef SPOLY_HOST_BUILD
// Isolation of the chains [base, base + width) by one warp (lane l < width
// takes chain base + l): per-chain numerics, then warp-aggregated counters
// and appends.  All lanes call it.
template <typename T>
SPOLY_D void isolate_warp(const K1Params& P, int64_t base, int lane, int width = 32) {
  const int64_t c = lane < width ? base + lane : P.n_chains;
  RootItem items[kRD + 1];
  int nq = 0;
  unsigned n_v = 0, n_pref = 0, n_deg = 0, n_cand = 0, n_side = 0;
  if (c < P.n_chains) {
    const int q = __ldg(P.chains + 3 * c);
    const int t = __ldg(P.chains + 3 * c + 1);
    if (__ldg(P.qv.k + q) == 1) {
      n_cand = 1;
      const QueryD qd = load_query(P.qv.x_first, P.qv.x_last, P.qv.eta, P.qv.types, q);
      const TriD tr = load_tri(P.mesh.tri, P.mesh.n_tris, t);
      int r = 0;
      if (qd.type == SPOLY_R) {
        K1Sys<4> s;
        r = k1_system<4>(tr, qd, s) ? k1_isolate_dispatch<T, 4>(s, items, int(c), n_v, n_pref) : -1;
      } else {
        K1Sys<6> s;
        r = k1_system<6>(tr, qd, s) ? k1_isolate_dispatch<T, 6>(s, items, int(c), n_v, n_pref) : -1;
      }
      if (sizeof(T) == 4 && r != -1 && flat_shaded(tr)) {
        r = -2;  // the FP32 brackets are discarded; the side kernel re-isolates in FP64
        n_v = n_pref = 0;
      }
      if (r == -1) n_deg = 1;
      if (r == -2) n_side = 1;
      nq = r > 0 ? r : 0;
    }
  }
  warp_count(P.counters + C_CANDIDATES, n_cand);
  warp_count(P.counters + C_DEGENERATE, n_deg);
  warp_count(P.counters + C_VROOTS, n_v);
  warp_count(P.counters + C_PREFILTERED, n_pref);
  const unsigned long long sslot = warp_append(P.counters + C_SIDE, n_side);
  if (n_side && sslot < (unsigned long long)P.side_cap) P.side[sslot] = int32_t(c);
  const unsigned long long slot = warp_append(P.counters + C_QUEUED, unsigned(nq));
  for (int k = 0; k < nq; ++k) {
    const unsigned long long idx = slot + k;
    if (idx < (unsigned long long)P.queue_cap) P.queue[idx] = items[k];
  }
}

// `width` chains per warp (a power of two up to 32).  A short list uses fewer
// lanes per warp and more warps: the chains' different Bezout sizes and loop
// counts then diverge within fewer lanes, and every FP64 warp instruction
// costs the same whatever its active lanes (one warp per SM sub-partition
// keeps the FP64 units busy either way).
template <typename T>
__global__ void __launch_bounds__(128) k1_isolate_kernel(K1Params P, int width) {
  const int lane = threadIdx.x & 31;
  const int64_t n_warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t base = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * width; base < P.n_chains;
       base += n_warps * width)
    isolate_warp<T>(P, base, lane, width);
}

// Persistent variant: a fixed grid whose warps take `chunk` chains at a time
// from a global ticket counter (counters[C_TICKET]) until the list is
// exhausted, so chains of uneven cost (Bezout sizes, root counts, the FP64
// side path) balance across the GPU.
template <typename T>
__global__ void __launch_bounds__(128) k1_isolate_persistent_kernel(K1Params P, int chunk) {
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(P.counters + C_TICKET, (unsigned long long)chunk);
    b = __shfl_sync(0xffffffffu, b, 0);
    if (b >= (unsigned long long)P.n_chains) break;
    for (int sub = 0; sub < chunk; sub += 32) {
      const int64_t base = int64_t(b) + sub;
      if (base >= P.n_chains) break;
      isolate_warp<T>(P, base, lane);
    }
  }
}
#endif

}  // namespace spoly
