// Side kernel of the 1-bounce solve, FP64 throughout.
//
// Handles the side queue: candidates whose trimmed Bezout size n is not one
// of the sizes the unrolled kernels are instantiated for (flat or degenerate
// triangles, index-matched refraction), which run the same algorithm with
// runtime loops, and candidates whose FP32 isolation was not certified, which
// re-run the unrolled expansion and the isolation in FP64.  Each chain's
// polish and path phase follow in the same thread.
#include "k1_polish.cuh"

namespace spoly {

// One side chain per thread: FP64 isolation, polish and path phase, so the
// kernel needs nothing from the bracket queue and can run beside the queue's
// polish.  A path re-run (P.rerun) repeats the solve but counts only paths.
// The isolation kernels' post-Laplace steps on the FP64 resultant, at the
// degree bound of the candidate's Bezout size (so that the FP64 loops run over
// that many coefficients, not kRD).
template <int RD, int DB>
SPOLY_D int finish_rd(const K1Sys<DB>& s, const double (&r64)[kRD + 1], RootItem (&items)[kRD + 1], int c,
                      unsigned& n_v, unsigned& n_pref) {
  double r[RD + 1];
#pragma unroll
  for (int k = 0; k <= RD; ++k) r[k] = r64[k];
  return k1_finish<double, RD, DB>(s, r, r, items, c, n_v, n_pref);
}

template <int DB>
SPOLY_D int finish_sized(const K1Sys<DB>& s, const double (&r64)[kRD + 1], RootItem (&items)[kRD + 1], int c,
                         unsigned& n_v, unsigned& n_pref) {
  constexpr int ED = DB + 1;  // entry degree bound of the Bezout matrix (a has total degree 2)
  if constexpr (DB == 4) {
    if (s.n == 4 || s.n == 2) return finish_rd<4 * (ED - 4 + 1), DB>(s, r64, items, c, n_v, n_pref);
    if (s.n == 3) return finish_rd<3 * (ED - 3 + 1), DB>(s, r64, items, c, n_v, n_pref);
  } else {
    if (s.n == 6 || s.n == 2) return finish_rd<6 * (ED - 6 + 1), DB>(s, r64, items, c, n_v, n_pref);
    if (s.n == 5 || s.n == 3) return finish_rd<5 * (ED - 5 + 1), DB>(s, r64, items, c, n_v, n_pref);
    if (s.n == 4) return finish_rd<4 * (ED - 4 + 1), DB>(s, r64, items, c, n_v, n_pref);
  }
  return finish_rd<kRD, DB>(s, r64, items, c, n_v, n_pref);
}

template <int DB, typename Emit>
SPOLY_D int side_solve(const TriD& tr, const QueryD& qd, int c, int q, int t, const PixelFilter& pix, unsigned& n_v,
                       unsigned& n_pref, unsigned& lost, unsigned& n_u, Emit&& emit) {
  K1Sys<DB> s;
  if (!k1_system<DB>(tr, qd, s)) return -1;
  // the FP64 resultant once, for the isolation (the isolation kernels'
  // post-Laplace steps on it; it is already normalised and trimmed, which
  // they repeat exactly) and for the polish
  double r64[kRD + 1];
  const int deg64 = k1_r64<DB>(s, r64);
  RootItem items[kRD + 1];
  const int r = finish_sized<DB>(s, r64, items, c, n_v, n_pref);
  if (r > 0) k1_chain_solve<DB>(s, true, tr, qd, items, r, q, t, pix, lost, n_u, emit, r64, deg64);
  return r;
}

__global__ void __launch_bounds__(64) k1_side_kernel(K1Params P) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const unsigned long long ns = *(volatile unsigned long long*)(P.counters + C_SIDE);
  const int64_t n_side = int64_t(ns < (unsigned long long)P.side_cap ? ns : P.side_cap);
  // A short side queue (no more chains than the grid has warps) takes one
  // chain per warp: its lanes would otherwise run the chains' different
  // Bezout sizes and root counts one after another.
  const int64_t n_warps = stride >> 5;
  const bool per_warp = n_side <= n_warps;
  const int64_t first = per_warp ? (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5
                                 : int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31);
  for (int64_t base = first; base < n_side; base += per_warp ? n_warps : stride) {
    const int64_t i = per_warp ? (lane == 0 ? base : n_side) : base + lane;
    unsigned n_v = 0, n_pref = 0, n_deg = 0, n_q = 0, lost = 0, n_u = 0, n_flag = 0;
    spoly_path out[6];
    int np = 0;
    if (i < n_side) {
      const int c = P.side[i];
      const int q = __ldg(P.chains + 3 * int64_t(c));
      const int t = __ldg(P.chains + 3 * int64_t(c) + 1);
      const QueryD qd = load_query(P.qv.x_first, P.qv.x_last, P.qv.eta, P.qv.types, q);
      const TriD tr = load_tri(P.mesh.tri, P.mesh.n_tris, t);
      auto emit = [&](const spoly_path& p) {
        if (np < 6) {
          out[np++] = p;
          if (p.flags & SPOLY_FLAG_ILL_COND) ++n_flag;
        } else {
          append_path(P, p);
        }
      };
      const int r = (qd.type == SPOLY_R) ? side_solve<4>(tr, qd, c, q, t, P.pix, n_v, n_pref, lost, n_u, emit)
                                         : side_solve<6>(tr, qd, c, q, t, P.pix, n_v, n_pref, lost, n_u, emit);
      n_deg = (r < 0) ? 1u : 0u;
      n_q = r > 0 ? unsigned(r) : 0u;
    }
    if (!P.rerun) {
      warp_count(P.counters + C_DEGENERATE, n_deg);
      warp_count(P.counters + C_VROOTS, n_v);
      warp_count(P.counters + C_PREFILTERED, n_pref);
      warp_count(P.counters + C_SIDE_QUEUED, n_q);
      warp_count(P.counters + C_POLISH_LOST, lost);
    }
    warp_count(P.counters + C_UROOTS, n_u);
    warp_count(P.counters + C_FLAGGED, n_flag);
    const unsigned long long slot = warp_append(P.counters + C_ADMISSIBLE, unsigned(np));
    for (int k = 0; k < np; ++k) {
      const unsigned long long idx = slot + k;
      if (P.chain_ids) out[k].chain = __ldg(P.chain_ids + out[k].chain);
      if (idx < (unsigned long long)P.path_cap) P.paths[idx] = out[k];
    }
  }
}

cudaError_t launch_k1_side(const K1Params& P, int num_sms, cudaStream_t st) {
  k1_side_kernel<<<num_sms * 4, 64, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace spoly
