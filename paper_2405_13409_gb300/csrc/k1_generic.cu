// Side kernel of the 1-bounce solve, FP64 throughout.
//
// Handles the side queue: candidates whose trimmed Bezout size n is not one
// of the sizes the unrolled kernels are instantiated for (flat or degenerate
// triangles, index-matched refraction), which run the same algorithm with
// runtime loops, and candidates whose FP32 isolation was not certified, which
// re-run the unrolled expansion and the isolation in FP64.
#include "k1_generic.cuh"

namespace spoly {

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
    RootItem items[kRD + 1];
    int nq = 0;
    unsigned n_v = 0, n_pref = 0, n_deg = 0;
    if (i < n_side) {
      const int c = P.side[i];
      const int q = __ldg(P.chains + 3 * int64_t(c));
      const int t = __ldg(P.chains + 3 * int64_t(c) + 1);
      const QueryD qd = load_query(P.qv.x_first, P.qv.x_last, P.qv.eta, P.qv.types, q);
      const TriD tr = load_tri(P.mesh.tri, P.mesh.n_tris, t);
      int r = 0;
      if (qd.type == SPOLY_R) {
        K1Sys<4> s;
        if (!k1_system<4>(tr, qd, s)) {
          r = -1;
        } else {
          r = k1_isolate_dispatch<double, 4>(s, items, c, n_v, n_pref);
          if (r == -2) r = k1_generic_one<4>(s, items, c, n_v, n_pref);
        }
      } else {
        K1Sys<6> s;
        if (!k1_system<6>(tr, qd, s)) {
          r = -1;
        } else {
          r = k1_isolate_dispatch<double, 6>(s, items, c, n_v, n_pref);
          if (r == -2) r = k1_generic_one<6>(s, items, c, n_v, n_pref);
        }
      }
      n_deg = (r < 0) ? 1u : 0u;
      nq = r > 0 ? r : 0;
    }
    warp_count(P.counters + C_DEGENERATE, n_deg);
    warp_count(P.counters + C_VROOTS, n_v);
    warp_count(P.counters + C_PREFILTERED, n_pref);
    const unsigned long long slot = warp_append(P.counters + C_QUEUED, unsigned(nq));
    for (int k = 0; k < nq; ++k) {
      const unsigned long long idx = slot + k;
      if (idx < (unsigned long long)P.queue_cap) P.queue[idx] = items[k];
    }
  }
}

cudaError_t launch_k1_generic(const K1Params& P, int num_sms, cudaStream_t st) {
  k1_side_kernel<<<num_sms * 4, 64, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace spoly
