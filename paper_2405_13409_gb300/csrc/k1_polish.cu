// FP64 polish and path phase kernel of the 1-bounce solve (Sec. 4.3), plus
// the host launchers of the 1-bounce kernels.
#include <algorithm>

#include "k1_polish.cuh"

namespace spoly {

SPOLY_D int64_t queue_items(const K1Params& P) {
  const unsigned long long queued = *(volatile unsigned long long*)(P.counters + C_QUEUED);
  return int64_t(queued < (unsigned long long)P.queue_cap ? queued : P.queue_cap);
}

// FP64 polish and path phase of every queued candidate.  The items of one
// candidate are contiguous in the queue; the lane on the first item of a run
// polishes the run in place (once: a path re-run finds it polished) and runs
// its path phase, so the candidate's system is built once for both.
// Admissible paths are appended with one atomic per warp.
__global__ void __launch_bounds__(32) k1_finish_kernel(K1Params P, int num_sms) {
  const int64_t n_items = queue_items(P);
  const int lane = threadIdx.x & 31;
  // lanes per warp: enough warps for one per SM sub-partition (a short queue
  // diverges within fewer lanes; FP64 warp instructions cost the same
  // whatever their active lanes)
  const int64_t per = (n_items + 4 * int64_t(num_sms) - 1) / (4 * int64_t(num_sms));
  int width = 1;
  while (width < 32 && width < per) width <<= 1;
  const int64_t n_warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t base = ((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * width; base < n_items;
       base += n_warps * width) {
    const int64_t i = lane < width ? base + lane : n_items;
    spoly_path out[6];
    int np = 0;
    unsigned lost = 0, n_u = 0, n_flag = 0;
    if (i < n_items && (i == 0 || P.queue[i - 1].chain != P.queue[i].chain)) {
      const int chain = P.queue[i].chain;
      int64_t end = i + 1;
      while (end < n_items && P.queue[end].chain == chain) ++end;
      const int q = __ldg(P.chains + 3 * int64_t(chain));
      const int t = __ldg(P.chains + 3 * int64_t(chain) + 1);
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
      if (qd.type == SPOLY_R) {
        K1Sys<4> s;
        const bool ok = k1_system<4>(tr, qd, s);
        k1_chain_solve<4>(s, ok, tr, qd, P.queue + i, int(end - i), q, t, P.pix, lost, n_u, emit);
      } else {
        K1Sys<6> s;
        const bool ok = k1_system<6>(tr, qd, s);
        k1_chain_solve<6>(s, ok, tr, qd, P.queue + i, int(end - i), q, t, P.pix, lost, n_u, emit);
      }
    }
    warp_count(P.counters + C_POLISH_LOST, lost);
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

__global__ void partition_kernel(const int32_t* __restrict__ chains, int64_t n, int32_t* k1, int32_t* k1_ids,
                                 int32_t* k2, int32_t* k2_ids, unsigned long long* counts) {
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < n; base += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = base + threadIdx.x;
    const bool ok = c < n;
    const bool two = ok && chains[3 * c + 2] >= 0;
    const unsigned long long s1 = warp_append(counts, (ok && !two) ? 1u : 0u);
    const unsigned long long s2 = warp_append(counts + 1, two ? 1u : 0u);
    if (!ok) continue;
    int32_t* dst = two ? k2 + 3 * s2 : k1 + 3 * s1;
    dst[0] = chains[3 * c];
    dst[1] = chains[3 * c + 1];
    dst[2] = chains[3 * c + 2];
    (two ? k2_ids[s2] : k1_ids[s1]) = int32_t(c);
  }
}

cudaError_t launch_partition(const int32_t* chains, int64_t n, int32_t* k1, int32_t* k1_ids, int32_t* k2,
                             int32_t* k2_ids, unsigned long long* counts, int num_sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t g = std::min<int64_t>((n + 255) / 256, int64_t(num_sms) * 8);
  partition_kernel<<<int(g), 256, 0, st>>>(chains, n, k1, k1_ids, k2, k2_ids, counts);
  return cudaGetLastError();
}

cudaError_t launch_k1_isolate_f32(const K1Params& P, int grid, int block, int width, cudaStream_t st);
cudaError_t launch_k1_isolate_f64(const K1Params& P, int grid, int block, int width, cudaStream_t st);

// Lanes per warp for n work items: enough warps to give every SM
// sub-partition one (4 per SM), at most 32 lanes.
static int lanes_for(int64_t n, int num_sms) {
  const int64_t per = (n + 4 * int64_t(num_sms) - 1) / (4 * int64_t(num_sms));
  int w = 1;
  while (w < 32 && w < per) w <<= 1;
  return w;
}
cudaError_t launch_k1_side(const K1Params& P, int num_sms, cudaStream_t st);

cudaError_t launch_k1_isolate(const K1Params& P, int precision, int num_sms, cudaStream_t st) {
  // lists too short to give every SM two blocks of 128 run in one-warp
  // blocks, so that their warps spread over all SMs (each chain is one
  // thread's long serial solve)
  const int block = (P.n_chains < int64_t(num_sms) * 256) ? 32 : 128;
  const int width = (block == 32) ? lanes_for(P.n_chains, num_sms) : 32;
  int64_t g = (P.n_chains + int64_t(width) * (block / 32) - 1) / (int64_t(width) * (block / 32));
  if (g < 1) g = 1;
  if (g > int64_t(num_sms) * 16 * (128 / block)) g = int64_t(num_sms) * 16 * (128 / block);
  return (precision == SPOLY_PLAIN_FP64) ? launch_k1_isolate_f64(P, int(g), block, width, st)
                                         : launch_k1_isolate_f32(P, int(g), block, width, st);
}

cudaError_t launch_k1_isolate_persistent_f32(const K1Params& P, int grid, int block, int chunk, cudaStream_t st);
cudaError_t launch_k1_isolate_persistent_f64(const K1Params& P, int grid, int block, int chunk, cudaStream_t st);
int k1_isolate_persistent_f32_blocks_per_sm(int block);
int k1_isolate_persistent_f64_blocks_per_sm(int block);

cudaError_t launch_k1_isolate_persistent(const K1Params& P, int precision, int num_sms, const K1Launch& cfg,
                                         cudaStream_t st) {
  const bool f64 = precision == SPOLY_PLAIN_FP64;
  const int occ = f64 ? k1_isolate_persistent_f64_blocks_per_sm(cfg.block) : k1_isolate_persistent_f32_blocks_per_sm(cfg.block);
  const int bps = std::max(1, std::min(cfg.blocks_per_sm, occ));
  const int grid = num_sms * bps;
  return f64 ? launch_k1_isolate_persistent_f64(P, grid, cfg.block, cfg.chunk, st)
             : launch_k1_isolate_persistent_f32(P, grid, cfg.block, cfg.chunk, st);
}

cudaError_t launch_k1_finish(const K1Params& P, int num_sms, cudaStream_t st, cudaStream_t side_st, cudaEvent_t fork,
                             cudaEvent_t join) {
  cudaError_t e;
  if (side_st) {
    // the side chains' FP64 solve (one warp each, a long serial chain of FP64
    // instructions) overlaps the polish of the main queue
    if ((e = cudaEventRecord(fork, st)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(side_st, fork, 0)) != cudaSuccess) return e;
    if ((e = launch_k1_side(P, num_sms, side_st)) != cudaSuccess) return e;
    if ((e = cudaEventRecord(join, side_st)) != cudaSuccess) return e;
  } else if ((e = launch_k1_side(P, num_sms, st)) != cudaSuccess) {
    return e;
  }
  // one-warp blocks: the few thousand candidates of a step spread evenly over
  // the SMs (each lane runs a long serial chain of FP64 instructions)
  k1_finish_kernel<<<num_sms * 32, 32, 0, st>>>(P, num_sms);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (side_st && (e = cudaStreamWaitEvent(st, join, 0)) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace spoly
