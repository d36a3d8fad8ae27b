// Host-side state behind the C ABI's opaque handles, shared by the
// translation units that implement the ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

#include "common.cuh"
#include "k1.cuh"

namespace spoly {

// Grow-only device buffer.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n) {
    if (n <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, n);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
};

}  // namespace spoly

// The opaque handle types of the C ABI.
struct spoly_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side_stream = nullptr;  // the library's own: the side chains' FP64 solve
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int num_sms = 0;
  char err[512] = {0};
  spoly::DevBuf mesh, xf, xl, eta, types, kk;  // staged host inputs
  spoly::DevBuf check;                          // first non-finite index of staged inputs
  spoly::DevBuf chain_stage, chain_valid;       // staged and validated explicit chain lists
  spoly::DevBuf vis_grid, vis_entries;          // visibility grid (cells, offsets, z ranges) and entries
  spoly::DevBuf boxes, flag;                    // cone cull scratch
  spoly::DevBuf cam, bounds, fp_scratch, fp_entries, fp_boxes, fp_mark;  // footprint builder
  spoly::DevBuf tt_pairs;                // 2-bounce cone: receiver-independent pairs
  spoly::K1Launch tune;                  // persistent isolation launch shape (spoly_autotune)
};

struct spoly_chains {
  spoly::DevBuf buf;        // [cap][3] int32
  int64_t n = 0;
  int64_t n_k2 = 0;         // chains with a second triangle (tri1 >= 0)
  int64_t n_footprint = 0;  // FOOTPRINT modes: (pixel, triangle) candidate pairs
  spoly::DevBuf counter;    // unsigned long long + int32 error flag
};

struct spoly_solution_set {
  spoly::DevBuf queue;      // RootItem[queue_cap]
  int64_t queue_cap = 0;
  spoly::DevBuf paths;      // spoly_path[path_cap]
  int64_t path_cap = 0;
  spoly::DevBuf side;       // int32[side_cap] chains for the generic-size kernel
  int64_t side_cap = 0;
  spoly::DevBuf counters;   // unsigned long long[C_COUNT]
  unsigned long long host[spoly::C_COUNT] = {0};
  bool host_valid = false;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // phase timing
  cudaEvent_t tt_ev[2] = {nullptr, nullptr};                  // 2-bounce sign pass timing
  float tt_sign_ms = 0.0f;
  bool timed = false;
  // 2-bounce chains: partitioned lists, systems, per-batch scratch
  spoly::DevBuf part, part_n, tt_counters, tt_chain_sys, tt_masks, tt_sys, tt_scratch, tt_coef32, tt_queue, tt_noisy,
      tt_active, tt_offsets;
  unsigned long long tt_host[16] = {0};  // TT_COUNT <= 16
  bool tt_device = false;  // the last 2-bounce pass ran device-driven: tt_host is read from the device
  int64_t n_k2 = 0;
  // captured 1-bounce solve (SPOLY_SOLVE_GRAPH) and the inputs it was captured for
  cudaGraphExec_t gexec = nullptr;
  uint64_t gkey[48] = {0};
};

namespace spoly {

// Records a message on the context and returns `st`.
spoly_status fail(spoly_ctx* ctx, spoly_status st, const char* fmt, ...);
// ENOMEM or ECUDA with the CUDA error string.
spoly_status cuda_fail(spoly_ctx* ctx, cudaError_t e, const char* what);
// Device views of mesh and queries; host arrays are checked for non-finite
// values and staged into the context's buffers.
spoly_status stage_inputs(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q, MeshView* mv,
                          QueryView* qv);

}  // namespace spoly

#define CK(call, what)                                      \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return spoly::cuda_fail(ctx, e_, what); \
  } while (0)
