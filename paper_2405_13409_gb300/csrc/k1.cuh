// Launch parameters and host launchers of the library's kernels.
#pragma once
#include "common.cuh"

namespace spoly {

struct K1Params {
  MeshView mesh;
  QueryView qv;
  const int32_t* chains;  // [n_chains][3] (query, tri0, tri1)
  const int32_t* chain_ids;  // chain index reported in the paths (NULL: position in `chains`)
  int64_t n_chains;
  RootItem* queue;        // bracket queue between isolation and polish
  int64_t queue_cap;
  int32_t* side;          // chains whose Bezout size needs the generic kernel
  int64_t side_cap;
  unsigned long long* counters;  // [C_COUNT]
  spoly_path* paths;
  int64_t path_cap;
  PixelFilter pix;  // optional: keep a path of query q only if x1 projects into pixel q
  int32_t rerun;    // 1: path phase again after a path-buffer overflow (no polish, no isolation counters)
};

#ifndef SPOLY_HOST_BUILD
// Splits a chain list into its 1-bounce (tri1 < 0) and 2-bounce chains, each
// with the original chain indices; counts[0], counts[1] receive the sizes.
cudaError_t launch_partition(const int32_t* chains, int64_t n, int32_t* k1, int32_t* k1_ids, int32_t* k2,
                             int32_t* k2_ids, unsigned long long* counts, int num_sms, cudaStream_t st);
cudaError_t launch_k1_isolate(const K1Params& P, int precision, int num_sms, cudaStream_t st);
// Launch shape of the persistent isolation kernel (block size 32..128, a
// multiple of 32; resident blocks per SM, capped by occupancy; chains per
// ticket, a multiple of 32).  counters[C_TICKET] must start at zero.
struct K1Launch {
  int block = 128;
  int blocks_per_sm = 4;
  int chunk = 64;
};
cudaError_t launch_k1_isolate_persistent(const K1Params& P, int precision, int num_sms, const K1Launch& cfg,
                                         cudaStream_t st);
// After the isolation: the FP64 solve of the side chains (isolation, polish
// and paths in one thread each) and the FP64 polish and path phase of the
// bracket queue.  With side_st, the side chains run on side_st concurrently
// (fork and join through the two events); otherwise both run on st.
cudaError_t launch_k1_finish(const K1Params& P, int num_sms, cudaStream_t st, cudaStream_t side_st, cudaEvent_t fork,
                             cudaEvent_t join);

// Candidate construction.
struct ChainParams {
  MeshView mesh;
  QueryView qv;
  int32_t tri_begin, tri_count;
  double margin;
  int32_t* out;            // [cap][3]
  int64_t cap;
  unsigned long long* count;  // device counter (chains produced)
  int32_t* error;          // device error flag (first bad index + 1)
  float* boxes;            // [n_tris][6] outgoing-direction boxes (shared x0)
  int32_t* shared_x0;      // device flag: all x_first rows equal
};

cudaError_t launch_chains_all(const ChainParams& P, int num_sms, cudaStream_t st);
cudaError_t launch_chains_explicit(const ChainParams& P, const int32_t* src, int64_t n, int num_sms,
                                   cudaStream_t st);
cudaError_t launch_chains_cone(const ChainParams& P, int num_sms, cudaStream_t st);
// Survivors of a validated explicit list under the CONE test of each chain's
// bounce count, appended to P.out (P.count; *k2 counts the 2-bounce ones).
cudaError_t launch_chains_explicit_cone(const ChainParams& P, const int32_t* src, int64_t n, unsigned long long* k2,
                                        int num_sms, cudaStream_t st);

// Cone cull of 2-bounce refraction chains (first triangle in
// [t1_begin, t1_begin + n1), second in [t2_begin, t2_begin + n2)).
struct TTConeParams {
  MeshView mesh;
  QueryView qv;
  int32_t t1_begin, n1, t2_begin, n2;
  double margin;
  float* fwd;                 // [n1][12]
  int32_t* pairs;             // [pair_cap][2] local indices
  int64_t pair_cap;
  unsigned long long* pair_count;
  int32_t* out;               // [cap][3]
  int64_t cap;
  unsigned long long* count;
};
cudaError_t launch_tt_cone_shared(const TTConeParams& P, int32_t* flag, int num_sms, cudaStream_t st, int32_t* host);
cudaError_t launch_tt_cone_pairs(const TTConeParams& P, int num_sms, cudaStream_t st);
cudaError_t launch_tt_cone_chains(const TTConeParams& P, int64_t n_pairs, int num_sms, cudaStream_t st);

// Pixel-footprint builder (footprint.cu).
struct FpGrid {
  double x0, y0, cell;
  int gx, gy;
};
size_t footprint_scratch_bytes(int64_t n_cells, int64_t n_pixels);
// `boxes` ([n_tris] float4: xl, xh, yl, yh) is written by compute_mesh_bounds
// and read by the later stages.
cudaError_t compute_mesh_bounds(const MeshView& M, int* bounds_dev, float* bounds_host, float4* boxes, int num_sms,
                                cudaStream_t st);
cudaError_t fp_grid_count(const MeshView& M, const float4* boxes, const FpGrid& g, void* scratch, int64_t n_pixels,
                          int64_t* n_entries, int num_sms, cudaStream_t st);
cudaError_t fp_grid_fill_and_count(const MeshView& M, const float4* boxes, const FpGrid& g, void* scratch,
                                   int32_t* entries, const double* cam_host, const int* bounds_dev, int64_t n_pixels,
                                   int64_t* total, int num_sms, cudaStream_t st);
// Distinct-triangle footprint in one pass with one read-back: mesh bounds,
// a g x g grid derived on the device, the grid fill (capacity entries_cap;
// counts->n_entries > entries_cap means it must be run again with more),
// the marks of every pixel's candidates, the equality of the queries and the
// distinct triangles as chains (0, t, -1) into out (capacity n_tris).
struct FpUniqueCounts {
  int64_t n_entries, pairs, n_unique;
  bool shared;
};
size_t fp_unique_info_bytes();
cudaError_t fp_unique_build(const MeshView& M, const QueryView& qv, float4* boxes, int* bounds_dev, int g,
                            void* scratch, int64_t n_pixels, int32_t* entries, int64_t entries_cap,
                            const double* cam_host, uint8_t* mark, int32_t* out, void* info_dev,
                            FpUniqueCounts* counts, int num_sms, cudaStream_t st);

cudaError_t fp_fill(const float4* boxes, const FpGrid& g, void* scratch, const int32_t* entries, const double* cam_host,
                    const int* bounds_dev, int64_t n_pixels, int32_t* out, int num_sms, cudaStream_t st);
#endif

}  // namespace spoly
