// Launch parameters and host launchers of the library's kernels.
#pragma once
#include "common.cuh"

namespace spoly {

struct K1Params {
  MeshView mesh;
  QueryView qv;
  const int32_t* chains;  // [n_chains][3] (query, tri0, tri1)
  int64_t n_chains;
  RootItem* queue;        // bracket queue between isolation and polish
  int64_t queue_cap;
  int32_t* side;          // chains whose Bezout size needs the generic kernel
  int64_t side_cap;
  unsigned long long* counters;  // [C_COUNT]
  spoly_path* paths;
  int64_t path_cap;
};

#ifndef SPOLY_HOST_BUILD
cudaError_t launch_k1_isolate(const K1Params& P, int precision, int num_sms, cudaStream_t st);
cudaError_t launch_k1_polish(const K1Params& P, int num_sms, cudaStream_t st);
cudaError_t launch_k1_paths(const K1Params& P, int num_sms, cudaStream_t st);

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
#endif

}  // namespace spoly
