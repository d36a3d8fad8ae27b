// Isolation kernel, mixed precision: FP32 Laplace expansion and isolation on
// Bezout entries built in FP64.
#include "k1_iso.cuh"

namespace spoly {

cudaError_t launch_k1_isolate_f32(const K1Params& P, int grid, int block, int width, cudaStream_t st) {
  k1_isolate_kernel<float><<<grid, block, 0, st>>>(P, width);
  return cudaGetLastError();
}

}  // namespace spoly
