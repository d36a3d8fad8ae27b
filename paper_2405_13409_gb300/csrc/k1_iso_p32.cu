// Persistent work-queue isolation kernel (mixed precision).
#include "k1_iso.cuh"

namespace spoly {

cudaError_t launch_k1_isolate_persistent_f32(const K1Params& P, int grid, int block, int chunk, cudaStream_t st) {
  k1_isolate_persistent_kernel<float><<<grid, block, 0, st>>>(P, chunk);
  return cudaGetLastError();
}

int k1_isolate_persistent_f32_blocks_per_sm(int block) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k1_isolate_persistent_kernel<float>, block, 0) != cudaSuccess)
    return 1;
  return b > 0 ? b : 1;
}

}  // namespace spoly
