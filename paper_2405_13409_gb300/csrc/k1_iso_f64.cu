// Isolation kernel, plain FP64: every step of the univariate phase in FP64.
#include "k1_iso.cuh"

namespace spoly {

cudaError_t launch_k1_isolate_f64(const K1Params& P, int grid, int block, int width, cudaStream_t st) {
  k1_isolate_kernel<double><<<grid, block, 0, st>>>(P, width);
  return cudaGetLastError();
}

}  // namespace spoly
