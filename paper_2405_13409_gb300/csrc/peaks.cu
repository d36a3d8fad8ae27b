// Peak-throughput microbenchmark of the scalar pipes the solver runs on:
// FP32 FFMA and FP64 DFMA, measured on the context's device.  Each thread
// runs 8 independent FMA chains so the pipe, not latency, bounds the loop;
// the grid covers every SM many times over.
#include "common.cuh"

namespace spoly {

template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T* out, int iters, T seed) {
  T a0 = seed + T(threadIdx.x), a1 = a0 + T(1), a2 = a0 + T(2), a3 = a0 + T(3);
  T a4 = a0 + T(4), a5 = a0 + T(5), a6 = a0 + T(6), a7 = a0 + T(7);
  const T m = T(0.999999), c = T(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fma(a0, m, c);
      a1 = fma(a1, m, c);
      a2 = fma(a2, m, c);
      a3 = fma(a3, m, c);
      a4 = fma(a4, m, c);
      a5 = fma(a5, m, c);
      a6 = fma(a6, m, c);
      a7 = fma(a7, m, c);
    }
  }
  const T s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == T(-12345.0)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

// Returns TFLOP/s (2 flop per FMA) of the best of `reps` timed launches.
double measure_fma_peak(int kind, int num_sms, cudaStream_t st, cudaError_t* err) {
  const int block = 256, grid = num_sms * 16;
  const int iters = kind == 0 ? 4096 : 256;
  void* out = nullptr;
  *err = cudaMalloc(&out, size_t(grid) * block * 8);
  if (*err != cudaSuccess) return 0.0;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double best = 0.0;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(a, st);
    if (kind == 0)
      fma_peak_kernel<float><<<grid, block, 0, st>>>(static_cast<float*>(out), iters, 1.0f);
    else
      fma_peak_kernel<double><<<grid, block, 0, st>>>(static_cast<double*>(out), iters, 1.0);
    cudaEventRecord(b, st);
    *err = cudaEventSynchronize(b);
    if (*err != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double flop = 2.0 * 8 * 16 * double(iters) * grid * block;
    if (rep > 0 && ms > 0.f) best = fmax(best, flop / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (*err == cudaSuccess) *err = cudaGetLastError();
  return best;
}

}  // namespace spoly
