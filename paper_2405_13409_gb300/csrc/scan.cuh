// Exclusive prefix sums on the device (shared by the footprint builder and
// the visibility grid): blocks of kScanBlock elements scanned with warp
// shuffles, then up to two levels of block sums (n <= 2^30).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace spoly {
namespace scan {

constexpr int kScanBlock = 1024;

// Exclusive scan of int64 (or int32 widened) values, in blocks of kScanBlock.
template <typename In>
static __global__ void scan_block_kernel(const In* in, int64_t* out, int64_t* block_sums, int64_t n) {
  __shared__ int64_t s[kScanBlock / 32];
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  const int64_t v = i < n ? int64_t(in[i]) : 0;
  int64_t x = v;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = s[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s[lane] = w;
  }
  __syncthreads();
  const int64_t incl = x + (warp ? s[warp - 1] : 0);
  if (i < n) out[i] = incl - v;
  if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = incl;
}

static __global__ void scan_add_kernel(int64_t* out, const int64_t* block_off, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  if (i < n) out[i] += block_off[blockIdx.x];
}

// Scratch for exclusive_scan over n elements: sums1 and sums1_off need
// (n / kScanBlock + 1) entries each, sums2 3 * kScanBlock.
template <typename In>
inline cudaError_t exclusive_scan(const In* in, int64_t* out, int64_t n, int64_t* sums1, int64_t* sums1_off,
                                  int64_t* sums2, cudaStream_t st) {
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  scan_block_kernel<In><<<unsigned(nb), kScanBlock, 0, st>>>(in, out, sums1, n);
  if (nb > 1) {
    const int64_t nb2 = (nb + kScanBlock - 1) / kScanBlock;
    scan_block_kernel<int64_t><<<unsigned(nb2), kScanBlock, 0, st>>>(sums1, sums1_off, sums2, nb);
    if (nb2 > 1) {
      int64_t* s2off = sums2 + kScanBlock;
      scan_block_kernel<int64_t><<<1, kScanBlock, 0, st>>>(sums2, s2off, sums2 + 2 * kScanBlock, nb2);
      scan_add_kernel<<<unsigned(nb2), kScanBlock, 0, st>>>(sums1_off, s2off, nb);
    }
    scan_add_kernel<<<unsigned(nb), kScanBlock, 0, st>>>(out, sums1_off, n);
  }
  return cudaGetLastError();
}

}  // namespace scan
}  // namespace spoly
