// FP64 instantiations of the TT sign phase (plain mode, and the re-sampling
// pass of systems whose FP32 signs changed too often) and of the FP64 polish.
#include "tt_sign.cuh"

namespace spoly {

cudaError_t launch_tt_sign_f64(const TTParams& P, int num_sms, cudaStream_t st) {
  if (P.resample_only) {
    // the kept stretches first, chunk by chunk; then scans and bisection
    cudaError_t e;
    if ((e = launch_resample_class<8, 2>(P, 0, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_resample_class<12, 4>(P, 8, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_resample_class<16, 4>(P, 12, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_resample_class<24, 8>(P, 16, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_resample_class<32, 16>(P, 24, num_sms, st)) != cudaSuccess) return e;
  }
  return launch_sign_t<double>(P, num_sms, st);
}

// The same size classes as the FP64 sign pass, so the group evaluations are
// shared.
cudaError_t launch_tt_polish(const TTParams& P, int num_sms, cudaStream_t st) {
  if (P.n_sys <= 0) return cudaSuccess;
  cudaError_t e;
  if ((e = launch_polish_class<8, 2>(P, 0, num_sms, st)) != cudaSuccess) return e;
  if ((e = launch_polish_class<12, 4>(P, 8, num_sms, st)) != cudaSuccess) return e;
  if ((e = launch_polish_class<16, 4>(P, 12, num_sms, st)) != cudaSuccess) return e;
  if ((e = launch_polish_class<24, 8>(P, 16, num_sms, st)) != cudaSuccess) return e;
  return launch_polish_class<32, 16>(P, 24, num_sms, st);
}

}  // namespace spoly
