// FP32 instantiation of the TT sign phase (mixed mode) and the launcher
// that picks the precision.
#include "tt_sign.cuh"

namespace spoly {

cudaError_t launch_tt_sign_f64(const TTParams& P, int num_sms, cudaStream_t st);

cudaError_t launch_tt_sign(const TTParams& P, int num_sms, cudaStream_t st) {
  if (P.n_sys <= 0) return cudaSuccess;
  if (P.n_intervals < 1 || P.n_intervals > kMaxSamples - 1) return cudaErrorInvalidValue;
  if (P.precision == SPOLY_PLAIN_FP64 || P.resample_only) return launch_tt_sign_f64(P, num_sms, st);
  return launch_sign_t<float>(P, num_sms, st);
}

}  // namespace spoly
