// Parameters and launchers of the 2-bounce refraction (TT) kernels.
#pragma once
#include <algorithm>

#include "tt.cuh"

namespace spoly {

// Counter slots of the TT pipeline (its own counter array).
enum TTCounter {
  TT_SYSTEMS = 0,   // (chain, sqrt piece) systems
  TT_DEGENERATE,    // systems whose a or b vanishes, or n < 1
  TT_TOO_LARGE,     // systems with a Bezout size above kTTMaxN (not solved)
  TT_BRACKETS,      // sign changes after the FP32 bisection (queue items)
  TT_BRACKET_OVERFLOW,
  TT_POLISH_LOST,   // brackets without an FP64 sign change nearby
  TT_UROOTS,        // (u1, v1) pairs sent to the path-space Newton
  TT_ADMISSIBLE,    // paths written
  TT_FLAGGED,       // with SPOLY_FLAG_ILL_COND
  TT_RESAMPLED,     // systems whose FP32 signs changed too often, sampled again in FP64
  TT_EVALS,         // Bezout determinant evaluations (samples + bisection steps)
  TT_EVAL_N3,       // sum over evaluations of n^3 (work model of the sign kernel)
  TT_NOISY,         // slots taken in the kept-signs buffer (per batch)
  TT_FP64_SAMPLES,  // samples evaluated again in FP64 by the re-sampling pass
  TT_EVALS32,       // determinant evaluations of the FP32 sign pass
  TT_EVAL32_N3,     // sum of n^3 over them
  TT_COUNT
};
static_assert(TT_COUNT <= 16, "the solution set keeps 16 host copies of the TT counters");

// The 2-bounce chain kinds of the pipeline, from the query's bounce types:
// two refractions (TT) or two reflections (RR); mixed types are not built.
constexpr int kChainTT = 0;
constexpr int kChainRR = 1;
constexpr int kChainOther = -1;
SPOLY_D int chain_kind(const int32_t* types, int q) {
  const int a = types[2 * q], b = types[2 * q + 1];
  if (a == SPOLY_T && b == SPOLY_T) return kChainTT;
  if (a == SPOLY_R && b == SPOLY_R) return kChainRR;
  return kChainOther;
}
constexpr uint32_t kTTResample = 1u << 29;  // TTSys flag: sample again in FP64
constexpr int kTTSampleSlots = 8193;         // samples per system at most (n_intervals <= 8192)
constexpr int kTTNoisyMargin = 8;            // FP64 re-sampling: samples kept beyond the outermost FP32 change
constexpr uint32_t kTTValid = 1u << 30;     // RootItem flag: polished (zlo = zhi = v1)

struct TTParams {
  MeshView mesh;
  QueryView qv;
  const int32_t* chains;   // [n_chains][3] (query, tri0, tri1)
  const int32_t* chain_ids;  // original chain index per chain (NULL: identity)
  int64_t n_chains;
  SqrtTable sqrt_tab;
  int32_t n_intervals;     // uniform samples - 1 over v1 in [0, 1]
  int32_t precision;       // SPOLY_MIXED: FP32 sign sampling; SPOLY_PLAIN_FP64: FP64
  int32_t resample_only;   // sign pass over the systems flagged kTTResample (FP64)
  int32_t* chain_sys;      // [n_chains][2] first system, count
  TTSys* sys;
  int64_t sys_cap;
  int64_t n_sys;           // systems of this batch (build, sign); with n_sys_dev, their bound
  int64_t sys_offset;      // first system of this batch
  // device-driven pass (no host read-backs): the system count on the device
  // (counters[TT_SYSTEMS], written by launch_tt_offsets), else NULL
  const unsigned long long* n_sys_dev;
  double* scratch;         // [n_sys][kTTKeep] FP64: a, b, u~, v~, kappa (batch-local)
  float* coef32;           // [n_sys][kTT32] FP32: scaled, normalised a and b (batch-local)
  RootItem* queue;         // brackets: zlo = zhi = v1 after the polish; chain = system (global index)
  int32_t* active;         // [n_chains] chains of the batch with a polished root (path phase)
  unsigned long long* active_n;  // their count
  int64_t queue_cap;
  unsigned long long* counters;  // [TT_COUNT]
  // FP32 signs and log2 |det| of re-sampled systems ([noisy_cap][kTTSampleSlots]):
  // the FP64 pass evaluates again only the stretch where the FP32 signs changed
  int8_t* noisy_sgn;
  float* noisy_lg;
  int32_t* noisy_span;     // [noisy_cap][3]: batch-local system, first and last sample to evaluate again
  int64_t noisy_cap;
  spoly_path* paths;
  int64_t path_cap;
  unsigned long long* path_counter;  // shared with the 1-bounce paths
};

#ifndef SPOLY_HOST_BUILD
// Systems of the current pass: the host's count, or (device-driven) the
// device's count capped by the host's bound.
SPOLY_D int64_t tt_n_sys(const TTParams& P) {
  if (!P.n_sys_dev) return P.n_sys;
  const unsigned long long n = *(volatile const unsigned long long*)P.n_sys_dev;
  return n < (unsigned long long)P.n_sys ? int64_t(n) : P.n_sys;
}
#endif

// Systems: counts per chain into chain_sys[2c + 1] and piece masks; then,
// with chain_sys[2c] set to the exclusive prefix of the counts, the records.
cudaError_t launch_tt_count(const TTParams& P, uint8_t* masks, int num_sms, cudaStream_t st);
cudaError_t launch_tt_fill(const TTParams& P, const uint8_t* masks, int num_sms, cudaStream_t st);
// Device-driven replacement of the host prefix sum: chain_sys[2c] = the
// exclusive prefix of the counts and counters[TT_SYSTEMS] = their total
// (scan scratch: tmp holds n_chains int32 + n_chains int64 + block sums).
size_t tt_offsets_scratch_bytes(int64_t n_chains);
cudaError_t launch_tt_offsets(const TTParams& P, void* tmp, int num_sms, cudaStream_t st);
// Per batch of systems [sys_offset, sys_offset + n_sys):
cudaError_t launch_tt_build(const TTParams& P, int num_sms, cudaStream_t st);
cudaError_t launch_tt_sign(const TTParams& P, int num_sms, cudaStream_t st);
// FP64 polish of the batch's brackets (after the sign pass).
cudaError_t launch_tt_polish(const TTParams& P, int num_sms, cudaStream_t st);
cudaError_t launch_tt_paths(const TTParams& P, int64_t chain_begin, int64_t chain_end, int num_sms, cudaStream_t st);

}  // namespace spoly
