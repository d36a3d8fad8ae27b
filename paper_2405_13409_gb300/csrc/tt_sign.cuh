// TT chains, sign phase: the sign of the Bezout determinant at the
// n_intervals + 1 uniform samples of v1 in [0, 1], bisection of every sign
// change for the paper's 10 iterations (Sec. 4.2), the ill-conditioning
// flag, and the bracket queue.  One block per system; each sample is
// evaluated by a group of G lanes (tt_group.cuh) with the matrix padded to N.
// Instantiated for FP32 (mixed mode) in tt_sign_f32.cu and for FP64 (plain
// mode and the FP64 re-sampling pass) in tt_sign_f64.cu.
#pragma once
#include "tt_group.cuh"

namespace spoly {

constexpr int kSignThreads = 128;
constexpr int kMaxBrackets = 128;  // per system: more re-samples the system in FP64 (FP32), or overflows (FP64)

// FP32 sign changes above which a system's FP32 signs count as noise and it
// is sampled again in FP64: one per 32 intervals (128 at 4096 intervals),
// at least 16.  Re-sampling in FP64 is exact, so the limit moves work
// between the passes and never drops a root.
SPOLY_HD constexpr int noisy_limit(int n_intervals) {
  return n_intervals / 32 > kMaxBrackets ? kMaxBrackets : (n_intervals / 32 < 16 ? 16 : n_intervals / 32);
}
static_assert(noisy_limit(4096) == kMaxBrackets && noisy_limit(100) == 16, "noise limits");
constexpr int kMaxSamples = kTTSampleSlots;  // n_intervals <= 8192

// The block stages the scaled FP64 coefficients of system i of the batch
// (u = 2^ks w) in `coef`, graded layout: a then b.
SPOLY_D void tt_stage_coef64(const TTParams& P, int64_t i, const TTSys& sy, double* coef) {
  const double* sc = P.scratch + i * kTTKeep;
  for (int k = threadIdx.x; k < kTT32; k += blockDim.x) {
    const bool in_a = k < bsize(kTTDa);
    const int idx = in_a ? k : k - bsize(kTTDa);
    int row, col;  // u-power of the graded index
    flat_to_ij(in_a ? kTTDa : kTTDb, idx, row, col);
    coef[k] = ldexp(sc[(in_a ? kOffA : kOffB) + idx], sy.ks * row);
  }
}

template <typename T>
struct SignSmem {
  T coef[kTT32];
  int8_t sgn[kMaxSamples];
  float lg[kMaxSamples];
  T blo[kMaxBrackets], bhi[kMaxBrackets];
  int8_t bs[kMaxBrackets];
  int bm[kMaxBrackets];  // sample index of the bracket's left end
  uint32_t bfl[kMaxBrackets];
  float wmax[kSignThreads / 32];
  int nb;
  float lmax;
  int base;
  int span_lo, span_hi;  // samples to evaluate
  long long slot;
};

template <typename T, int N, int G>
SPOLY_D int sign_g(const SignSmem<T>& S, T v, const TTSys& sy, int g, float* l2) {
  const GroupSign r = tt_group_sign<T, N, G>(S.coef, S.coef + bsize(kTTDa), v, sy.da, sy.db, sy.n, g);
  *l2 = r.log2;
  return r.sign;
}

template <typename T, int N, int G>
SPOLY_D void sign_system(SignSmem<T>& S, const TTParams& P, int64_t i, TTSys& sy) {
  constexpr int kGroups = kSignThreads / G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gi = tid / G, g = tid % G;
  const int NI = P.n_intervals;
  const T dv = T(1) / T(NI);
  if (tid == 0) {
    S.span_lo = 0;
    S.span_hi = NI;
  }
  __syncthreads();
  if (P.resample_only && sy.noisy > 0 && sy.noisy <= P.noisy_cap) {
    // FP64 re-sampling: tt_resample_chunk_kernel has evaluated the stretch
    // where the FP32 signs changed; the kept FP32 signs stand elsewhere
    const int64_t base = int64_t(sy.noisy - 1) * kTTSampleSlots;
    for (int m = tid; m <= NI; m += kSignThreads) {
      S.sgn[m] = P.noisy_sgn[base + m];
      S.lg[m] = P.noisy_lg[base + m];
    }
    if (tid == 0) {
      S.span_lo = 1;
      S.span_hi = 0;
    }
    __syncthreads();
  } else if (P.resample_only && tid == 0) {
    atomicAdd(P.counters + TT_FP64_SAMPLES, (unsigned long long)(NI + 1));
  }
  const int m_lo = S.span_lo, m_hi = S.span_hi;
  // samples: the whole block steps together, so every warp stays converged
#pragma unroll 1
  for (int m0 = m_lo; m0 <= m_hi; m0 += kGroups) {
    const int m = m0 + gi;
    float l2;
    const int s = sign_g<T, N, G>(S, T(min(m, m_hi)) * dv, sy, g, &l2);
    if (m <= m_hi && g == 0) {
      S.sgn[m] = int8_t(s);
      S.lg[m] = l2;
    }
  }
  __syncthreads();
  // largest log2 |det| over the samples, and the sign changes
  float lm = -1e30f;
  for (int m = tid; m <= NI; m += kSignThreads)
    if (S.sgn[m] != 0) lm = fmaxf(lm, S.lg[m]);
  for (int o = 16; o > 0; o >>= 1) lm = fmaxf(lm, __shfl_xor_sync(kGroupFull, lm, o));
  if (lane == 0) S.wmax[warp] = lm;
  if (tid == 0) S.nb = 0;
  __syncthreads();
  if (tid == 0) {
    float x = S.wmax[0];
    for (int w = 1; w < kSignThreads / 32; ++w) x = fmaxf(x, S.wmax[w]);
    S.lmax = x;
  }
  for (int m = tid; m < NI; m += kSignThreads) {
    const int s0 = S.sgn[m], s1 = S.sgn[m + 1];
    T lo = T(0), hi = T(0);
    bool br = false;
    if (s1 == 0) {  // an exact zero at a sample belongs to the interval on its left
      lo = hi = T(m + 1) * dv;
      br = true;
    } else if (s0 != 0 && s0 != s1) {
      lo = T(m) * dv;
      hi = T(m + 1) * dv;
      br = true;
    }
    if (br) {
      const int k = atomicAdd(&S.nb, 1);
      if (k < kMaxBrackets) {
        S.blo[k] = lo;
        S.bhi[k] = hi;
        S.bs[k] = int8_t(s0);
        S.bfl[k] = 0u;
        S.bm[k] = m;
      }
    }
  }
  __syncthreads();
  if (sizeof(T) == 4 && S.nb > noisy_limit(NI)) {
    // FP32 rounding noise in a near-singular stretch of v: the system is
    // sampled again in FP64 (re-sampling pass), which keeps these signs
    // outside the stretch
    if (tid == 0) {
      atomicAdd(P.counters + TT_RESAMPLED, 1ull);
      atomicAdd(P.counters + TT_EVALS, (unsigned long long)(NI + 1));
      atomicAdd(P.counters + TT_EVAL_N3, (unsigned long long)(NI + 1) * (unsigned long long)(sy.n * sy.n * sy.n));
      atomicAdd(P.counters + TT_EVALS32, (unsigned long long)(NI + 1));
      atomicAdd(P.counters + TT_EVAL32_N3, (unsigned long long)(NI + 1) * (unsigned long long)(sy.n * sy.n * sy.n));
      S.slot = (long long)atomicAdd(P.counters + TT_NOISY, 1ull);
      S.span_lo = NI + 1;
      S.span_hi = -1;
    }
    __syncthreads();
    const long long slot = S.slot;
    if (slot < P.noisy_cap) {
      const int64_t base = int64_t(slot) * kTTSampleSlots;
      int lo = NI + 1, hi = -1;
      for (int m = tid; m <= NI; m += kSignThreads) {
        P.noisy_sgn[base + m] = S.sgn[m];
        P.noisy_lg[base + m] = S.lg[m];
        if (m < NI && (S.sgn[m + 1] == 0 || S.sgn[m] == 0 || S.sgn[m] != S.sgn[m + 1])) {
          lo = min(lo, m);
          hi = max(hi, m + 1);
        }
      }
      atomicMin(&S.span_lo, lo);
      atomicMax(&S.span_hi, hi);
      __syncthreads();
      // the stretch where the FP32 signs changed, widened by kTTNoisyMargin
      // samples on each side, is evaluated again in FP64
      if (tid == 0) {
        P.noisy_span[3 * slot] = int32_t(i);
        P.noisy_span[3 * slot + 1] = max(0, S.span_lo - kTTNoisyMargin);
        P.noisy_span[3 * slot + 2] = min(NI, S.span_hi + kTTNoisyMargin);
      }
    }
    if (tid == 0) {
      sy.first_item = 0;
      sy.n_items = 0;
      sy.flags |= kTTResample;
      sy.noisy = slot < P.noisy_cap ? int32_t(slot + 1) : 0;
      P.sys[P.sys_offset + i] = sy;
    }
    return;
  }
  const int nb = min(S.nb, kMaxBrackets);
  if (tid == 0 && S.nb > kMaxBrackets) atomicAdd(P.counters + TT_BRACKET_OVERFLOW, 1ull);
  // bisection, one bracket per group at a time (block-uniform trip counts);
  // brackets fill the lowest groups, and a warp without one skips the round
  // (the evaluation synchronises within the warp only)
  for (int k0 = 0; k0 < nb; k0 += kGroups) {
    const int k = k0 + gi;
    const bool valid = k < nb;
    if (!__any_sync(kGroupFull, valid)) continue;
    T lo = valid ? S.blo[k] : T(0), hi = valid ? S.bhi[k] : T(1);
    const int slo = valid ? S.bs[k] : 1;
    bool active = valid && lo < hi;
    const bool bisect = active;
    float la = 0.0f, lb = 0.0f;
    // the paper's bisection steps, then |det| at both ends (one call site)
#pragma unroll 1
    for (int it = 0; it < kTTPaperIters + 2; ++it) {
      const T x = it < kTTPaperIters ? T(0.5) * (lo + hi) : (it == kTTPaperIters ? lo : hi);
      float l2;
      const int s = sign_g<T, N, G>(S, x, sy, g, &l2);
      if (it == kTTPaperIters) la = l2;
      if (it == kTTPaperIters + 1) lb = l2;
      if (active && it < kTTPaperIters) {
        if (s == 0) {
          lo = hi = x;
          active = false;
        } else if (s == slo) {
          lo = x;
        } else {
          hi = x;
        }
      }
    }
    if (bisect && lo < hi) {
      // ill-conditioning (k = 2): |det| at the bracket ends against the
      // largest |det| of the five samples around the bracket
      float lloc = -1e30f;
      for (int o = -2; o <= 3; ++o) {
        const int mm = min(max(S.bm[k] + o, 0), NI);
        if (S.sgn[mm] != 0) lloc = fmaxf(lloc, S.lg[mm]);
      }
      const float top = fmaxf(la, lb) - lloc;
      const float rel = top + log2f(1.0f + exp2f(fminf(la, lb) - fmaxf(la, lb)));
      if (g == 0 && rel < log2f(float(kTTIllCond))) S.bfl[k] = SPOLY_FLAG_ILL_COND;
    }
    if (valid && g == 0) {
      S.blo[k] = lo;
      S.bhi[k] = hi;
    }
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long ev = (unsigned long long)(m_hi >= m_lo ? m_hi - m_lo + 1 : 0);
    for (int k = 0; k < nb; ++k) ev += (S.blo[k] < S.bhi[k]) ? kTTPaperIters + 2 : 0;
    atomicAdd(P.counters + TT_EVALS, ev);
    atomicAdd(P.counters + TT_EVAL_N3, ev * (unsigned long long)(sy.n * sy.n * sy.n));
    if (sizeof(T) == 4) {
      atomicAdd(P.counters + TT_EVALS32, ev);
      atomicAdd(P.counters + TT_EVAL32_N3, ev * (unsigned long long)(sy.n * sy.n * sy.n));
    }
    S.base = int(atomicAdd(P.counters + TT_BRACKETS, (unsigned long long)nb));
    sy.first_item = S.base;
    sy.n_items = nb;
    P.sys[P.sys_offset + i] = sy;
  }
  __syncthreads();
  for (int k = tid; k < nb; k += kSignThreads) {
    const int64_t slot = int64_t(S.base) + k;
    if (slot < P.queue_cap) {
      RootItem it{};
      it.zlo = S.blo[k];
      it.zhi = S.bhi[k];
      it.chain = int32_t(P.sys_offset + i);
      it.flags = S.bfl[k];
      P.queue[slot] = it;
    }
  }
}

// One kernel per padded size N (group width G), over the systems with
// n_lo < n <= N, so that each size class runs at its own register count.
// The class with n_lo = 0 also records the degenerate and oversized systems.
template <typename T, int N, int G>
__global__ void __launch_bounds__(kSignThreads) tt_sign_kernel(TTParams P, int n_lo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SignSmem<T>& S = *reinterpret_cast<SignSmem<T>*>(smem_raw);
  const int64_t n_sys = tt_n_sys(P);
  for (int64_t i = blockIdx.x; i < n_sys; i += gridDim.x) {
    TTSys sy = P.sys[P.sys_offset + i];
    if (P.resample_only) {
      if (!(sy.flags & kTTResample)) continue;
      sy.flags &= ~kTTResample;
    }
    if (sy.n < 1 || sy.n > kTTMaxN - 1) {
      if (n_lo == 0 && threadIdx.x == 0) {
        atomicAdd(P.counters + (sy.n < 1 ? TT_DEGENERATE : TT_TOO_LARGE), 1ull);
        sy.first_item = 0;
        sy.n_items = 0;
        P.sys[P.sys_offset + i] = sy;
      }
      continue;
    }
    if (sy.n <= n_lo || sy.n > N) continue;
    if constexpr (sizeof(T) == 4) {
      for (int k = threadIdx.x; k < kTT32; k += blockDim.x) S.coef[k] = T(P.coef32[i * kTT32 + k]);
    } else {
      tt_stage_coef64(P, i, sy, S.coef);
    }
    __syncthreads();
    sign_system<T, N, G>(S, P, i, sy);
    __syncthreads();
  }
}

template <typename T, int N, int G>
cudaError_t launch_sign_class(const TTParams& P, int n_lo, int num_sms, cudaStream_t st) {
  const size_t smem = sizeof(SignSmem<T>);
  static bool attr = false;
  static int per_sm = 1;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(tt_sign_kernel<T, N, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tt_sign_kernel<T, N, G>, kSignThreads, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    attr = true;
  }
  const int64_t g = std::min<int64_t>(P.n_sys, int64_t(num_sms) * per_sm);
  tt_sign_kernel<T, N, G><<<int(g), kSignThreads, smem, st>>>(P, n_lo);
  return cudaGetLastError();
}

// -------------------------------------------------- FP64 re-sampling
// The stretches kept by the FP32 pass, in chunks of kResampleChunk samples:
// one block per (slot, chunk) item, items interleaved across slots so that
// long stretches spread over the grid; the FP64 signs and log2 |det|
// overwrite the kept FP32 values.  The sign kernel's re-sampling pass then
// scans and bisects the merged samples.
constexpr int kResampleChunk = 128;
constexpr int kResampleChunks = (kTTSampleSlots + kResampleChunk - 1) / kResampleChunk;

template <int N, int G>
__global__ void __launch_bounds__(kSignThreads) tt_resample_chunk_kernel(TTParams P, int n_lo) {
  __shared__ double coef[kTT32];
  constexpr int kGroups = kSignThreads / G;
  const int tid = threadIdx.x, gi = tid / G, g = tid % G;
  const unsigned long long taken = *(volatile unsigned long long*)(P.counters + TT_NOISY);
  const int64_t n_noisy = taken < (unsigned long long)P.noisy_cap ? int64_t(taken) : P.noisy_cap;
  const double dv = 1.0 / P.n_intervals;
  for (int64_t item = blockIdx.x; item < n_noisy * kResampleChunks; item += gridDim.x) {
    const int64_t slot = item % n_noisy;
    const int c = int(item / n_noisy);
    const int32_t i = P.noisy_span[3 * slot], lo = P.noisy_span[3 * slot + 1], hi = P.noisy_span[3 * slot + 2];
    const int m0 = lo + c * kResampleChunk;
    if (m0 > hi) continue;
    const TTSys sy = P.sys[P.sys_offset + i];
    if (sy.n <= n_lo || sy.n > N) continue;
    tt_stage_coef64(P, i, sy, coef);
    __syncthreads();
    const int m1 = min(hi, m0 + kResampleChunk - 1);
    const int64_t base = slot * kTTSampleSlots;
#pragma unroll 1
    for (int mm = m0; mm <= m1; mm += kGroups) {
      const int m = mm + gi;
      const GroupSign r =
          tt_group_sign<double, N, G>(coef, coef + bsize(kTTDa), double(min(m, m1)) * dv, sy.da, sy.db, sy.n, g);
      if (m <= m1 && g == 0) {
        P.noisy_sgn[base + m] = int8_t(r.sign);
        P.noisy_lg[base + m] = r.log2;
      }
    }
    if (tid == 0) {
      const unsigned long long k = (unsigned long long)(m1 - m0 + 1);
      atomicAdd(P.counters + TT_FP64_SAMPLES, k);
      atomicAdd(P.counters + TT_EVALS, k);
      atomicAdd(P.counters + TT_EVAL_N3, k * (unsigned long long)(sy.n * sy.n * sy.n));
    }
    __syncthreads();
  }
}

template <int N, int G>
cudaError_t launch_resample_class(const TTParams& P, int n_lo, int num_sms, cudaStream_t st) {
  static int per_sm = 0;
  if (per_sm == 0) {
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tt_resample_chunk_kernel<N, G>, kSignThreads, 0);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
  }
  tt_resample_chunk_kernel<N, G><<<num_sms * per_sm, kSignThreads, 0, st>>>(P, n_lo);
  return cudaGetLastError();
}

// ------------------------------------------------------------ FP64 polish
// Every FP32 bracket of a system is polished by bisection of the FP64
// determinant to kTTRootTol, one group per bracket.  Work items are (system,
// chunk of one block's worth of brackets), interleaved across systems so
// that systems with many brackets spread over the grid; each item stages
// its system's coefficients.  Loops run in warp-uniform steps (a warp leaves
// a loop when none of its groups needs another step).  A bracket whose FP64
// signs agree is widened once, to one sample interval on each side of its
// centre; if the signs still agree it is lost.
constexpr int kPolishWiden = 1;
constexpr int kPolishMaxSteps = 40;  // bisection steps from one sample interval to kTTRootTol: 23

// Polish of the brackets of one size class, packed: the groups of a warp take
// consecutive queue slots, whichever systems they belong to (a system has
// one or two brackets as a rule, and the slots of a size class are written
// in runs by its sign kernel).  A group reads its system's FP64 coefficients
// from the system's scratch row (through L1), scaling row i by 2^(ks i) after
// Horner, which gives the same values as the scaled copy the sign kernels
// stage.  Loops run in warp-uniform steps (every group calls the evaluation;
// a group with nothing to do evaluates a fixed point of the batch's first
// system).
template <int N, int G>
__global__ void __launch_bounds__(kSignThreads) tt_polish_kernel(TTParams P, int n_lo) {
  constexpr int kWarps = kSignThreads / 32;
  constexpr int kGroups = 32 / G;
  const int lane = threadIdx.x & 31, gi = lane / G, g = lane % G;
  const double reach = 1.0 / P.n_intervals;
  const unsigned long long nb = P.counters[TT_BRACKETS];
  const int64_t nq = int64_t(nb) < P.queue_cap ? int64_t(nb) : P.queue_cap;
  const int64_t stride = int64_t(gridDim.x) * kWarps * kGroups;
  for (int64_t base = (int64_t(blockIdx.x) * kWarps + (threadIdx.x >> 5)) * kGroups; base < nq; base += stride) {
    const int64_t q = base + gi;
    RootItem item{};
    TTSys sy{};
    bool valid = q < nq;
    if (valid) {
      item = P.queue[q];
      const int64_t si = int64_t(item.chain) - P.sys_offset;
      valid = si >= 0 && si < P.n_sys;
      if (valid) {
        sy = P.sys[item.chain];
        valid = sy.n > n_lo && sy.n <= N;
      }
    }
    if (!__any_sync(kGroupFull, valid)) continue;
    const double* coef = valid ? P.scratch + (int64_t(item.chain) - P.sys_offset) * kTTKeep : P.scratch;
    const int da = valid ? sy.da : 0, db = valid ? sy.db : 0, n = valid ? sy.n : 1, ks = valid ? sy.ks : 0;
    auto ev = [&](double x) { return tt_group_sign<double, N, G>(coef, coef + bsize(kTTDa), x, da, db, n, g, ks).sign; };
    double lo = valid ? item.zlo : 0.0, hi = valid ? item.zhi : 1.0;
    const bool act = valid && lo < hi;  // lo == hi: a root exactly at a sample, kept
    bool ok = true;
    int slo = ev(lo), shi = ev(hi);
    double w = hi - lo;
#pragma unroll 1
    for (int d = 0; d < kPolishWiden; ++d) {
      const bool need = act && slo != 0 && shi != 0 && slo == shi && w < reach;
      if (!__any_sync(kGroupFull, need)) break;
      const double c = 0.5 * (lo + hi);
      const double l2 = fmax(0.0, c - reach), h2 = fmin(1.0, c + reach);
      const int s1 = ev(need ? l2 : lo), s2 = ev(need ? h2 : hi);
      if (need) {
        w = reach;
        lo = l2;
        hi = h2;
        slo = s1;
        shi = s2;
      }
    }
    bool bis = false;
    if (act) {
      if (slo == 0) {
        hi = lo;
      } else if (shi == 0) {
        lo = hi;
      } else if (slo == shi) {
        ok = false;
      } else {
        bis = true;
      }
    }
#pragma unroll 1
    for (int it = 0; it < kPolishMaxSteps; ++it) {
      const double mid = 0.5 * (lo + hi);
      const bool need = bis && hi - lo > kTTRootTol && mid > lo && mid < hi;
      if (!__any_sync(kGroupFull, need)) break;
      const int sgn = ev(need ? mid : lo);
      if (need) {
        if (sgn == 0) {
          lo = hi = mid;
          bis = false;
        } else if (sgn == slo) {
          lo = mid;
        } else {
          hi = mid;
        }
      }
    }
    if (valid && g == 0) {
      if (ok) {
        item.zlo = item.zhi = 0.5 * (lo + hi);
        item.flags |= kTTValid;
      } else {
        atomicAdd(P.counters + TT_POLISH_LOST, 1ull);
      }
      P.queue[q] = item;
    }
  }
}

template <int N, int G>
cudaError_t launch_polish_class(const TTParams& P, int n_lo, int num_sms, cudaStream_t st) {
  static int per_sm = 0;
  if (per_sm == 0) {
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tt_polish_kernel<N, G>, kSignThreads, 0);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
  }
  // the bracket count is on the device: a full grid strides over the queue
  tt_polish_kernel<N, G><<<num_sms * per_sm, kSignThreads, 0, st>>>(P, n_lo);
  return cudaGetLastError();
}

// Padded sizes and group widths per arithmetic type: about 4 rows of
// registers per lane (FP64 rows take twice the registers).
template <typename T>
cudaError_t launch_sign_t(const TTParams& P, int num_sms, cudaStream_t st) {
  cudaError_t e;
  if constexpr (sizeof(T) == 4) {
    if ((e = launch_sign_class<T, 8, 2>(P, 0, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_sign_class<T, 12, 4>(P, 8, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_sign_class<T, 16, 4>(P, 12, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_sign_class<T, 20, 4>(P, 16, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_sign_class<T, 24, 8>(P, 20, num_sms, st)) != cudaSuccess) return e;
    return launch_sign_class<T, 32, 8>(P, 24, num_sms, st);
  } else {
    if ((e = launch_sign_class<T, 8, 2>(P, 0, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_sign_class<T, 12, 4>(P, 8, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_sign_class<T, 16, 4>(P, 12, num_sms, st)) != cudaSuccess) return e;
    if ((e = launch_sign_class<T, 24, 8>(P, 16, num_sms, st)) != cudaSuccess) return e;
    return launch_sign_class<T, 32, 16>(P, 24, num_sms, st);
  }
}

}  // namespace spoly
