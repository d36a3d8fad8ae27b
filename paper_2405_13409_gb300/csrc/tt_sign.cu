// TT chains, FP32 phase: the sign of the Bezout determinant at the 2^12 + 1
// uniform samples of v1 in [0, 1], bisection of every sign change for the
// paper's 10 iterations (Sec. 5.2), and the bracket queue.
#include "tt_det.cuh"

namespace spoly {

constexpr int kSignWarps = 4;
constexpr int kMaxBrackets = 128;  // per system: more re-samples the system in FP64 (FP32), or overflows (FP64)
constexpr int kMaxSamples = 8193;  // n_intervals <= 8192

template <typename T>
struct SignSmem {
  T coef[kTT32];
  T sa[kSignWarps][32], sb[kSignWarps][32];
  int8_t sgn[kMaxSamples];
  float lg[kMaxSamples];
  T blo[kMaxBrackets], bhi[kMaxBrackets];
  int8_t bs[kMaxBrackets];
  int bm[kMaxBrackets];  // sample index of the bracket's left end
  uint32_t bfl[kMaxBrackets];
  float wmax[kSignWarps];
  int nb;
  float lmax;
  int base;
};

template <typename T, int N>
SPOLY_D int sign_t(SignSmem<T>& S, T v, const TTSys& sy, int warp, int lane, float* l2) {
  auto ca = [&](int i, int j) { return S.coef[bidx(kTTDa, i, j)]; };
  auto cb = [&](int i, int j) { return S.coef[bsize(kTTDa) + bidx(kTTDb, i, j)]; };
  return tt_sign_at<T, N>(v, sy.da, sy.db, sy.n, lane, ca, cb, S.sa[warp], S.sb[warp], l2);
}

template <typename T, int N>
SPOLY_D void sign_system(SignSmem<T>& S, const TTParams& P, int64_t i, TTSys& sy) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NI = P.n_intervals;
  const T dv = T(1) / T(NI);
  for (int m = warp; m <= NI; m += kSignWarps) {
    float l2;
    const int s = sign_t<T, N>(S, T(m) * dv, sy, warp, lane, &l2);
    if (lane == 0) {
      S.sgn[m] = int8_t(s);
      S.lg[m] = l2;
    }
  }
  __syncthreads();
  // largest log2 |det| over the samples, and the sign changes
  float lm = -1e30f;
  for (int m = tid; m <= NI; m += blockDim.x)
    if (S.sgn[m] != 0) lm = fmaxf(lm, S.lg[m]);
  for (int o = 16; o > 0; o >>= 1) lm = fmaxf(lm, __shfl_xor_sync(kFull, lm, o));
  if (lane == 0) S.wmax[warp] = lm;
  if (tid == 0) S.nb = 0;
  __syncthreads();
  if (tid == 0) {
    float x = S.wmax[0];
    for (int w = 1; w < kSignWarps; ++w) x = fmaxf(x, S.wmax[w]);
    S.lmax = x;
  }
  for (int m = tid; m < NI; m += blockDim.x) {
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
  if (sizeof(T) == 4 && S.nb > kMaxBrackets) {
    // FP32 rounding noise in a near-singular stretch of v: the system is
    // sampled again in FP64 (resample pass)
    if (tid == 0) {
      atomicAdd(P.counters + TT_RESAMPLED, 1ull);
      sy.first_item = 0;
      sy.n_items = 0;
      sy.flags |= kTTResample;
      P.sys[P.sys_offset + i] = sy;
    }
    return;
  }
  const int nb = min(S.nb, kMaxBrackets);
  if (tid == 0 && S.nb > kMaxBrackets) atomicAdd(P.counters + TT_BRACKET_OVERFLOW, 1ull);
  // bisection, one bracket per warp at a time
  for (int k = warp; k < nb; k += kSignWarps) {
    T lo = S.blo[k], hi = S.bhi[k];
    const int slo = S.bs[k];
    if (lo < hi) {
      for (int it = 0; it < kTTPaperIters; ++it) {
        const T mid = T(0.5) * (lo + hi);
        float l2;
        const int s = sign_t<T, N>(S, mid, sy, warp, lane, &l2);
        if (s == 0) {
          lo = hi = mid;
          break;
        }
        if (s == slo)
          lo = mid;
        else
          hi = mid;
      }
      if (lo < hi) {
        float la, lb;
        sign_t<T, N>(S, lo, sy, warp, lane, &la);
        sign_t<T, N>(S, hi, sy, warp, lane, &lb);
        // reading 7 (k = 2), normalised by the largest |det| of the five
        // samples around the bracket
        float lloc = -1e30f;
        for (int o = -2; o <= 3; ++o) {
          const int mm = min(max(S.bm[k] + o, 0), NI);
          if (S.sgn[mm] != 0) lloc = fmaxf(lloc, S.lg[mm]);
        }
        const float top = fmaxf(la, lb) - lloc;
        const float rel = top + log2f(1.0f + exp2f(fminf(la, lb) - fmaxf(la, lb)));
        if (lane == 0 && rel < log2f(float(kTTIllCond))) S.bfl[k] = SPOLY_FLAG_ILL_COND;
      }
    }
    if (lane == 0) {
      S.blo[k] = lo;
      S.bhi[k] = hi;
    }
  }
  __syncthreads();
  if (tid == 0) {
    unsigned long long ev = (unsigned long long)(NI + 1);
    for (int k = 0; k < nb; ++k) ev += (S.blo[k] < S.bhi[k]) ? kTTPaperIters + 2 : 0;
    atomicAdd(P.counters + TT_EVALS, ev);
    atomicAdd(P.counters + TT_EVAL_N3, ev * (unsigned long long)(sy.n * sy.n * sy.n));
    S.base = int(atomicAdd(P.counters + TT_BRACKETS, (unsigned long long)nb));
    sy.first_item = S.base;
    sy.n_items = nb;
    P.sys[P.sys_offset + i] = sy;
  }
  __syncthreads();
  for (int k = tid; k < nb; k += blockDim.x) {
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

template <typename T>
__global__ void __launch_bounds__(128) tt_sign_kernel(TTParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SignSmem<T>& S = *reinterpret_cast<SignSmem<T>*>(smem_raw);
  for (int64_t i = blockIdx.x; i < P.n_sys; i += gridDim.x) {
    TTSys sy = P.sys[P.sys_offset + i];
    if (P.resample_only) {
      if (!(sy.flags & kTTResample)) continue;
      sy.flags &= ~kTTResample;
    }
    if (sy.n < 1 || sy.n > kTTMaxN - 1) {
      if (threadIdx.x == 0) {
        atomicAdd(P.counters + (sy.n < 1 ? TT_DEGENERATE : TT_TOO_LARGE), 1ull);
        sy.first_item = 0;
        sy.n_items = 0;
        P.sys[P.sys_offset + i] = sy;
      }
      continue;
    }
    if (sizeof(T) == 4) {
      for (int k = threadIdx.x; k < kTT32; k += blockDim.x) S.coef[k] = T(P.coef32[int64_t(k) * P.n_sys + i]);
    } else {
      // plain FP64: the scaled FP64 coefficients (u = 2^ks w)
      const double* sc = P.scratch + i;
      for (int k = threadIdx.x; k < kTT32; k += blockDim.x) {
        const bool in_a = k < bsize(kTTDa);
        const int idx = in_a ? k : k - bsize(kTTDa);
        const int D = in_a ? kTTDa : kTTDb;
        int row = 0;  // u-power of the graded index
        while (row < D && bidx(D, row + 1, 0) <= idx) ++row;
        const double c = sc[int64_t((in_a ? kOffA : kOffB) + idx) * P.n_sys];
        S.coef[k] = T(ldexp(c, sy.ks * row));
      }
    }
    __syncthreads();
    if (sy.n <= 16)
      sign_system<T, 16>(S, P, i, sy);
    else
      sign_system<T, 32>(S, P, i, sy);
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_sign_t(const TTParams& P, int num_sms, cudaStream_t st) {
  const size_t smem = sizeof(SignSmem<T>);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(tt_sign_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int64_t g = std::min<int64_t>(P.n_sys, int64_t(num_sms) * 4);
  tt_sign_kernel<T><<<int(g), kSignWarps * 32, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_tt_sign(const TTParams& P, int num_sms, cudaStream_t st) {
  if (P.n_sys <= 0) return cudaSuccess;
  if (P.n_intervals < 1 || P.n_intervals > kMaxSamples - 1) return cudaErrorInvalidValue;
  return (P.precision == SPOLY_PLAIN_FP64 || P.resample_only) ? launch_sign_t<double>(P, num_sms, st)
                                                              : launch_sign_t<float>(P, num_sms, st);
}

}  // namespace spoly
