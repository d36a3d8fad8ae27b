// Training of the gate network on the GPU: BF16 tensor-core matrix products
// with FP32 accumulation for the forward and backward passes, the weighted
// binary cross-entropy head, bias reductions and Adam on the FP32 master
// parameters.  One training step on a batch X [B][32], y [B]:
//
//   Z1 = X W1 + b1,  Z2 = relu(Z1) W2 + b2,  Z3 = relu(Z2) W3 + b3,
//   z4 = relu(Z3) w4 + b4,  L = mean_r w_r (softplus(z4_r) - y_r z4_r)
//   dz4 = w (sigmoid(z4) - y) / B
//   dZ3 = (dz4 w4^T) * [Z3 > 0],   gW3 = relu(Z2)^T dZ3,  gb3 = sum_r dZ3
//   dZ2 = (dZ3 W3^T) * [Z2 > 0],   gW2 = relu(Z1)^T dZ2,  gb2 = sum_r dZ2
//   dZ1 = (dZ2 W2^T) * [Z1 > 0],   gW1 = X^T dZ1,         gb1 = sum_r dZ1
//
// Every matrix-product operand is rounded to BF16 when staged in shared
// memory (the straight-through reading of the BF16 network), so the forward
// pass computes what the inference kernel computes.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mlp.cuh"

namespace spoly {
namespace {

// ------------------------------------------------------------- BF16 GEMM
// C(m, n) = sum_k A(m, k) B(k, n) [+ bias(n)] [* (mask(m, n) > 0)], with
// A(m, k) = A[m sam + k sak] (clamped at 0 when relu_a) and
// B(k, n) = B[k sbk + n sbn].  blockIdx.z splits K into chunks whose partial
// products are added atomically into C (which the caller zeroed).
struct Gemm {
  const float* A;
  int64_t sam, sak;
  const float* B;
  int64_t sbk, sbn;
  float* C;
  int64_t scm, scn;
  int M, N, K, k_chunk;
  const float* bias;
  const float* mask;
  int relu_a, atomic;
};

constexpr int BM = 64, BN = 64, BK = 32, SST = BK + 8;  // SST: padded BF16 row stride

SPOLY_D uint32_t ld_pair(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__global__ void __launch_bounds__(128) gemm_kernel(Gemm g) {
  __shared__ __align__(16) __nv_bfloat16 As[BM * SST];  // [m][k]
  __shared__ __align__(16) __nv_bfloat16 Bs[BN * SST];  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1, gr = lane >> 2, c2 = 2 * (lane & 3);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * g.k_chunk, ke = min(g.K, kb + g.k_chunk);
  float acc[2][4][4] = {};
  const bool a_kfast = g.sak == 1, b_nfast = g.sbn == 1;
  for (int k0 = kb; k0 < ke; k0 += BK) {
    for (int i = tid; i < BM * BK; i += 128) {
      const int mm = a_kfast ? i / BK : i % BM, kk = a_kfast ? i % BK : i / BM;
      const int m = m0 + mm, k = k0 + kk;
      float v = 0.0f;
      if (m < g.M && k < ke) v = g.A[int64_t(m) * g.sam + int64_t(k) * g.sak];
      if (g.relu_a) v = fmaxf(v, 0.0f);
      As[mm * SST + kk] = __float2bfloat16_rn(v);
    }
    for (int i = tid; i < BN * BK; i += 128) {
      const int nn = b_nfast ? i % BN : i / BK, kk = b_nfast ? i / BN : i % BK;
      const int n = n0 + nn, k = k0 + kk;
      float v = 0.0f;
      if (n < g.N && k < ke) v = g.B[int64_t(k) * g.sbk + int64_t(n) * g.sbn];
      Bs[nn * SST + kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
      uint32_t a[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const __nv_bfloat16* p = As + (wm * 32 + mt * 16 + gr) * SST + ks + c2;
        a[mt][0] = ld_pair(p);
        a[mt][1] = ld_pair(p + 8 * SST);
        a[mt][2] = ld_pair(p + 8);
        a[mt][3] = ld_pair(p + 8 * SST + 8);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const __nv_bfloat16* p = Bs + (wn * 32 + nt * 8 + gr) * SST + ks + c2;
        const uint32_t b0 = ld_pair(p), b1 = ld_pair(p + 8);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]), "+f"(acc[mt][nt][3])
              : "r"(a[mt][0]), "r"(a[mt][1]), "r"(a[mt][2]), "r"(a[mt][3]), "r"(b0), "r"(b1));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm * 32 + mt * 16 + gr + (r >= 2 ? 8 : 0);
        const int n = n0 + wn * 32 + nt * 8 + c2 + (r & 1);
        if (m >= g.M || n >= g.N) continue;
        float v = acc[mt][nt][r];
        if (g.bias && blockIdx.z == 0) v += g.bias[n];
        if (g.mask && !(g.mask[int64_t(m) * g.scm + int64_t(n) * g.scn] > 0.0f)) v = 0.0f;
        float* c = g.C + int64_t(m) * g.scm + int64_t(n) * g.scn;
        if (g.atomic)
          atomicAdd(c, v);
        else
          *c = v;
      }
}

cudaError_t gemm(const Gemm& g0, cudaStream_t st) {
  Gemm g = g0;
  int splits = 1;
  if (g.atomic) splits = std::max(1, std::min(64, g.K / 256));
  g.k_chunk = ((g.K + splits - 1) / splits + BK - 1) / BK * BK;
  splits = (g.K + g.k_chunk - 1) / g.k_chunk;
  dim3 grid((g.M + BM - 1) / BM, (g.N + BN - 1) / BN, std::max(splits, 1));
  gemm_kernel<<<grid, 128, 0, st>>>(g);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ head
// One warp per group of rows; lane j holds hidden units j and j + 32.
__global__ void __launch_bounds__(256) head_kernel(const float* __restrict__ Z3, const float* __restrict__ theta,
                                                   const float* __restrict__ y, int B, float pos_weight,
                                                   float* __restrict__ dZ3, float* __restrict__ grad,
                                                   float* __restrict__ loss) {
  const int lane = threadIdx.x & 31;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const float wa = theta[kOffW4 + lane], wb = theta[kOffW4 + lane + 32], b4 = theta[kOffB4];
  const float inv_b = 1.0f / float(B);
  float ga = 0.f, gb = 0.f, gbias = 0.f, lsum = 0.f;
  for (int r = wid; r < B; r += nw) {
    const float za = Z3[int64_t(r) * kHid + lane], zb = Z3[int64_t(r) * kHid + lane + 32];
    const float ha = fmaxf(za, 0.f), hb = fmaxf(zb, 0.f);
    float z = ha * wa + hb * wb;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    z += b4;
    const float yr = y[r];
    const float w = yr > 0.5f ? pos_weight : 1.0f;
    const float sig = 1.0f / (1.0f + expf(-z));
    const float dz = w * (sig - yr) * inv_b;
    dZ3[int64_t(r) * kHid + lane] = za > 0.f ? dz * wa : 0.f;
    dZ3[int64_t(r) * kHid + lane + 32] = zb > 0.f ? dz * wb : 0.f;
    ga += ha * dz;
    gb += hb * dz;
    gbias += dz;
    lsum += w * (fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - yr * z);
  }
  atomicAdd(grad + kOffW4 + lane, ga);
  atomicAdd(grad + kOffW4 + lane + 32, gb);
  if (lane == 0) {
    atomicAdd(grad + kOffB4, gbias);
    atomicAdd(loss, lsum * inv_b);
  }
}

// Column sums of dZ [B][64] added into g[64].
__global__ void __launch_bounds__(256) colsum_kernel(const float* __restrict__ dZ, int B, float* __restrict__ g) {
  __shared__ float part[4][kHid];
  const int c = threadIdx.x & 63, r0 = threadIdx.x >> 6;
  float s = 0.f;
  for (int r = blockIdx.x * 4 + r0; r < B; r += gridDim.x * 4) s += dZ[int64_t(r) * kHid + c];
  part[r0][c] = s;
  __syncthreads();
  if (threadIdx.x < kHid)
    atomicAdd(g + c, part[0][c] + part[1][c] + part[2][c] + part[3][c]);
}

// Adam (Kingma and Ba, Algorithm 1) with bias corrections c1 = 1 / (1 -
// beta1^t), c2 = 1 / (1 - beta2^t).  The padding rows of W1 stay zero.
__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, float lr, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kParams) return;
  if (i >= kOffW1 + kFeat * kHid && i < kOffB1) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

// Index lists of the positive and negative rows: lists[0..n_pos) and
// lists[n - n_neg .. n) (negatives written from the back).
__global__ void split_kernel(const uint8_t* __restrict__ labels, int64_t n, int32_t* __restrict__ lists,
                             unsigned long long* __restrict__ counts) {
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < n; base += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = base + threadIdx.x;
    const bool ok = i < n;
    const bool pos = ok && labels[i] != 0;
    const unsigned long long sp = warp_append(counts, pos ? 1u : 0u);
    const unsigned long long sn = warp_append(counts + 1, (ok && !pos) ? 1u : 0u);
    if (pos) lists[sp] = int32_t(i);
    if (ok && !pos) lists[n - 1 - int64_t(sn)] = int32_t(i);
  }
}

// splitmix64 finaliser as a counter-based generator (Steele, Lea and Flood,
// 2014) for the batch sampler.
SPOLY_D uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Batch row b: a positive for b < n_pos_batch, else a negative, drawn
// uniformly with replacement; or row b itself when lists is NULL.
__global__ void gather_kernel(const float* __restrict__ feat, const uint8_t* __restrict__ labels,
                              const int32_t* __restrict__ lists, int64_t n, int64_t n_pos, int B, int n_pos_batch,
                              uint64_t key, float* __restrict__ xb, float* __restrict__ yb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int64_t row = b;
  if (lists) {
    const uint64_t r = mix64(key ^ (uint64_t(b) * 0xd1b54a32d192ed03ull));
    if (b < n_pos_batch)
      row = lists[r % uint64_t(n_pos)];
    else
      row = lists[n_pos + int64_t(r % uint64_t(n - n_pos))];
  }
  const float* src = feat + row * kFeat;
  float* dst = xb + int64_t(b) * kIn;
#pragma unroll
  for (int j = 0; j < kFeat; ++j) dst[j] = src[j];
#pragma unroll
  for (int j = kFeat; j < kIn; ++j) dst[j] = 0.f;
  yb[b] = labels[row] ? 1.0f : 0.0f;
}

// Forward and backward of one batch already gathered in m->xb / m->yb;
// gradients into m->grad (zeroed here), the batch loss added to *loss_slot.
cudaError_t step_grads(spoly_mlp* m, int B, float pos_weight, float* loss_slot, int num_sms, cudaStream_t st) {
  const float* th = static_cast<const float*>(m->theta.p);
  float* gr = static_cast<float*>(m->grad.p);
  float* X = static_cast<float*>(m->xb.p);
  float* Z1 = static_cast<float*>(m->z1.p);
  float* Z2 = static_cast<float*>(m->z2.p);
  float* Z3 = static_cast<float*>(m->z3.p);
  float* D1 = static_cast<float*>(m->dz1.p);
  float* D2 = static_cast<float*>(m->dz2.p);
  float* D3 = static_cast<float*>(m->dz3.p);
  cudaError_t e = cudaMemsetAsync(gr, 0, kParams * sizeof(float), st);
  if (e != cudaSuccess) return e;
  auto fwd = [&](const float* A, int lda, int K, int relu, int off_w, int off_b, float* C) {
    Gemm g{A, lda, 1, th + off_w, kHid, 1, C, kHid, 1, B, kHid, K, 0, th + off_b, nullptr, relu, 0};
    return gemm(g, st);
  };
  // dW[in][out] += relu?(H)^T D  (H: [B][ldh], D: [B][64])
  auto wgrad = [&](const float* H, int ldh, int K_in, int relu, const float* D, int off_w) {
    Gemm g{H, 1, ldh, D, kHid, 1, gr + off_w, kHid, 1, K_in, kHid, B, 0, nullptr, nullptr, relu, 1};
    return gemm(g, st);
  };
  // Dprev = (D W^T) * [Zprev > 0]  with W [64][64]
  auto dgrad = [&](const float* D, int off_w, const float* Zprev, float* Dprev) {
    Gemm g{D, kHid, 1, th + off_w, 1, kHid, Dprev, kHid, 1, B, kHid, kHid, 0, nullptr, Zprev, 0, 0};
    return gemm(g, st);
  };
  const int cs_grid = std::min(num_sms * 2, (B + 3) / 4);
  if ((e = fwd(X, kIn, kIn, 0, kOffW1, kOffB1, Z1)) != cudaSuccess) return e;
  if ((e = fwd(Z1, kHid, kHid, 1, kOffW2, kOffB2, Z2)) != cudaSuccess) return e;
  if ((e = fwd(Z2, kHid, kHid, 1, kOffW3, kOffB3, Z3)) != cudaSuccess) return e;
  head_kernel<<<std::min(num_sms * 4, (B + 7) / 8), 256, 0, st>>>(Z3, th, static_cast<const float*>(m->yb.p), B,
                                                                    pos_weight, D3, gr, loss_slot);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = wgrad(Z2, kHid, kHid, 1, D3, kOffW3)) != cudaSuccess) return e;
  colsum_kernel<<<cs_grid, 256, 0, st>>>(D3, B, gr + kOffB3);
  if ((e = dgrad(D3, kOffW3, Z2, D2)) != cudaSuccess) return e;
  if ((e = wgrad(Z1, kHid, kHid, 1, D2, kOffW2)) != cudaSuccess) return e;
  colsum_kernel<<<cs_grid, 256, 0, st>>>(D2, B, gr + kOffB2);
  if ((e = dgrad(D2, kOffW2, Z1, D1)) != cudaSuccess) return e;
  if ((e = wgrad(X, kIn, kIn, 0, D1, kOffW1)) != cudaSuccess) return e;
  colsum_kernel<<<cs_grid, 256, 0, st>>>(D1, B, gr + kOffB1);
  return cudaGetLastError();
}

cudaError_t ensure_batch(spoly_mlp* m, int B, int n_loss) {
  cudaError_t e = m->xb.ensure(size_t(B) * kIn * 4);
  if (e == cudaSuccess) e = m->yb.ensure(size_t(B) * 4);
  for (DevBuf* b : {&m->z1, &m->z2, &m->z3, &m->dz1, &m->dz2, &m->dz3})
    if (e == cudaSuccess) e = b->ensure(size_t(B) * kHid * 4);
  if (e == cudaSuccess) e = m->grad.ensure(kParams * 4);
  if (e == cudaSuccess) e = m->loss.ensure(size_t(std::max(n_loss, 1)) * 4);
  return e;
}

}  // namespace
}  // namespace spoly

using namespace spoly;

extern "C" {

spoly_status spoly_mlp_grad(spoly_ctx* ctx, spoly_mlp* m, const float* feat, const uint8_t* labels, int64_t n,
                            float pos_weight, float* grad_host, float* loss_host) {
  if (!ctx) return SPOLY_EINVAL;
  if (!m || !feat || !labels || !grad_host || n <= 0 || n > (1 << 24) || !(pos_weight > 0.0f))
    return fail(ctx, SPOLY_EINVAL, "mlp_grad: bad arguments (0 < n <= 2^24, pos_weight > 0)");
  const int B = int(n);
  CK(ensure_batch(m, B, 1), "mlp_grad scratch");
  float* loss = static_cast<float*>(m->loss.p);
  CK(cudaMemsetAsync(loss, 0, 4, ctx->stream), "mlp_grad");
  gather_kernel<<<(B + 255) / 256, 256, 0, ctx->stream>>>(feat, labels, nullptr, n, 0, B, 0, 0,
                                                          static_cast<float*>(m->xb.p), static_cast<float*>(m->yb.p));
  CK(cudaGetLastError(), "mlp_grad gather");
  CK(step_grads(m, B, pos_weight, loss, ctx->num_sms, ctx->stream), "mlp_grad");
  CK(cudaMemcpyAsync(grad_host, m->grad.p, kParams * 4, cudaMemcpyDeviceToHost, ctx->stream), "mlp_grad copy");
  float l = 0.f;
  CK(cudaMemcpyAsync(&l, loss, 4, cudaMemcpyDeviceToHost, ctx->stream), "mlp_grad copy");
  CK(cudaStreamSynchronize(ctx->stream), "mlp_grad sync");
  if (loss_host) *loss_host = l;
  return SPOLY_OK;
}

spoly_status spoly_mlp_train(spoly_ctx* ctx, spoly_mlp* m, const float* feat, const uint8_t* labels, int64_t n,
                             const spoly_mlp_train_opts* opts, float* final_loss) {
  if (!ctx) return SPOLY_EINVAL;
  if (!m || !feat || !labels || !opts || n <= 0 || n > INT32_MAX)
    return fail(ctx, SPOLY_EINVAL, "mlp_train: bad arguments");
  const spoly_mlp_train_opts o = *opts;
  if (o.steps <= 0 || o.batch < 32 || o.batch > (1 << 20) || !(o.lr > 0.f) || !(o.pos_weight > 0.f) ||
      !(o.pos_fraction > 0.f && o.pos_fraction < 1.f) || o.lr_final < 0.f)
    return fail(ctx, SPOLY_EINVAL, "mlp_train: bad options");
  cudaStream_t st = ctx->stream;
  CK(m->lists.ensure(size_t(n) * 4), "mlp_train lists");
  CK(m->list_n.ensure(16), "mlp_train lists");
  CK(cudaMemsetAsync(m->list_n.p, 0, 16, st), "mlp_train lists");
  {
    const int64_t grid = std::min<int64_t>((n + 255) / 256, int64_t(ctx->num_sms) * 8);
    split_kernel<<<int(grid), 256, 0, st>>>(labels, n, static_cast<int32_t*>(m->lists.p),
                                            static_cast<unsigned long long*>(m->list_n.p));
    CK(cudaGetLastError(), "mlp_train split");
  }
  unsigned long long cnt[2] = {0, 0};
  CK(cudaMemcpyAsync(cnt, m->list_n.p, 16, cudaMemcpyDeviceToHost, st), "mlp_train counts");
  CK(cudaStreamSynchronize(st), "mlp_train counts");
  const int64_t n_pos = int64_t(cnt[0]);
  if (n_pos == 0 || n_pos == n) return fail(ctx, SPOLY_EINVAL, "mlp_train: labels of a single class");
  const int B = o.batch;
  const int n_pos_batch = std::max(1, std::min(B - 1, int(std::lround(double(o.pos_fraction) * B))));
  const int n_tail = int(std::min<int64_t>(o.steps, 64));
  CK(ensure_batch(m, B, n_tail + 1), "mlp_train scratch");
  float* losses = static_cast<float*>(m->loss.p);
  CK(cudaMemsetAsync(losses, 0, size_t(n_tail + 1) * 4, st), "mlp_train");
  float* th = static_cast<float*>(m->theta.p);
  for (int64_t s = 0; s < o.steps; ++s) {
    const uint64_t key = o.seed * 0x9e3779b97f4a7c15ull + uint64_t(m->adam_step + 1);
    gather_kernel<<<(B + 255) / 256, 256, 0, st>>>(feat, labels, static_cast<const int32_t*>(m->lists.p), n, n_pos, B,
                                                   n_pos_batch, key, static_cast<float*>(m->xb.p),
                                                   static_cast<float*>(m->yb.p));
    CK(cudaGetLastError(), "mlp_train gather");
    // The last n_tail steps keep their batch loss; earlier ones add theirs
    // into a slot that is not read back.
    float* slot = losses + (s >= o.steps - n_tail ? s - (o.steps - n_tail) : n_tail);
    CK(step_grads(m, B, o.pos_weight, slot, ctx->num_sms, st), "mlp_train step");
    ++m->adam_step;
    const double t = double(m->adam_step);
    const double frac = double(s) / double(std::max<int64_t>(o.steps - 1, 1));
    const double lr = o.lr_final > 0.f ? o.lr * std::pow(double(o.lr_final) / o.lr, frac) : o.lr;
    adam_kernel<<<(kParams + 255) / 256, 256, 0, st>>>(th, static_cast<float*>(m->adam_m.p),
                                                        static_cast<float*>(m->adam_v.p),
                                                        static_cast<const float*>(m->grad.p), float(lr),
                                                        float(1.0 / (1.0 - std::pow(0.9, t))),
                                                        float(1.0 / (1.0 - std::pow(0.999, t))));
    CK(cudaGetLastError(), "mlp_train adam");
  }
  CK(launch_pack(th, static_cast<uint32_t*>(m->packed.p), st), "mlp_train pack");
  std::vector<float> tail(static_cast<size_t>(n_tail));
  CK(cudaMemcpyAsync(tail.data(), losses, size_t(n_tail) * 4, cudaMemcpyDeviceToHost, st), "mlp_train loss");
  CK(cudaStreamSynchronize(st), "mlp_train sync");
  if (final_loss) {
    double s = 0;
    for (float v : tail) s += v;
    *final_loss = float(s / n_tail);
  }
  return SPOLY_OK;
}

}  // extern "C"
