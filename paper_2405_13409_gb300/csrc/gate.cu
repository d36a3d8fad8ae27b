// Learned candidate gate: feature kernel, the fused feature + BF16 tensor-core
// (tcgen05) MLP + compaction kernel, weight packing, labels from a solve, and the C ABI
// of the network handle (create, parameters, save/load, forward, calibrate,
// gate).  Training lives in mlp_train.cu.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mlp.cuh"
#include "umma.cuh"

namespace spoly {

// ---------------------------------------------------------------- kernels
__global__ void __launch_bounds__(128) features_kernel(MeshView mesh, QueryView qv, const int32_t* chains, int64_t n,
                                                       float* out) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    float f[kFeat];
    chain_features(mesh, qv, chains, i, f);
    float4* o = reinterpret_cast<float4*>(out + i * kFeat);
#pragma unroll
    for (int j = 0; j < kFeat / 4; ++j) o[j] = make_float4(f[4 * j], f[4 * j + 1], f[4 * j + 2], f[4 * j + 3]);
  }
}

SPOLY_D uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x (low half) = lo
  return *reinterpret_cast<uint32_t*>(&v);
}

// Inference weights: W1, W2, W3 as the K-major B operands of the tensor-core
// MMA (row n = output unit, K = input units, BF16 pairs along k in the
// no-swizzle core-matrix layout of umma_off), then the FP32 vectors b1 b2 b3
// w4 b4.  theta holds W[k][n] row-major.
__global__ void pack_kernel(const float* __restrict__ theta, uint32_t* __restrict__ packed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kPackB) {
    int w = i, off = kOffW1, K = kIn;
    if (w >= kFragW1 + kFragW23) {
      w -= kFragW1 + kFragW23;
      off = kOffW3;
      K = kHid;
    } else if (w >= kFragW1) {
      w -= kFragW1;
      off = kOffW2;
      K = kHid;
    }
    // invert umma_off: byte 4 w of the matrix holds (n, k), (n, k + 1)
    const int b = 4 * w, grp = b / (16 * K), rem = b % (16 * K);
    const int n = 8 * grp + (rem & 127) / 16, k = 8 * (rem / 128) + (rem & 15) / 2;
    packed[i] = pack_bf16(theta[off + k * kHid + n], theta[off + (k + 1) * kHid + n]);
  } else if (i < kPackWords) {
    const int j = i - kPackB;  // b1 b2 b3 w4 b4 pad
    float v = 0.0f;
    if (j < kHid)
      v = theta[kOffB1 + j];
    else if (j < 2 * kHid)
      v = theta[kOffB2 + j - kHid];
    else if (j < 3 * kHid)
      v = theta[kOffB3 + j - 2 * kHid];
    else if (j < 4 * kHid)
      v = theta[kOffW4 + j - 3 * kHid];
    else if (j == 4 * kHid)
      v = theta[kOffB4];
    packed[i] = __float_as_uint(v);
  }
}

// ReLU, then BF16 rounding (nearest even) of two values in one instruction;
// the low half holds lo.
SPOLY_D uint32_t pack_relu_bf16(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;\n" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Two FP32 additions in one instruction (each rounded to nearest, as two
// scalar additions would be).
SPOLY_D void add2(float a0, float a1, float b0, float b1, float& r0, float& r1) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a0), "f"(a1));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b0), "f"(b1));
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r0), "=f"(r1) : "l"(rd));
}

constexpr int kGateRows = 128;                 // candidates per tile: the MMA's M, one per thread and TMEM lane
constexpr uint32_t kGateTmemCols = kHid;       // one 128 x 64 FP32 accumulator, reused by the three layers
constexpr uint32_t kGateIdesc = umma_idesc_bf16(kGateRows, kHid);
constexpr long long kGateWaitCycles = 1ll << 31;  // default wait limit: about one second at the SM clock
constexpr int kGateMaxPerSm = 512 / kGateTmemCols;  // CTAs whose accumulators fit one SM's tensor memory
static_assert(umma_off(kGateRows - 1, kHid - 1, kHid) == kGateRows * kHid * 2 - 2, "A tile layout");
static_assert(umma_off(kHid - 1, kIn - 1, kIn) == 4 * kFragW1 - 2, "W1 tile layout");
static_assert(umma_off(kHid - 1, kHid - 1, kHid) == 4 * kFragW23 - 2, "W2, W3 tile layout");

// The layer's MMAs (K / 16 steps of M = 128, N = 64) over A at a_s and the
// weights at w_s, then the commit; thread 0 only.
SPOLY_D void gate_issue(uint32_t tmem, uint32_t a_s, uint32_t w_s, int K, uint32_t bar_s) {
  tc_fence_after();
  const uint32_t sbo = uint32_t(K) * 16u;
  for (int s = 0; s < K / 16; ++s)
    umma_bf16(tmem, umma_desc(a_s + 256u * s, 128u, sbo), umma_desc(w_s + 256u * s, 128u, sbo), kGateIdesc,
              s > 0 ? 1u : 0u);
  umma_commit(bar_s);
}

// Fused gate over tiles of 128 candidates: features (FP32), three BF16 layers
// on the tensor cores (tcgen05.mma, accumulator in tensor memory), the FP32
// output layer, the threshold, compaction.  Thread t owns row t of the tile:
// it writes the row's features and hidden activations into the A tile and
// reads the row's accumulator from TMEM lane t.  Every wait for the tensor
// core is bounded (G.wait_cycles per layer); a wait that gives up sets
// *G.status and ends the CTA's loop, and the CTA then waits for the MMA
// still in flight with the full default limit before it frees its tensor
// memory.
__global__ void __launch_bounds__(128, 4) gate_kernel(GateParams G) {
  __shared__ __align__(1024) uint8_t sa[kGateRows * kHid * 2];  // A: 128 rows x K (32 or 64) BF16
  __shared__ __align__(1024) uint32_t sw[kPackWords];            // W1 W2 W3 (B tiles), then FP32 vectors
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = 4 * tid; i < kPackWords; i += 4 * blockDim.x)
    *reinterpret_cast<uint4*>(sw + i) = __ldg(reinterpret_cast<const uint4*>(G.packed + i));
  __syncwarp();  // tcgen05.alloc and dealloc are executed by a converged warp
  if (warp == 0) tmem_alloc(&tmem_slot, kGateTmemCols);
  if (tid == 0) mbar_init(&bar, 1);
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t t_row = tmem + (uint32_t(warp * 32) << 16);  // the warp's 32 lanes
  const uint32_t a_s = smem_addr(sa), w_s = smem_addr(sw), bar_s = smem_addr(&bar);
  const float* bv = reinterpret_cast<const float*>(sw + kPackB);
  uint8_t* a_row32 = sa + (tid >> 3) * (kIn * 16) + (tid & 7) * 16;   // row tid of a K = 32 tile
  uint8_t* a_row64 = sa + (tid >> 3) * (kHid * 16) + (tid & 7) * 16;  // row tid of a K = 64 tile
  uint32_t parity = 0;
  bool bad = false;
  const long long limit = G.wait_cycles > 0 ? G.wait_cycles : kGateWaitCycles;
  // completion of the layer just issued; warp-uniform result
  auto wait = [&]() {
    const bool ok = __all_sync(0xffffffffu, mbar_wait(bar_s, parity, limit));
    parity ^= 1u;
    tc_fence_after();
    return ok;
  };
  // relu(acc + bias) rounded to BF16 into the A tile (K = 64) of the next layer
  auto hidden = [&](const float* bias) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[32];
      tmem_ld32(t_row + 32u * h, v);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float* x = v + 8 * c;
        const float* bb = bias + 32 * h + 8 * c;
        float y[8];
#pragma unroll
        for (int e = 0; e < 8; e += 2) add2(x[e], x[e + 1], bb[e], bb[e + 1], y[e], y[e + 1]);
        uint4 q;
        q.x = pack_relu_bf16(y[0], y[1]);
        q.y = pack_relu_bf16(y[2], y[3]);
        q.z = pack_relu_bf16(y[4], y[5]);
        q.w = pack_relu_bf16(y[6], y[7]);
        *reinterpret_cast<uint4*>(a_row64 + (4 * h + c) * 128) = q;
      }
    }
  };
  QueryF qc;  // the last query's FP32 data, reused while the chains share it
  for (int64_t base = int64_t(blockIdx.x) * kGateRows; base < G.n; base += int64_t(gridDim.x) * kGateRows) {
    const int64_t row = base + tid;
    const bool valid = row < G.n;
    float f[kFeat];
    if (valid && G.feat) {
      const float4* src = reinterpret_cast<const float4*>(G.feat + row * kFeat);
#pragma unroll
      for (int j = 0; j < kFeat / 4; ++j) {
        const float4 v = __ldg(src + j);
        f[4 * j] = v.x;
        f[4 * j + 1] = v.y;
        f[4 * j + 2] = v.z;
        f[4 * j + 3] = v.w;
      }
    } else if (valid) {
      chain_features(G.mesh, G.qv, G.chains, row, f, qc);
    } else {
#pragma unroll
      for (int j = 0; j < kFeat; ++j) f[j] = 0.0f;
    }
    const bool inside = f[kFeatMinBary] >= kGateInside;
    // layer 1 input: features 0-23, zeros 24-31
#pragma unroll
    for (int c = 0; c < kIn / 8; ++c) {
      uint4 q = make_uint4(0u, 0u, 0u, 0u);
      if (8 * c < kFeat) {
        q.x = pack_bf16(f[8 * c], f[8 * c + 1]);
        q.y = pack_bf16(f[8 * c + 2], f[8 * c + 3]);
        q.z = pack_bf16(f[8 * c + 4], f[8 * c + 5]);
        q.w = pack_bf16(f[8 * c + 6], f[8 * c + 7]);
      }
      *reinterpret_cast<uint4*>(a_row32 + c * 128) = q;
    }
    fence_async_smem();
    tc_fence_before();
    if (__syncthreads_or(bad)) break;
    if (tid == 0) gate_issue(tmem, a_s, w_s, kIn, bar_s);
    bool ok = wait();
    if (ok) hidden(bv);
    fence_async_smem();
    tc_fence_before();
    if (__syncthreads_or(!ok)) {
      bad = true;
      break;
    }
    if (tid == 0) gate_issue(tmem, a_s, w_s + 4u * kFragW1, kHid, bar_s);
    ok = wait();
    if (ok) hidden(bv + kHid);
    fence_async_smem();
    tc_fence_before();
    if (__syncthreads_or(!ok)) {
      bad = true;
      break;
    }
    if (tid == 0) gate_issue(tmem, a_s, w_s + 4u * (kFragW1 + kFragW23), kHid, bar_s);
    ok = wait();
    // output layer in FP32: z = b4 + w4 . relu(acc + b3)
    float z = bv[4 * kHid];
    if (ok) {
      const float* b3 = bv + 2 * kHid;
      const float* w4 = bv + 3 * kHid;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float v[32];
        tmem_ld32(t_row + 32u * h, v);
#pragma unroll
        for (int j = 0; j < 32; j += 2) {
          float y0, y1;
          add2(v[j], v[j + 1], b3[32 * h + j], b3[32 * h + j + 1], y0, y1);
          z = fmaf(fmaxf(y0, 0.0f), w4[32 * h + j], z);
          z = fmaf(fmaxf(y1, 0.0f), w4[32 * h + j + 1], z);
        }
      }
    }
    bad = !ok;
    if (valid && ok && G.logits) G.logits[row] = z;
    if (G.out_chains) {
      // 2-bounce chains are outside the network's domain and pass ungated;
      // a chain whose tangential-mismatch zero lies inside the triangle
      // always passes (the network only rejects chains whose zero lies
      // outside it)
      const bool keep = valid && ok && (z >= G.tau_logit || inside || __ldg(G.chains + 3 * row + 2) >= 0);
      const unsigned long long slot = warp_append(G.out_n, keep ? 1u : 0u);
      if (keep) {
        G.out_chains[3 * slot] = __ldg(G.chains + 3 * row);
        G.out_chains[3 * slot + 1] = __ldg(G.chains + 3 * row + 1);
        G.out_chains[3 * slot + 2] = __ldg(G.chains + 3 * row + 2);
      }
    }
  }
  tc_fence_before();
  if (__syncthreads_or(bad)) {
    // a wait gave up: report it, and give the MMA still in flight one more
    // bounded wait before its accumulator is freed
    if (tid == 0) {
      if (G.status) atomicOr(G.status, 1ull);
      mbar_wait(bar_s, parity ^ 1u, kGateWaitCycles);
    }
    __syncthreads();
  }
  __syncwarp();
  if (warp == 0) {
    tc_fence_after();
    tmem_free(tmem, kGateTmemCols);
  }
}

// labels[chain] = 1 for every chain with a returned path.
__global__ void labels_kernel(const spoly_path* __restrict__ paths, int64_t n_paths, int64_t n_chains,
                              uint8_t* __restrict__ labels) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_paths; i += int64_t(gridDim.x) * blockDim.x) {
    const int c = paths[i].chain;
    if (c >= 0 && c < n_chains) labels[c] = 1;
  }
}

// Resident blocks of `threads` threads per SM for a kernel without dynamic
// shared memory, from its registers (allocated per warp in units of 256) and
// static shared memory against the SM's limits.  The occupancy API answers
// one block per SM for the tensor-memory kernel below, which limits only its
// tensor memory to 64 of 512 columns per block.
int resident_blocks(const void* fn, int threads) {
  cudaFuncAttributes a{};
  int dev = 0, regs = 0, smem = 0, thr = 0, reserved = 0;
  if (cudaFuncGetAttributes(&a, fn) != cudaSuccess || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&thr, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
    return 1;
  const int warps = (threads + 31) / 32;
  const int per_warp = (a.numRegs * 32 + 255) / 256 * 256;
  int b = thr / (32 * warps);
  if (per_warp > 0) b = std::min(b, regs / (per_warp * warps));
  b = std::min(b, smem / int(a.sharedSizeBytes + size_t(reserved)));
  return std::max(b, 1);
}

cudaError_t launch_gate(const GateParams& G, int num_sms, cudaStream_t st) {
  if (G.n <= 0) return cudaSuccess;
  static int per_sm = 0;  // resident blocks per SM (same for every launch of this kernel)
  if (per_sm == 0) per_sm = std::min(resident_blocks(reinterpret_cast<const void*>(gate_kernel), 128), kGateMaxPerSm);
  int64_t grid = (G.n + kGateRows - 1) / kGateRows;
  grid = std::min<int64_t>(grid, int64_t(num_sms) * per_sm);
  gate_kernel<<<int(grid), 128, 0, st>>>(G);
  return cudaGetLastError();
}

cudaError_t launch_pack(const float* theta, uint32_t* packed, cudaStream_t st) {
  pack_kernel<<<(kPackWords + 255) / 256, 256, 0, st>>>(theta, packed);
  return cudaGetLastError();
}

}  // namespace spoly

using namespace spoly;

namespace {

// splitmix64 (Steele, Lea and Flood, 2014): the initial weights' generator.
uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

spoly_status upload_params(spoly_ctx* ctx, spoly_mlp* m, const float* host) {
  CK(cudaMemcpyAsync(m->theta.p, host, kParams * sizeof(float), cudaMemcpyHostToDevice, ctx->stream), "params");
  CK(launch_pack(static_cast<const float*>(m->theta.p), static_cast<uint32_t*>(m->packed.p), ctx->stream), "pack");
  CK(cudaStreamSynchronize(ctx->stream), "params sync");
  return SPOLY_OK;
}

spoly_status alloc_mlp(spoly_ctx* ctx, spoly_mlp** out) {
  spoly_mlp* m = new (std::nothrow) spoly_mlp();
  if (!m) return fail(ctx, SPOLY_ENOMEM, "mlp: host allocation");
  m->device = ctx->device;
  cudaError_t e = m->theta.ensure(kParams * sizeof(float));
  if (e == cudaSuccess) e = m->adam_m.ensure(kParams * sizeof(float));
  if (e == cudaSuccess) e = m->adam_v.ensure(kParams * sizeof(float));
  if (e == cudaSuccess) e = m->packed.ensure(kPackWords * sizeof(uint32_t));
  if (e == cudaSuccess) e = m->status.ensure(16);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->adam_m.p, 0, kParams * sizeof(float), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->adam_v.p, 0, kParams * sizeof(float), ctx->stream);
  if (e != cudaSuccess) {
    spoly_mlp_free(m);
    return cuda_fail(ctx, e, "mlp: device allocation");
  }
  *out = m;
  return SPOLY_OK;
}

const char kMagic[8] = {'S', 'P', 'O', 'L', 'Y', 'M', 'L', 'P'};

}  // namespace

extern "C" {

spoly_status spoly_mlp_create(spoly_ctx* ctx, uint64_t seed, spoly_mlp** out) {
  if (!ctx) return SPOLY_EINVAL;
  if (!out) return fail(ctx, SPOLY_EINVAL, "mlp_create: out is NULL");
  *out = nullptr;
  spoly_mlp* m = nullptr;
  spoly_status s = alloc_mlp(ctx, &m);
  if (s != SPOLY_OK) return s;
  // He-uniform weights (bound sqrt(6 / fan_in)), zero biases.
  std::vector<float> h(kParams, 0.0f);
  uint64_t st = seed;
  auto fill = [&](int off, int fan_in, int count) {
    const double bound = std::sqrt(6.0 / fan_in);
    for (int i = 0; i < count; ++i) {
      const double u = double(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
      h[off + i] = float((2.0 * u - 1.0) * bound);
    }
  };
  fill(kOffW1, kFeat, kIn * kHid);
  fill(kOffW2, kHid, kHid * kHid);
  fill(kOffW3, kHid, kHid * kHid);
  fill(kOffW4, kHid, kHid);
  for (int r = kFeat; r < kIn; ++r)
    for (int c = 0; c < kHid; ++c) h[kOffW1 + r * kHid + c] = 0.0f;  // padding inputs
  s = upload_params(ctx, m, h.data());
  if (s != SPOLY_OK) {
    spoly_mlp_free(m);
    return s;
  }
  *out = m;
  return SPOLY_OK;
}

spoly_status spoly_mlp_free(spoly_mlp* m) {
  if (!m) return SPOLY_EINVAL;
  for (DevBuf* b : {&m->theta, &m->adam_m, &m->adam_v, &m->packed, &m->status, &m->xb, &m->yb, &m->z1, &m->z2, &m->z3, &m->dz1,
                    &m->dz2, &m->dz3, &m->grad, &m->loss, &m->lists, &m->list_n, &m->logits})
    b->release();
  delete m;
  return SPOLY_OK;
}

spoly_status spoly_mlp_set_wait_limit(spoly_mlp* m, int64_t cycles) {
  if (!m || cycles < 0) return SPOLY_EINVAL;
  m->wait_cycles = (long long)cycles;
  return SPOLY_OK;
}

spoly_status spoly_mlp_get_params(spoly_ctx* ctx, const spoly_mlp* m, float* dst) {
  if (!ctx) return SPOLY_EINVAL;
  if (!m || !dst) return fail(ctx, SPOLY_EINVAL, "mlp_get_params: NULL argument");
  CK(cudaMemcpyAsync(dst, m->theta.p, kParams * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "params");
  CK(cudaStreamSynchronize(ctx->stream), "params sync");
  return SPOLY_OK;
}

spoly_status spoly_mlp_set_params(spoly_ctx* ctx, spoly_mlp* m, const float* src) {
  if (!ctx) return SPOLY_EINVAL;
  if (!m || !src) return fail(ctx, SPOLY_EINVAL, "mlp_set_params: NULL argument");
  for (int i = 0; i < kParams; ++i)
    if (!std::isfinite(src[i])) return fail(ctx, SPOLY_EINVAL, "mlp_set_params: non-finite value at %d", i);
  return upload_params(ctx, m, src);
}

spoly_status spoly_mlp_save(spoly_ctx* ctx, const spoly_mlp* m, const char* path) {
  if (!ctx) return SPOLY_EINVAL;
  if (!m || !path) return fail(ctx, SPOLY_EINVAL, "mlp_save: NULL argument");
  std::vector<float> h(3 * size_t(kParams));
  CK(cudaMemcpyAsync(h.data(), m->theta.p, kParams * 4, cudaMemcpyDeviceToHost, ctx->stream), "save");
  CK(cudaMemcpyAsync(h.data() + kParams, m->adam_m.p, kParams * 4, cudaMemcpyDeviceToHost, ctx->stream), "save");
  CK(cudaMemcpyAsync(h.data() + 2 * kParams, m->adam_v.p, kParams * 4, cudaMemcpyDeviceToHost, ctx->stream), "save");
  CK(cudaStreamSynchronize(ctx->stream), "save sync");
  FILE* fp = fopen(path, "wb");
  if (!fp) return fail(ctx, SPOLY_EINVAL, "mlp_save: cannot open %s", path);
  const int32_t hdr[2] = {1, kParams};
  const int64_t step = m->adam_step;
  bool ok = fwrite(kMagic, 1, 8, fp) == 8 && fwrite(hdr, 4, 2, fp) == 2 && fwrite(&step, 8, 1, fp) == 1 &&
            fwrite(h.data(), 4, h.size(), fp) == h.size();
  ok = (fclose(fp) == 0) && ok;
  if (!ok) return fail(ctx, SPOLY_EINVAL, "mlp_save: write to %s failed", path);
  return SPOLY_OK;
}

spoly_status spoly_mlp_load(spoly_ctx* ctx, const char* path, spoly_mlp** out) {
  if (!ctx) return SPOLY_EINVAL;
  if (!path || !out) return fail(ctx, SPOLY_EINVAL, "mlp_load: NULL argument");
  *out = nullptr;
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(ctx, SPOLY_EINVAL, "mlp_load: cannot open %s", path);
  char mg[8];
  int32_t hdr[2];
  int64_t step = 0;
  std::vector<float> h(3 * size_t(kParams));
  const bool ok = fread(mg, 1, 8, fp) == 8 && std::memcmp(mg, kMagic, 8) == 0 && fread(hdr, 4, 2, fp) == 2 &&
                  hdr[0] == 1 && hdr[1] == kParams && fread(&step, 8, 1, fp) == 1 &&
                  fread(h.data(), 4, h.size(), fp) == h.size();
  fclose(fp);
  if (!ok) return fail(ctx, SPOLY_EINVAL, "mlp_load: %s is not a version-1 network file of %d parameters", path, kParams);
  for (float v : h)
    if (!std::isfinite(v)) return fail(ctx, SPOLY_EINVAL, "mlp_load: non-finite value in %s", path);
  spoly_mlp* m = nullptr;
  spoly_status s = alloc_mlp(ctx, &m);
  if (s != SPOLY_OK) return s;
  m->adam_step = step;
  cudaError_t e = cudaMemcpyAsync(m->adam_m.p, h.data() + kParams, kParams * 4, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->adam_v.p, h.data() + 2 * kParams, kParams * 4, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) {
    spoly_mlp_free(m);
    return cuda_fail(ctx, e, "mlp_load");
  }
  s = upload_params(ctx, m, h.data());
  if (s != SPOLY_OK) {
    spoly_mlp_free(m);
    return s;
  }
  *out = m;
  return SPOLY_OK;
}

spoly_status spoly_mlp_features(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q,
                                const spoly_chains* chains, float* dst) {
  if (!ctx) return SPOLY_EINVAL;
  if (!chains || !dst) return fail(ctx, SPOLY_EINVAL, "mlp_features: NULL argument");
  MeshView mv;
  QueryView qv;
  spoly_status s = stage_inputs(ctx, mesh, q, &mv, &qv);
  if (s != SPOLY_OK) return s;
  if (chains->n > 0) {
    const int64_t grid = std::min<int64_t>((chains->n + 127) / 128, int64_t(ctx->num_sms) * 16);
    features_kernel<<<int(grid), 128, 0, ctx->stream>>>(mv, qv, static_cast<const int32_t*>(chains->buf.p), chains->n,
                                                         dst);
    CK(cudaGetLastError(), "features");
  }
  CK(cudaStreamSynchronize(ctx->stream), "features sync");
  return SPOLY_OK;
}

spoly_status spoly_chain_labels(spoly_ctx* ctx, const spoly_solution_set* set, int64_t n_chains, uint8_t* dst) {
  if (!ctx) return SPOLY_EINVAL;
  if (!set || !dst || n_chains < 0) return fail(ctx, SPOLY_EINVAL, "chain_labels: bad arguments");
  if (!set->host_valid) return fail(ctx, SPOLY_EINVAL, "chain_labels: the solve was asynchronous; read its stats first");
  if (n_chains > 0) CK(cudaMemsetAsync(dst, 0, size_t(n_chains), ctx->stream), "labels clear");
  const int64_t np = std::min<int64_t>(int64_t(set->host[C_ADMISSIBLE]), set->path_cap);
  if (np > 0) {
    const int64_t grid = std::min<int64_t>((np + 255) / 256, int64_t(ctx->num_sms) * 8);
    labels_kernel<<<int(grid), 256, 0, ctx->stream>>>(static_cast<const spoly_path*>(set->paths.p), np, n_chains, dst);
    CK(cudaGetLastError(), "labels");
  }
  CK(cudaStreamSynchronize(ctx->stream), "labels sync");
  return SPOLY_OK;
}

spoly_status spoly_mlp_forward(spoly_ctx* ctx, const spoly_mlp* m, const float* feat, int64_t n, float* logits) {
  if (!ctx) return SPOLY_EINVAL;
  if (!m || (n > 0 && (!feat || !logits)) || n < 0) return fail(ctx, SPOLY_EINVAL, "mlp_forward: bad arguments");
  GateParams G{};
  G.feat = feat;
  G.n = n;
  G.packed = static_cast<const uint32_t*>(m->packed.p);
  G.logits = logits;
  G.status = static_cast<unsigned long long*>(m->status.p);
  G.wait_cycles = m->wait_cycles;
  unsigned long long status = 0;
  CK(cudaMemsetAsync(m->status.p, 0, 8, ctx->stream), "mlp_forward status");
  CK(launch_gate(G, ctx->num_sms, ctx->stream), "mlp_forward");
  CK(cudaMemcpyAsync(&status, m->status.p, 8, cudaMemcpyDeviceToHost, ctx->stream), "mlp_forward status");
  CK(cudaStreamSynchronize(ctx->stream), "mlp_forward sync");
  if (status) return fail(ctx, SPOLY_ETIMEOUT, "mlp_forward: a tensor-core completion wait gave up");
  return SPOLY_OK;
}

spoly_status spoly_mlp_calibrate(spoly_ctx* ctx, spoly_mlp* m, const float* feat, const uint8_t* labels, int64_t n,
                                 double target_recall, float* tau_logit, double* pass_fraction) {
  if (!ctx) return SPOLY_EINVAL;
  if (!m || !feat || !labels || !tau_logit || n <= 0 || !(target_recall > 0.0 && target_recall <= 1.0))
    return fail(ctx, SPOLY_EINVAL, "mlp_calibrate: bad arguments");
  CK(m->logits.ensure(size_t(n) * 4), "calibrate scratch");
  spoly_status s = spoly_mlp_forward(ctx, m, feat, n, static_cast<float*>(m->logits.p));
  if (s != SPOLY_OK) return s;
  std::vector<float> z(static_cast<size_t>(n));
  std::vector<uint8_t> y(static_cast<size_t>(n));
  CK(cudaMemcpyAsync(z.data(), m->logits.p, size_t(n) * 4, cudaMemcpyDeviceToHost, ctx->stream), "calibrate copy");
  CK(cudaMemcpyAsync(y.data(), labels, size_t(n), cudaMemcpyDeviceToHost, ctx->stream), "calibrate copy");
  CK(cudaStreamSynchronize(ctx->stream), "calibrate sync");
  std::vector<float> pos;
  for (int64_t i = 0; i < n; ++i)
    if (y[size_t(i)]) pos.push_back(z[size_t(i)]);
  if (pos.empty()) return fail(ctx, SPOLY_EINVAL, "mlp_calibrate: no positive labels");
  std::sort(pos.begin(), pos.end());
  // Largest threshold that keeps at least target_recall of the positives.
  const int64_t drop = int64_t(std::floor((1.0 - target_recall) * double(pos.size()) + 1e-9));
  const float tau = pos[size_t(std::min<int64_t>(drop, int64_t(pos.size()) - 1))];
  *tau_logit = tau;
  if (pass_fraction) {
    int64_t pass = 0;
    for (float v : z) pass += v >= tau;
    *pass_fraction = double(pass) / double(n);
  }
  return SPOLY_OK;
}

spoly_status spoly_gate(spoly_ctx* ctx, const spoly_mlp* m, const spoly_mesh* mesh, const spoly_queries* q,
                        const spoly_chains* in, float tau_logit, spoly_chains** inout) {
  if (!ctx) return SPOLY_EINVAL;
  if (!m || !in || !inout || in == *inout) return fail(ctx, SPOLY_EINVAL, "gate: bad arguments");
  if (!std::isfinite(tau_logit)) return fail(ctx, SPOLY_EINVAL, "gate: non-finite threshold");
  MeshView mv;
  QueryView qv;
  spoly_status s = stage_inputs(ctx, mesh, q, &mv, &qv);
  if (s != SPOLY_OK) return s;
  spoly_chains* ch = *inout;
  const bool fresh = ch == nullptr;
  if (fresh) {
    ch = new (std::nothrow) spoly_chains();
    if (!ch) return fail(ctx, SPOLY_ENOMEM, "gate: host allocation");
  }
  auto bail = [&](spoly_status st) {
    if (fresh) spoly_chains_free(ch);
    return st;
  };
  cudaError_t e = ch->buf.ensure(size_t(std::max<int64_t>(in->n, 1)) * 12);
  if (e == cudaSuccess) e = ch->counter.ensure(16);
  if (e == cudaSuccess) e = cudaMemsetAsync(ch->counter.p, 0, 16, ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "gate: allocation"));
  GateParams G{};
  G.mesh = mv;
  G.qv = qv;
  G.chains = static_cast<const int32_t*>(in->buf.p);
  G.n = in->n;
  G.packed = static_cast<const uint32_t*>(m->packed.p);
  G.tau_logit = tau_logit;
  G.out_chains = static_cast<int32_t*>(ch->buf.p);
  G.out_n = static_cast<unsigned long long*>(ch->counter.p);
  G.status = G.out_n + 1;  // second word of the cleared counter
  G.wait_cycles = m->wait_cycles;
  e = launch_gate(G, ctx->num_sms, ctx->stream);
  unsigned long long cnt[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, ch->counter.p, 16, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "gate"));
  if (cnt[1]) return bail(fail(ctx, SPOLY_ETIMEOUT, "gate: a tensor-core completion wait gave up"));
  ch->n = int64_t(cnt[0]);
  ch->n_k2 = in->n_k2;  // every 2-bounce chain passes
  *inout = ch;
  return SPOLY_OK;
}

}  // extern "C"
