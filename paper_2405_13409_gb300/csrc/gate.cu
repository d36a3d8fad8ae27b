// Learned candidate gate: feature kernel, the fused feature + BF16 tensor-core
// MLP + compaction kernel, weight packing, labels from a solve, and the C ABI
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

// B fragments of mma.m16n8k16 for W[K][N] (row-major FP32): register r of
// lane (g = lane / 4, c = lane % 4) in tile (kt, nt) holds W[k][n], W[k+1][n]
// with k = 16 kt + 2 c + 8 r and n = 8 nt + g.
__global__ void pack_kernel(const float* __restrict__ theta, uint32_t* __restrict__ packed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kPackB) {
    int w = i, off = kOffW1;
    if (w >= kFragW1 + kFragW23) {
      w -= kFragW1 + kFragW23;
      off = kOffW3;
    } else if (w >= kFragW1) {
      w -= kFragW1;
      off = kOffW2;
    }
    const int r = w & 1, lane = (w >> 1) & 31, tile = w >> 6;
    const int nt = tile % (kHid / 8), kt = tile / (kHid / 8);
    const int k = 16 * kt + 2 * (lane & 3) + 8 * r, n = 8 * nt + (lane >> 2);
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

// d = a b + c with c given apart (the bias), so the accumulators need no
// initialising moves.
SPOLY_D void mma_bf16_c(float (&d)[4], const uint32_t (&a)[4], uint2 b, float c0, float c1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%11,%10,%11};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y), "f"(c0), "f"(c1));
}

SPOLY_D void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint2 b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b.x), "r"(b.y));
}

constexpr int kGateRows = 128;  // rows per tile: 4 warps x 32
constexpr int kXStride = 40;    // BF16 per feature row in shared memory (32 + 8 pad: no bank conflicts)

// One dense layer for the warp's 32 rows (two m16 tiles): acc = bias + A W,
// with A in registers (KT k-tiles) and W's fragments in shared memory.
template <int KT>
SPOLY_D void layer(float (&acc)[2][8][4], const uint32_t (&a)[2][4][4], const uint2* __restrict__ wf,
                   const float* __restrict__ bias, int lane) {
  const int c2 = 2 * (lane & 3);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float b0 = bias[8 * nt + c2], b1 = bias[8 * nt + c2 + 1];
    const uint2 b = wf[nt * 32 + lane];
    mma_bf16_c(acc[0][nt], a[0][0], b, b0, b1);
    mma_bf16_c(acc[1][nt], a[1][0], b, b0, b1);
  }
#pragma unroll
  for (int kt = 1; kt < KT; ++kt)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const uint2 b = wf[(kt * 8 + nt) * 32 + lane];
      mma_bf16(acc[0][nt], a[0][kt], b);
      mma_bf16(acc[1][nt], a[1][kt], b);
    }
}

// ReLU of the layer output, rounded to BF16 and laid out as the next layer's
// A fragments: output n-tiles 2j and 2j+1 form input k-tile j.
SPOLY_D void relu_to_a(const float (&acc)[2][8][4], uint32_t (&a)[2][4][4]) {
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float* lo = acc[mt][2 * j];
      const float* hi = acc[mt][2 * j + 1];
      a[mt][j][0] = pack_relu_bf16(lo[0], lo[1]);
      a[mt][j][1] = pack_relu_bf16(lo[2], lo[3]);
      a[mt][j][2] = pack_relu_bf16(hi[0], hi[1]);
      a[mt][j][3] = pack_relu_bf16(hi[2], hi[3]);
    }
}

__global__ void __launch_bounds__(128, 4) gate_kernel(GateParams G) {
  __shared__ __align__(16) uint32_t sw[kPackWords];
  __shared__ __align__(16) __nv_bfloat16 sx[kGateRows * kXStride];
  __shared__ float sz[kGateRows];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = 4 * tid; i < kPackWords; i += 4 * blockDim.x)
    *reinterpret_cast<uint4*>(sw + i) = __ldg(reinterpret_cast<const uint4*>(G.packed + i));
  const uint2* w1 = reinterpret_cast<const uint2*>(sw);
  const uint2* w2 = reinterpret_cast<const uint2*>(sw + kFragW1);
  const uint2* w3 = reinterpret_cast<const uint2*>(sw + kFragW1 + kFragW23);
  const float* bv = reinterpret_cast<const float*>(sw + kPackB);
  const int g = lane >> 2, c2 = 2 * (lane & 3);
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
      chain_features(G.mesh, G.qv, G.chains, row, f);
    } else {
#pragma unroll
      for (int j = 0; j < kFeat; ++j) f[j] = 0.0f;
    }
    const bool inside = f[kFeatMinBary] >= kGateInside;
    uint32_t* xr = reinterpret_cast<uint32_t*>(sx + tid * kXStride);
#pragma unroll
    for (int j = 0; j < kFeat / 2; ++j) xr[j] = pack_bf16(f[2 * j], f[2 * j + 1]);
#pragma unroll
    for (int j = kFeat / 2; j < kIn / 2; ++j) xr[j] = 0u;
    __syncthreads();  // also orders the weight staging before the first tile

    uint32_t a[2][4][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) {
        const __nv_bfloat16* p = sx + (warp * 32 + mt * 16 + g) * kXStride + kt * 16 + c2;
        a[mt][kt][0] = *reinterpret_cast<const uint32_t*>(p);
        a[mt][kt][1] = *reinterpret_cast<const uint32_t*>(p + 8 * kXStride);
        a[mt][kt][2] = *reinterpret_cast<const uint32_t*>(p + 8);
        a[mt][kt][3] = *reinterpret_cast<const uint32_t*>(p + 8 * kXStride + 8);
      }
    float acc[2][8][4];
    layer<2>(acc, a, w1, bv, lane);
    relu_to_a(acc, a);
    layer<4>(acc, a, w2, bv + kHid, lane);
    relu_to_a(acc, a);
    layer<4>(acc, a, w3, bv + 2 * kHid, lane);
    const float* w4 = bv + 3 * kHid;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      float zl = 0.0f, zh = 0.0f;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float wa = w4[8 * nt + c2], wb = w4[8 * nt + c2 + 1];
        zl += fmaxf(acc[mt][nt][0], 0.f) * wa + fmaxf(acc[mt][nt][1], 0.f) * wb;
        zh += fmaxf(acc[mt][nt][2], 0.f) * wa + fmaxf(acc[mt][nt][3], 0.f) * wb;
      }
      zl += __shfl_xor_sync(0xffffffffu, zl, 1);
      zl += __shfl_xor_sync(0xffffffffu, zl, 2);
      zh += __shfl_xor_sync(0xffffffffu, zh, 1);
      zh += __shfl_xor_sync(0xffffffffu, zh, 2);
      if ((lane & 3) == 0) {
        sz[warp * 32 + mt * 16 + g] = zl + bv[4 * kHid];
        sz[warp * 32 + mt * 16 + g + 8] = zh + bv[4 * kHid];
      }
    }
    __syncthreads();
    const float z = sz[tid];
    if (valid && G.logits) G.logits[row] = z;
    if (G.out_chains) {
      // 2-bounce chains are outside the network's domain and pass ungated;
      // a chain whose tangential-mismatch zero lies inside the triangle
      // always passes (the network only rejects chains whose zero lies
      // outside it)
      const bool keep = valid && (z >= G.tau_logit || inside || __ldg(G.chains + 3 * row + 2) >= 0);
      const unsigned long long slot = warp_append(G.out_n, keep ? 1u : 0u);
      if (keep) {
        G.out_chains[3 * slot] = __ldg(G.chains + 3 * row);
        G.out_chains[3 * slot + 1] = __ldg(G.chains + 3 * row + 1);
        G.out_chains[3 * slot + 2] = __ldg(G.chains + 3 * row + 2);
      }
    }
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

cudaError_t launch_gate(const GateParams& G, int num_sms, cudaStream_t st) {
  if (G.n <= 0) return cudaSuccess;
  static int per_sm = 0;  // resident blocks per SM (same for every launch of this kernel)
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gate_kernel, 128, 0) != cudaSuccess || b < 1) b = 1;
    per_sm = b;
  }
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
  for (DevBuf* b : {&m->theta, &m->adam_m, &m->adam_v, &m->packed, &m->xb, &m->yb, &m->z1, &m->z2, &m->z3, &m->dz1,
                    &m->dz2, &m->dz3, &m->grad, &m->loss, &m->lists, &m->list_n, &m->logits})
    b->release();
  delete m;
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
  CK(launch_gate(G, ctx->num_sms, ctx->stream), "mlp_forward");
  CK(cudaStreamSynchronize(ctx->stream), "mlp_forward sync");
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
  e = launch_gate(G, ctx->num_sms, ctx->stream);
  unsigned long long cnt = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, ch->counter.p, 8, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "gate"));
  ch->n = int64_t(cnt);
  ch->n_k2 = in->n_k2;  // every 2-bounce chain passes
  *inout = ch;
  return SPOLY_OK;
}

}  // extern "C"
