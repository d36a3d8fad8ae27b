// C ABI of the specular-polynomial library (declared in include/spoly.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ctx.cuh"
#include "k1.cuh"
#include "sqrt_table.cuh"
#include "tt_kernels.cuh"

using namespace spoly;

namespace spoly {
double measure_fma_peak(int kind, int num_sms, cudaStream_t st, cudaError_t* err);
}

namespace spoly {

spoly_status fail(spoly_ctx* ctx, spoly_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

spoly_status cuda_fail(spoly_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(ctx, SPOLY_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(ctx, SPOLY_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Smallest index i < n with x[i] not finite, into *first (all ones: none).
__global__ void nonfinite_kernel(const double* __restrict__ x, int64_t n, unsigned long long* first) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride)
    if (!isfinite(x[i])) atomicMin(first, (unsigned long long)i);
}

// Device views of mesh / queries.  Host arrays are copied into context
// buffers and then checked for non-finite values on the device (one pass
// over the copies and one read-back), which keeps the host off the data.
spoly_status stage_inputs(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q, MeshView* mv,
                          QueryView* qv) {
  if (!mesh || !q) return fail(ctx, SPOLY_EINVAL, "mesh and queries are required");
  if (!mesh->tri || mesh->n_tris <= 0 || mesh->n_tris > INT32_MAX)
    return fail(ctx, SPOLY_EINVAL, "mesh: tri must be non-null and 0 < n_tris <= 2^31-1 (got %lld)",
                (long long)mesh->n_tris);
  if (!q->x_first || !q->x_last || !q->eta || !q->types || !q->k || q->n_queries <= 0 ||
      q->n_queries > INT32_MAX)
    return fail(ctx, SPOLY_EINVAL, "queries: all arrays must be non-null and 0 < n_queries <= 2^31-1");
  const int64_t T = mesh->n_tris, Q = q->n_queries;
  // first non-finite index of the staged mesh ([0]) and query rows ([1..3])
  const bool staged = !mesh->on_device || !q->on_device;
  unsigned long long* first = nullptr;
  if (staged) {
    CK(ctx->check.ensure(4 * sizeof(unsigned long long)), "input check");
    first = static_cast<unsigned long long*>(ctx->check.p);
    CK(cudaMemsetAsync(first, 0xff, 4 * sizeof(unsigned long long), ctx->stream), "input check");
  }
  auto check = [&](const double* x, int64_t n, int slot) -> cudaError_t {
    const int64_t g = std::min<int64_t>((n + 255) / 256, int64_t(ctx->num_sms) * 8);
    nonfinite_kernel<<<unsigned(std::max<int64_t>(g, 1)), 256, 0, ctx->stream>>>(x, n, first + slot);
    return cudaGetLastError();
  };
  if (mesh->on_device) {
    mv->tri = mesh->tri;
  } else {
    CK(ctx->mesh.ensure(size_t(18 * T) * sizeof(double)), "mesh staging");
    CK(cudaMemcpyAsync(ctx->mesh.p, mesh->tri, size_t(18 * T) * sizeof(double), cudaMemcpyHostToDevice,
                       ctx->stream),
       "mesh copy");
    mv->tri = static_cast<const double*>(ctx->mesh.p);
    CK(check(mv->tri, 18 * T, 0), "mesh check");
  }
  mv->n_tris = T;
  if (q->on_device) {
    qv->x_first = q->x_first;
    qv->x_last = q->x_last;
    qv->eta = q->eta;
    qv->types = q->types;
    qv->k = q->k;
  } else {
    for (int64_t i = 0; i < Q; ++i) {
      if (q->k[i] < 1 || q->k[i] > 2) return fail(ctx, SPOLY_EINVAL, "queries: k[%lld] = %d", (long long)i, q->k[i]);
      if ((q->types[2 * i] != SPOLY_R && q->types[2 * i] != SPOLY_T))
        return fail(ctx, SPOLY_EINVAL, "queries: types[%lld] = %d", (long long)i, q->types[2 * i]);
    }
    struct {
      DevBuf* b;
      const void* src;
      size_t n;
    } items[] = {{&ctx->xf, q->x_first, size_t(3 * Q) * 8}, {&ctx->xl, q->x_last, size_t(3 * Q) * 8},
                 {&ctx->eta, q->eta, size_t(3 * Q) * 8},    {&ctx->types, q->types, size_t(2 * Q) * 4},
                 {&ctx->kk, q->k, size_t(Q) * 4}};
    for (auto& it : items) {
      CK(it.b->ensure(it.n), "query staging");
      CK(cudaMemcpyAsync(it.b->p, it.src, it.n, cudaMemcpyHostToDevice, ctx->stream), "query copy");
    }
    qv->x_first = static_cast<const double*>(ctx->xf.p);
    qv->x_last = static_cast<const double*>(ctx->xl.p);
    qv->eta = static_cast<const double*>(ctx->eta.p);
    qv->types = static_cast<const int32_t*>(ctx->types.p);
    qv->k = static_cast<const int32_t*>(ctx->kk.p);
    CK(check(qv->x_first, 3 * Q, 1), "query check");
    CK(check(qv->x_last, 3 * Q, 2), "query check");
    CK(check(qv->eta, 3 * Q, 3), "query check");
  }
  qv->n = Q;
  if (staged) {
    unsigned long long h[4];
    CK(cudaMemcpyAsync(h, first, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "input check");
    CK(cudaStreamSynchronize(ctx->stream), "input check");
    if (h[0] != ~0ull)
      return fail(ctx, SPOLY_EINVAL, "mesh: non-finite value at row %lld, triangle %lld", (long long)(h[0] / T),
                  (long long)(h[0] % T));
    for (int k = 1; k < 4; ++k)
      if (h[k] != ~0ull)
        return fail(ctx, SPOLY_EINVAL, "queries: non-finite value in query %lld", (long long)(h[k] / 3));
  }
  return SPOLY_OK;
}

}  // namespace spoly

namespace spoly {

// 2-bounce chains of a solve: systems, then per batch of systems the FP64
// construction, the FP32 sign sampling and bisection, the FP64 polish and
// the path phase.  Paths are appended through `path_counter`.
spoly_status solve_tt(spoly_ctx* ctx, spoly_solution_set* set, const MeshView& mv, const QueryView& qv,
                      const int32_t* k2, const int32_t* k2_ids, int64_t n2, const spoly_solve_opts* opts,
                      unsigned long long* path_counter, spoly_path* paths, int64_t path_cap) {
  cudaStream_t st = ctx->stream;
  const bool timing = (opts->flags & SPOLY_SOLVE_TIMING) != 0;
  set->tt_sign_ms = 0.0f;
  if (timing && !set->tt_ev[0]) {
    CK(cudaEventCreate(&set->tt_ev[0]), "tt timing");
    CK(cudaEventCreate(&set->tt_ev[1]), "tt timing");
  }
  TTParams T{};
  T.mesh = mv;
  T.qv = qv;
  T.chains = k2;
  T.chain_ids = k2_ids;
  T.n_chains = n2;
  if (opts->sqrt_table) {
    const double* t = opts->sqrt_table;
    for (int i = 0; i <= kSqrtPieces; ++i) T.sqrt_tab.breaks[i] = t[i];
    for (int k = 0; k < kSqrtPieces; ++k)
      for (int j = 0; j < 3; ++j) T.sqrt_tab.c[k][j] = t[kSqrtPieces + 1 + 3 * k + j];
    if (T.sqrt_tab.breaks[0] != 0.0 || T.sqrt_tab.breaks[kSqrtPieces] != 1.0)
      return fail(ctx, SPOLY_EINVAL, "sqrt_table: breaks must run from 0 to 1");
    for (int i = 0; i < kSqrtPieces; ++i)
      if (!(T.sqrt_tab.breaks[i + 1] > T.sqrt_tab.breaks[i]))
        return fail(ctx, SPOLY_EINVAL, "sqrt_table: breaks must increase");
  } else {
    T.sqrt_tab = default_sqrt_table();
  }
  T.n_intervals = opts->n_intervals > 0 ? opts->n_intervals : 4096;
  T.precision = opts->precision;
  if (T.n_intervals > 8192) return fail(ctx, SPOLY_EINVAL, "n_intervals %d exceeds 8192", T.n_intervals);
  T.paths = paths;
  T.path_cap = path_cap;
  T.path_counter = path_counter;
  CK(set->tt_counters.ensure(16 * sizeof(unsigned long long)), "tt counters");
  T.counters = static_cast<unsigned long long*>(set->tt_counters.p);
  CK(cudaMemsetAsync(T.counters, 0, 16 * sizeof(unsigned long long), st), "tt counters");
  CK(set->tt_chain_sys.ensure(size_t(n2) * 2 * sizeof(int32_t)), "tt chain systems");
  CK(set->tt_masks.ensure(size_t(n2)), "tt masks");
  CK(set->tt_active.ensure(8 + size_t(n2) * sizeof(int32_t)), "tt active chains");
  T.active_n = static_cast<unsigned long long*>(set->tt_active.p);
  T.active = reinterpret_cast<int32_t*>(static_cast<char*>(set->tt_active.p) + 8);
  T.chain_sys = static_cast<int32_t*>(set->tt_chain_sys.p);
  CK(launch_tt_count(T, static_cast<uint8_t*>(set->tt_masks.p), ctx->num_sms, st), "tt count");
  // exclusive prefix of the per-chain system counts (host)
  std::vector<int32_t> cs(size_t(n2) * 2);
  CK(cudaMemcpyAsync(cs.data(), T.chain_sys, cs.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "tt counts");
  CK(cudaStreamSynchronize(st), "tt counts");
  int64_t n_sys = 0;
  for (int64_t c = 0; c < n2; ++c) {
    cs[size_t(2 * c)] = int32_t(n_sys);
    n_sys += cs[size_t(2 * c + 1)];
  }
  if (n_sys > INT32_MAX) return fail(ctx, SPOLY_EINVAL, "too many 2-bounce systems");
  CK(cudaMemcpyAsync(T.chain_sys, cs.data(), cs.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st), "tt offsets");
  CK(set->tt_sys.ensure(size_t(std::max<int64_t>(n_sys, 1)) * sizeof(TTSys)), "tt systems");
  T.sys = static_cast<TTSys*>(set->tt_sys.p);
  T.sys_cap = n_sys;
  CK(launch_tt_fill(T, static_cast<const uint8_t*>(set->tt_masks.p), ctx->num_sms, st), "tt fill");
  // batches of whole chains, at most kBatch systems
  constexpr int64_t kBatch = 16384;
  const int64_t bmax = std::min<int64_t>(kBatch, std::max<int64_t>(n_sys, 1));
  CK(set->tt_scratch.ensure(size_t(bmax) * kTTKeep * sizeof(double)), "tt scratch");
  CK(set->tt_coef32.ensure(size_t(bmax) * kTT32 * sizeof(float)), "tt scratch");
  CK(set->tt_queue.ensure(size_t(bmax) * 128 * sizeof(RootItem)), "tt queue");  // 128 brackets per system at most
  T.scratch = static_cast<double*>(set->tt_scratch.p);
  T.coef32 = static_cast<float*>(set->tt_coef32.p);
  T.queue = static_cast<RootItem*>(set->tt_queue.p);
  T.queue_cap = bmax * 128;
  // kept FP32 signs of up to kNoisy re-sampled systems per batch (others are
  // sampled again in full)
  constexpr int64_t kNoisy = 1024;
  CK(set->tt_noisy.ensure(size_t(kNoisy) * (kTTSampleSlots * (sizeof(int8_t) + sizeof(float)) + 3 * sizeof(int32_t))),
     "tt noisy");
  T.noisy_lg = static_cast<float*>(set->tt_noisy.p);
  T.noisy_span = reinterpret_cast<int32_t*>(T.noisy_lg + kNoisy * kTTSampleSlots);
  T.noisy_sgn = reinterpret_cast<int8_t*>(T.noisy_span + 3 * kNoisy);
  T.noisy_cap = kNoisy;
  unsigned long long brackets_total = 0, resampled_total = 0;
  int64_t c0 = 0;
  while (c0 < n2) {
    const int64_t s0 = cs[size_t(2 * c0)];
    int64_t c1 = c0;
    while (c1 < n2 && cs[size_t(2 * c1)] + cs[size_t(2 * c1 + 1)] - s0 <= bmax) ++c1;
    if (c1 == c0) c1 = c0 + 1;  // one chain spans at most six systems < bmax
    const int64_t s1 = c1 < n2 ? cs[size_t(2 * c1)] : n_sys;
    T.sys_offset = s0;
    T.n_sys = s1 - s0;
    CK(cudaMemsetAsync(T.counters + TT_BRACKETS, 0, sizeof(unsigned long long), st), "tt memset");
    CK(launch_tt_build(T, ctx->num_sms, st), "tt build");
    CK(cudaMemsetAsync(T.counters + TT_RESAMPLED, 0, sizeof(unsigned long long), st), "tt memset");
    CK(cudaMemsetAsync(T.counters + TT_NOISY, 0, sizeof(unsigned long long), st), "tt memset");
    if (timing) CK(cudaEventRecord(set->tt_ev[0], st), "tt timing");
    CK(launch_tt_sign(T, ctx->num_sms, st), "tt sign");
    if (timing) CK(cudaEventRecord(set->tt_ev[1], st), "tt timing");
    unsigned long long nres = 0;
    CK(cudaMemcpyAsync(&nres, T.counters + TT_RESAMPLED, sizeof(nres), cudaMemcpyDeviceToHost, st), "tt resample");
    CK(cudaStreamSynchronize(st), "tt resample");
    if (timing) {
      float ms = 0.0f;
      CK(cudaEventElapsedTime(&ms, set->tt_ev[0], set->tt_ev[1]), "tt timing");
      set->tt_sign_ms += ms;
    }
    resampled_total += nres;
    if (nres > 0) {
      T.resample_only = 1;
      CK(launch_tt_sign(T, ctx->num_sms, st), "tt sign (FP64 resample)");
      T.resample_only = 0;
    }
    unsigned long long nb = 0;
    CK(cudaMemcpyAsync(&nb, T.counters + TT_BRACKETS, sizeof(nb), cudaMemcpyDeviceToHost, st), "tt brackets");
    CK(cudaStreamSynchronize(st), "tt brackets");
    brackets_total += nb;
    CK(launch_tt_polish(T, ctx->num_sms, st), "tt polish");
    CK(launch_tt_paths(T, c0, c1, ctx->num_sms, st), "tt paths");
    c0 = c1;
  }
  CK(cudaMemcpyAsync(set->tt_host, T.counters, sizeof(set->tt_host), cudaMemcpyDeviceToHost, st), "tt counters");
  CK(cudaStreamSynchronize(st), "tt counters");
  set->tt_host[TT_BRACKETS] = brackets_total;
  set->tt_host[TT_RESAMPLED] = resampled_total;
  set->tt_host[TT_SYSTEMS] = (unsigned long long)n_sys;
  set->n_k2 = n2;
  return SPOLY_OK;
}

// The 2-bounce chains of a solve without a host read-back, so that the whole
// solve can be captured into one CUDA graph: the system offsets come from a
// device scan, every system runs in one pass (scratch sized for the bound of
// kSqrtPieces systems per chain), the FP64 re-sampling pass always runs and
// finds its systems on the device.  Counters stay on the device; the caller
// reads them after the work completes.  Returns ENOMEM when the bound's
// scratch exceeds kDeviceDrivenBytes (the caller then uses the staged solve).
constexpr size_t kDeviceDrivenBytes = size_t(48) << 30;

size_t tt_device_bytes(int64_t n2) {
  const int64_t nb = n2 * kSqrtPieces;
  return size_t(nb) * (sizeof(TTSys) + kTTKeep * sizeof(double) + kTT32 * sizeof(float) + 128 * sizeof(RootItem)) +
         tt_offsets_scratch_bytes(n2) + size_t(n2) * 13;
}

spoly_status solve_tt_device(spoly_ctx* ctx, spoly_solution_set* set, const MeshView& mv, const QueryView& qv,
                             const int32_t* k2, const int32_t* k2_ids, int64_t n2, const spoly_solve_opts* opts,
                             unsigned long long* path_counter, spoly_path* paths, int64_t path_cap,
                             bool enqueue = true) {
  cudaStream_t st = ctx->stream;
  if (tt_device_bytes(n2) > kDeviceDrivenBytes) return SPOLY_ENOMEM;
  TTParams T{};
  T.mesh = mv;
  T.qv = qv;
  T.chains = k2;
  T.chain_ids = k2_ids;
  T.n_chains = n2;
  if (opts->sqrt_table) {
    const double* t = opts->sqrt_table;
    for (int i = 0; i <= kSqrtPieces; ++i) T.sqrt_tab.breaks[i] = t[i];
    for (int k = 0; k < kSqrtPieces; ++k)
      for (int j = 0; j < 3; ++j) T.sqrt_tab.c[k][j] = t[kSqrtPieces + 1 + 3 * k + j];
  } else {
    T.sqrt_tab = default_sqrt_table();
  }
  T.n_intervals = opts->n_intervals > 0 ? opts->n_intervals : 4096;
  T.precision = opts->precision;
  T.paths = paths;
  T.path_cap = path_cap;
  T.path_counter = path_counter;
  const int64_t bound = n2 * kSqrtPieces;
  CK(set->tt_counters.ensure(16 * sizeof(unsigned long long)), "tt counters");
  CK(set->tt_chain_sys.ensure(size_t(n2) * 2 * sizeof(int32_t)), "tt chain systems");
  CK(set->tt_masks.ensure(size_t(n2)), "tt masks");
  CK(set->tt_active.ensure(8 + size_t(n2) * sizeof(int32_t)), "tt active chains");
  CK(set->tt_offsets.ensure(tt_offsets_scratch_bytes(n2)), "tt offsets");
  CK(set->tt_sys.ensure(size_t(bound) * sizeof(TTSys)), "tt systems");
  CK(set->tt_scratch.ensure(size_t(bound) * kTTKeep * sizeof(double)), "tt scratch");
  CK(set->tt_coef32.ensure(size_t(bound) * kTT32 * sizeof(float)), "tt scratch");
  CK(set->tt_queue.ensure(size_t(bound) * 128 * sizeof(RootItem)), "tt queue");
  constexpr int64_t kNoisy = 1024;
  CK(set->tt_noisy.ensure(size_t(kNoisy) * (kTTSampleSlots * (sizeof(int8_t) + sizeof(float)) + 3 * sizeof(int32_t))),
     "tt noisy");
  T.counters = static_cast<unsigned long long*>(set->tt_counters.p);
  T.active_n = static_cast<unsigned long long*>(set->tt_active.p);
  T.active = reinterpret_cast<int32_t*>(static_cast<char*>(set->tt_active.p) + 8);
  T.chain_sys = static_cast<int32_t*>(set->tt_chain_sys.p);
  T.sys = static_cast<TTSys*>(set->tt_sys.p);
  T.sys_cap = bound;
  T.n_sys = bound;
  T.sys_offset = 0;
  T.n_sys_dev = T.counters + TT_SYSTEMS;
  T.scratch = static_cast<double*>(set->tt_scratch.p);
  T.coef32 = static_cast<float*>(set->tt_coef32.p);
  T.queue = static_cast<RootItem*>(set->tt_queue.p);
  T.queue_cap = bound * 128;
  T.noisy_lg = static_cast<float*>(set->tt_noisy.p);
  T.noisy_span = reinterpret_cast<int32_t*>(T.noisy_lg + kNoisy * kTTSampleSlots);
  T.noisy_sgn = reinterpret_cast<int8_t*>(T.noisy_span + 3 * kNoisy);
  T.noisy_cap = kNoisy;
  set->n_k2 = n2;
  set->tt_device = true;
  if (!enqueue) return SPOLY_OK;  // the buffers are sized (outside a capture)
  CK(cudaMemsetAsync(T.counters, 0, 16 * sizeof(unsigned long long), st), "tt counters");
  CK(launch_tt_count(T, static_cast<uint8_t*>(set->tt_masks.p), ctx->num_sms, st), "tt count");
  CK(launch_tt_offsets(T, set->tt_offsets.p, ctx->num_sms, st), "tt offsets");
  CK(launch_tt_fill(T, static_cast<const uint8_t*>(set->tt_masks.p), ctx->num_sms, st), "tt fill");
  CK(launch_tt_build(T, ctx->num_sms, st), "tt build");
  CK(launch_tt_sign(T, ctx->num_sms, st), "tt sign");
  T.resample_only = 1;
  CK(launch_tt_sign(T, ctx->num_sms, st), "tt sign (FP64 resample)");
  T.resample_only = 0;
  CK(launch_tt_polish(T, ctx->num_sms, st), "tt polish");
  CK(launch_tt_paths(T, 0, n2, ctx->num_sms, st), "tt paths");
  set->n_k2 = n2;
  set->tt_device = true;
  return SPOLY_OK;
}

}  // namespace spoly

extern "C" {

const char* spoly_version(void) { return "spoly-gb300 0.2 (sm_103a)"; }

spoly_status spoly_default_sqrt_table(double* dst, int32_t n) {
  if (!dst || n < 1 + kSqrtPieces * 4) return SPOLY_EINVAL;
  const SqrtTable t = default_sqrt_table();
  for (int i = 0; i <= kSqrtPieces; ++i) dst[i] = t.breaks[i];
  for (int k = 0; k < kSqrtPieces; ++k)
    for (int j = 0; j < 3; ++j) dst[kSqrtPieces + 1 + 3 * k + j] = t.c[k][j];
  return SPOLY_OK;
}

spoly_status spoly_ctx_create(int device, void* cuda_stream, spoly_ctx** out) {
  if (!out) return SPOLY_EINVAL;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return SPOLY_ECUDA;
  if (cudaSetDevice(device) != cudaSuccess) return SPOLY_ECUDA;
  spoly_ctx* ctx = new (std::nothrow) spoly_ctx();
  if (!ctx) return SPOLY_ENOMEM;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  int lo = 0, hi = 0;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&ctx->side_stream, cudaStreamNonBlocking, hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming) != cudaSuccess) {
    if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    delete ctx;
    return SPOLY_ECUDA;
  }
  *out = ctx;
  return SPOLY_OK;
}

spoly_status spoly_ctx_destroy(spoly_ctx* ctx) {
  if (!ctx) return SPOLY_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (DevBuf* b : {&ctx->mesh, &ctx->xf, &ctx->xl, &ctx->eta, &ctx->types, &ctx->kk, &ctx->boxes, &ctx->flag,
                    &ctx->cam, &ctx->bounds, &ctx->fp_scratch, &ctx->fp_entries, &ctx->fp_boxes, &ctx->fp_mark,
                    &ctx->tt_pairs, &ctx->check, &ctx->chain_stage, &ctx->chain_valid,
                    &ctx->vis_grid, &ctx->vis_entries})
    b->release();
  cudaStreamSynchronize(ctx->side_stream);
  cudaStreamDestroy(ctx->side_stream);
  cudaEventDestroy(ctx->fork_ev);
  cudaEventDestroy(ctx->join_ev);
  delete ctx;
  return SPOLY_OK;
}

const char* spoly_last_error(const spoly_ctx* ctx) { return ctx ? ctx->err : "no context"; }

spoly_status spoly_upload(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q, spoly_mesh* mesh_out,
                          spoly_queries* q_out) {
  if (!ctx) return SPOLY_EINVAL;
  if (!mesh_out || !q_out) return fail(ctx, SPOLY_EINVAL, "upload: outputs are required");
  CK(cudaSetDevice(ctx->device), "set device");
  MeshView mv;
  QueryView qv;
  spoly_status st = stage_inputs(ctx, mesh, q, &mv, &qv);
  if (st != SPOLY_OK) return st;
  *mesh_out = *mesh;
  mesh_out->tri = mv.tri;
  mesh_out->on_device = 1;
  *q_out = *q;
  q_out->x_first = qv.x_first;
  q_out->x_last = qv.x_last;
  q_out->eta = qv.eta;
  q_out->types = qv.types;
  q_out->k = qv.k;
  q_out->on_device = 1;
  return SPOLY_OK;
}

spoly_status spoly_build_chains(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q,
                                const spoly_chain_opts* opts, spoly_chains** inout) {
  if (!ctx) return SPOLY_EINVAL;
  if (!opts || !inout) return fail(ctx, SPOLY_EINVAL, "opts and inout are required");
  CK(cudaSetDevice(ctx->device), "set device");
  MeshView mv;
  QueryView qv;
  spoly_status st = stage_inputs(ctx, mesh, q, &mv, &qv);
  if (st != SPOLY_OK) return st;
  int32_t tb = opts->tri_begin, te = opts->tri_end <= 0 ? int32_t(mv.n_tris) : opts->tri_end;
  if (tb < 0 || te > mv.n_tris || tb >= te)
    return fail(ctx, SPOLY_EINVAL, "triangle range [%d, %d) outside [0, %lld)", tb, te, (long long)mv.n_tris);
  if (opts->mode == SPOLY_CHAINS_CONE && !(opts->margin >= 0.0))
    return fail(ctx, SPOLY_EINVAL, "cone margin must be >= 0");
  spoly_chains* ch = *inout;
  bool fresh = false;
  if (!ch) {
    ch = new (std::nothrow) spoly_chains();
    if (!ch) return fail(ctx, SPOLY_ENOMEM, "chains handle");
    fresh = true;
  }
  auto bail = [&](spoly_status s) {
    if (fresh) {
      ch->buf.release();
      ch->counter.release();
      delete ch;
    }
    return s;
  };
  if (ch->counter.ensure(16) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "chain counter"));
  ch->n_k2 = 0;
  ch->n_footprint = 0;
  ChainParams P{};
  P.mesh = mv;
  P.qv = qv;
  P.tri_begin = tb;
  P.tri_count = te - tb;
  P.margin = opts->margin;
  P.count = static_cast<unsigned long long*>(ch->counter.p);
  P.error = reinterpret_cast<int32_t*>(static_cast<char*>(ch->counter.p) + 8);
  cudaError_t e = cudaMemsetAsync(ch->counter.p, 0, 16, ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "memset"));
  const int64_t pairs = qv.n * int64_t(P.tri_count);
  if (opts->mode == SPOLY_CHAINS_ALL) {
    if (ch->buf.ensure(size_t(pairs) * 12) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "chain list"));
    P.out = static_cast<int32_t*>(ch->buf.p);
    P.cap = pairs;
    e = launch_chains_all(P, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chains_all"));
    ch->n = pairs;
  } else if (opts->mode == SPOLY_CHAINS_EXPLICIT) {
    const int64_t n = opts->n_explicit;
    if (!opts->explicit_chains || n <= 0) return bail(fail(ctx, SPOLY_EINVAL, "explicit chain list is empty"));
    if (ch->buf.ensure(size_t(n) * 12) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "chain list"));
    P.out = static_cast<int32_t*>(ch->buf.p);
    P.cap = n;
    const int32_t* src = opts->explicit_chains;
    if (!opts->explicit_on_device) {
      if (ctx->chain_stage.ensure(size_t(n) * 12) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "chain staging"));
      e = cudaMemcpyAsync(ctx->chain_stage.p, src, size_t(n) * 12, cudaMemcpyHostToDevice, ctx->stream);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chain copy"));
      src = static_cast<const int32_t*>(ctx->chain_stage.p);
    }
    e = launch_chains_explicit(P, src, n, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chains_explicit"));
    int32_t herr = 0;
    unsigned long long hk2 = 0;
    e = cudaMemcpyAsync(&herr, P.error, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hk2, P.count, 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chains_explicit sync"));
    if (herr) return bail(fail(ctx, SPOLY_EINVAL, "explicit chain %d references a missing query or triangle", herr - 1));
    ch->n = n;
    ch->n_k2 = int64_t(hk2);
  } else if (opts->mode == SPOLY_CHAINS_EXPLICIT_CONE) {
    // the caller's list, validated, then culled chain by chain
    const int64_t n = opts->n_explicit;
    if (!opts->explicit_chains || n <= 0) return bail(fail(ctx, SPOLY_EINVAL, "explicit chain list is empty"));
    if (!(opts->margin >= 0.0)) return bail(fail(ctx, SPOLY_EINVAL, "cone margin must be >= 0"));
    if (ctx->chain_valid.ensure(size_t(n) * 12) != cudaSuccess || ctx->flag.ensure(16) != cudaSuccess)
      return bail(fail(ctx, SPOLY_ENOMEM, "chain staging"));
    const int32_t* src = opts->explicit_chains;
    if (!opts->explicit_on_device) {
      if (ctx->chain_stage.ensure(size_t(n) * 12) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "chain staging"));
      e = cudaMemcpyAsync(ctx->chain_stage.p, src, size_t(n) * 12, cudaMemcpyHostToDevice, ctx->stream);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chain copy"));
      src = static_cast<const int32_t*>(ctx->chain_stage.p);
    }
    P.out = static_cast<int32_t*>(ctx->chain_valid.p);
    P.cap = n;
    e = launch_chains_explicit(P, src, n, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chains_explicit"));
    int32_t herr = 0;
    e = cudaMemcpyAsync(&herr, P.error, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chains_explicit sync"));
    if (herr) return bail(fail(ctx, SPOLY_EINVAL, "explicit chain %d references a missing query or triangle", herr - 1));
    unsigned long long* k2 = static_cast<unsigned long long*>(ctx->flag.p) + 1;
    e = cudaMemsetAsync(P.count, 0, 8, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(k2, 0, 8, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chain counters"));
    if (ch->buf.ensure(size_t(n) * 12) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "chain list"));
    P.out = static_cast<int32_t*>(ch->buf.p);
    e = launch_chains_explicit_cone(P, static_cast<const int32_t*>(ctx->chain_valid.p), n, k2, ctx->num_sms,
                                    ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chains_explicit_cone"));
    unsigned long long hn = 0, hk2 = 0;
    e = cudaMemcpyAsync(&hn, P.count, 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hk2, k2, 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chains_explicit_cone sync"));
    ch->n = int64_t(hn);
    ch->n_k2 = int64_t(hk2);
  } else if (opts->mode == SPOLY_CHAINS_CONE && opts->second_end > 0) {
    // 2-bounce refraction chains: second triangle in [second_begin, second_end)
    const int32_t sb = opts->second_begin, se = opts->second_end;
    if (sb < 0 || se > mv.n_tris || sb >= se)
      return bail(fail(ctx, SPOLY_EINVAL, "second triangle range [%d, %d) outside [0, %lld)", sb, se,
                       (long long)mv.n_tris));
    TTConeParams T{};
    T.mesh = mv;
    T.qv = qv;
    T.t1_begin = tb;
    T.n1 = te - tb;
    T.t2_begin = sb;
    T.n2 = se - sb;
    T.margin = opts->margin;
    if (ctx->flag.ensure(16) != cudaSuccess || ctx->boxes.ensure(size_t(T.n1) * 12 * sizeof(float)) != cudaSuccess)
      return bail(fail(ctx, SPOLY_ENOMEM, "cone scratch"));
    T.fwd = static_cast<float*>(ctx->boxes.p);
    int32_t shared = 0;
    e = launch_tt_cone_shared(T, static_cast<int32_t*>(ctx->flag.p), ctx->num_sms, ctx->stream, &shared);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "tt cone"));
    if (!shared)
      return bail(fail(ctx, SPOLY_EUNSUPPORTED,
                       "2-bounce cone: every query must be k = 2, types T T or R R (all alike), with the same x0 and IORs"));
    // receiver-independent pairs, then the per-receiver test; both grow to
    // the exact count when their first capacity is exceeded
    int64_t pcap = std::max<int64_t>(4096, int64_t(T.n1) * T.n2 / 16);
    unsigned long long np = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (ctx->tt_pairs.ensure(size_t(pcap) * 8) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "pair list"));
      T.pairs = static_cast<int32_t*>(ctx->tt_pairs.p);
      T.pair_cap = pcap;
      T.pair_count = P.count;
      e = cudaMemsetAsync(P.count, 0, 8, ctx->stream);
      if (e == cudaSuccess) e = launch_tt_cone_pairs(T, ctx->num_sms, ctx->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&np, P.count, 8, cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "tt cone pairs"));
      if (int64_t(np) <= pcap) break;
      pcap = int64_t(np);
    }
    int64_t cap = std::max<int64_t>(int64_t(ch->buf.bytes / 12), qv.n * 64 + 4096);
    unsigned long long nc2 = 0;
    for (int attempt = 0; attempt < 2; ++attempt) {
      if (ch->buf.ensure(size_t(cap) * 12) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "chain list"));
      T.out = static_cast<int32_t*>(ch->buf.p);
      T.cap = cap;
      T.count = P.count;
      e = cudaMemsetAsync(P.count, 0, 8, ctx->stream);
      if (e == cudaSuccess) e = launch_tt_cone_chains(T, int64_t(np), ctx->num_sms, ctx->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&nc2, P.count, 8, cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "tt cone chains"));
      if (int64_t(nc2) <= cap) break;
      cap = int64_t(nc2);
    }
    ch->n = int64_t(nc2);
    ch->n_k2 = int64_t(nc2);
  } else if (opts->mode == SPOLY_CHAINS_CONE) {
    if (ctx->boxes.ensure(size_t(P.tri_count) * 12 * sizeof(float)) != cudaSuccess ||
        ctx->flag.ensure(16) != cudaSuccess)
      return bail(fail(ctx, SPOLY_ENOMEM, "cone scratch"));
    P.boxes = static_cast<float*>(ctx->boxes.p);
    P.shared_x0 = static_cast<int32_t*>(ctx->flag.p);
    // Capacity: start from 1/64 of the pairs, grow to the exact count if exceeded.
    int64_t cap = ch->buf.bytes / 12;
    const int64_t want = pairs / 64 + 4096;
    if (cap < want) {
      if (ch->buf.ensure(size_t(want) * 12) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "chain list"));
      cap = want;
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
      P.out = static_cast<int32_t*>(ch->buf.p);
      P.cap = cap;
      e = launch_chains_cone(P, ctx->num_sms, ctx->stream);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chains_cone"));
      unsigned long long cnt = 0;
      e = cudaMemcpyAsync(&cnt, P.count, 8, cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chains_cone sync"));
      if (int64_t(cnt) <= cap) {
        ch->n = int64_t(cnt);
        break;
      }
      cap = int64_t(cnt);
      if (ch->buf.ensure(size_t(cap) * 12) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "chain list"));
      e = cudaMemsetAsync(ch->counter.p, 0, 16, ctx->stream);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "memset"));
    }
  } else if (opts->mode == SPOLY_CHAINS_FOOTPRINT || opts->mode == SPOLY_CHAINS_FOOTPRINT_UNIQUE) {
    const bool unique = opts->mode == SPOLY_CHAINS_FOOTPRINT_UNIQUE;
    if (!opts->camera) return bail(fail(ctx, SPOLY_EINVAL, "footprint mode needs a camera"));
    const double* cam = opts->camera;
    if (int64_t(cam[14]) * int64_t(cam[15]) != qv.n || cam[14] < 1 || cam[15] < 1)
      return bail(fail(ctx, SPOLY_EINVAL, "footprint: width x height (%g x %g) must equal n_queries (%lld)", cam[14],
                       cam[15], (long long)qv.n));
    if (unique) {
      // one chain per distinct candidate triangle, for query 0 (every pixel
      // must share its endpoints); one read-back, a second pass only when the
      // grid outgrew its capacity
      const int g = int(std::min(8192.0, std::max(1.0, std::ceil(std::sqrt(double(mv.n_tris) / 2.0)))));
      const int64_t n_cells = int64_t(g) * g;
      if (ctx->bounds.ensure(64) != cudaSuccess || ctx->flag.ensure(fp_unique_info_bytes()) != cudaSuccess ||
          ctx->fp_boxes.ensure(size_t(mv.n_tris) * sizeof(float4)) != cudaSuccess ||
          ctx->fp_mark.ensure(size_t(mv.n_tris)) != cudaSuccess ||
          ctx->fp_scratch.ensure(footprint_scratch_bytes(n_cells, qv.n)) != cudaSuccess ||
          ch->buf.ensure(size_t(mv.n_tris) * 12) != cudaSuccess)
        return bail(fail(ctx, SPOLY_ENOMEM, "footprint scratch"));
      int64_t cap = std::max<int64_t>(int64_t(ctx->fp_entries.bytes / 4), 4 * mv.n_tris);
      FpUniqueCounts cnt{};
      for (int attempt = 0; attempt < 2; ++attempt) {
        if (ctx->fp_entries.ensure(size_t(cap) * 4) != cudaSuccess)
          return bail(fail(ctx, SPOLY_ENOMEM, "footprint grid entries"));
        e = fp_unique_build(mv, qv, static_cast<float4*>(ctx->fp_boxes.p), static_cast<int*>(ctx->bounds.p), g,
                            ctx->fp_scratch.p, qv.n, static_cast<int32_t*>(ctx->fp_entries.p), cap, cam,
                            static_cast<uint8_t*>(ctx->fp_mark.p), static_cast<int32_t*>(ch->buf.p), ctx->flag.p,
                            &cnt, ctx->num_sms, ctx->stream);
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "footprint distinct triangles"));
        if (cnt.n_entries <= cap) break;
        cap = cnt.n_entries;
      }
      if (!cnt.shared)
        return bail(fail(ctx, SPOLY_EINVAL, "distinct-triangle footprint: every query must share x_first, x_last, "
                                            "eta, types and k"));
      ch->n = cnt.n_unique;
      ch->n_footprint = cnt.pairs;
      *inout = ch;
      return SPOLY_OK;
    }
    if (ctx->bounds.ensure(64) != cudaSuccess) return bail(fail(ctx, SPOLY_ENOMEM, "footprint scratch"));
    if (ctx->fp_boxes.ensure(size_t(mv.n_tris) * sizeof(float4)) != cudaSuccess)
      return bail(fail(ctx, SPOLY_ENOMEM, "footprint triangle boxes"));
    float4* boxes = static_cast<float4*>(ctx->fp_boxes.p);
    float bh[6];
    e = compute_mesh_bounds(mv, static_cast<int*>(ctx->bounds.p), bh, boxes, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "mesh bounds"));
    const double wx = double(bh[3]) - bh[0], wy = double(bh[4]) - bh[1];
    double cell = opts->cell;
    if (!(cell > 0.0)) cell = std::sqrt(std::max(wx * wy, 1e-30) / std::max<double>(1.0, double(mv.n_tris) / 2.0));
    FpGrid g;
    g.cell = cell;
    g.x0 = bh[0];
    g.y0 = bh[1];
    g.gx = int(std::min(8192.0, std::max(1.0, std::ceil(wx / cell) + 1.0)));
    g.gy = int(std::min(8192.0, std::max(1.0, std::ceil(wy / cell) + 1.0)));
    const int64_t n_cells = int64_t(g.gx) * g.gy;
    if (ctx->fp_scratch.ensure(footprint_scratch_bytes(n_cells, qv.n)) != cudaSuccess)
      return bail(fail(ctx, SPOLY_ENOMEM, "footprint scratch"));
    int64_t n_entries = 0, total = 0;
    e = fp_grid_count(mv, boxes, g, ctx->fp_scratch.p, qv.n, &n_entries, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "footprint grid"));
    if (ctx->fp_entries.ensure(size_t(std::max<int64_t>(n_entries, 1)) * 4) != cudaSuccess)
      return bail(fail(ctx, SPOLY_ENOMEM, "footprint grid entries"));
    const int* bounds_dev = static_cast<const int*>(ctx->bounds.p);
    e = fp_grid_fill_and_count(mv, boxes, g, ctx->fp_scratch.p, static_cast<int32_t*>(ctx->fp_entries.p), cam,
                               bounds_dev, qv.n, &total, ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "footprint count"));
    ch->n_footprint = total;
    if (ch->buf.ensure(size_t(std::max<int64_t>(total, 1)) * 12) != cudaSuccess)
      return bail(fail(ctx, SPOLY_ENOMEM, "chain list"));
    e = fp_fill(boxes, g, ctx->fp_scratch.p, static_cast<const int32_t*>(ctx->fp_entries.p), cam, bounds_dev, qv.n,
                static_cast<int32_t*>(ch->buf.p), ctx->num_sms, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "footprint fill"));
    ch->n = total;
  } else {
    return bail(fail(ctx, SPOLY_EINVAL, "unknown chain mode %d", opts->mode));
  }
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "build_chains"));
  *inout = ch;
  return SPOLY_OK;
}

spoly_status spoly_chains_count(const spoly_chains* chains, int64_t* n) {
  if (!chains || !n) return SPOLY_EINVAL;
  *n = chains->n;
  return SPOLY_OK;
}

spoly_status spoly_chains_footprint_pairs(const spoly_chains* chains, int64_t* n) {
  if (!chains || !n) return SPOLY_EINVAL;
  *n = chains->n_footprint;
  return SPOLY_OK;
}

spoly_status spoly_chains_copy(spoly_ctx* ctx, const spoly_chains* chains, int32_t* dst, int64_t capacity,
                               int64_t* n_total, int32_t dst_is_device) {
  if (!ctx) return SPOLY_EINVAL;
  if (!chains || !n_total || (!dst && capacity > 0)) return fail(ctx, SPOLY_EINVAL, "bad arguments");
  *n_total = chains->n;
  const int64_t m = capacity < chains->n ? capacity : chains->n;
  if (m > 0) {
    CK(cudaMemcpyAsync(dst, chains->buf.p, size_t(m) * 12,
                       dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream),
       "chains copy");
    CK(cudaStreamSynchronize(ctx->stream), "chains copy sync");
  }
  if (capacity < chains->n) return fail(ctx, SPOLY_ECAPACITY, "chains: capacity %lld < %lld", (long long)capacity,
                                        (long long)chains->n);
  return SPOLY_OK;
}

spoly_status spoly_chains_free(spoly_chains* chains) {
  if (!chains) return SPOLY_EINVAL;
  chains->buf.release();
  chains->counter.release();
  delete chains;
  return SPOLY_OK;
}

spoly_status spoly_solve(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q,
                         const spoly_chains* chains, const spoly_solve_opts* opts, spoly_solution_set** inout) {
  if (!ctx) return SPOLY_EINVAL;
  if (!chains || !opts || !inout) return fail(ctx, SPOLY_EINVAL, "chains, opts and inout are required");
  if (opts->precision != SPOLY_PLAIN_FP64 && opts->precision != SPOLY_MIXED)
    return fail(ctx, SPOLY_EINVAL, "unknown precision %d", opts->precision);
  CK(cudaSetDevice(ctx->device), "set device");
  MeshView mv;
  QueryView qv;
  spoly_status st = stage_inputs(ctx, mesh, q, &mv, &qv);
  if (st != SPOLY_OK) return st;
  if (!q->on_device) {
    for (int64_t i = 0; i < q->n_queries; ++i) {
      if (q->k[i] != 1 && q->k[i] != 2)
        return fail(ctx, SPOLY_EUNSUPPORTED, "query %lld has k = %d; k = 1 and 2 are built", (long long)i, q->k[i]);
      if (q->k[i] == 2 && q->types[2 * i] != q->types[2 * i + 1])
        return fail(ctx, SPOLY_EUNSUPPORTED, "query %lld: 2-bounce chains are built for types T T and R R",
                    (long long)i);
    }
  }
  spoly_solution_set* set = *inout;
  bool fresh = false;
  if (!set) {
    set = new (std::nothrow) spoly_solution_set();
    if (!set) return fail(ctx, SPOLY_ENOMEM, "solution set");
    fresh = true;
  }
  auto bail = [&](spoly_status s) {
    if (fresh) {
      set->queue.release();
      set->paths.release();
      set->side.release();
      set->counters.release();
      delete set;
    }
    return s;
  };
  const int64_t nc = chains->n;
  int64_t qcap = nc / 4 + 4096;
  if (int64_t(set->queue.bytes / sizeof(RootItem)) > qcap) qcap = int64_t(set->queue.bytes / sizeof(RootItem));
  int64_t pcap = opts->path_capacity > 0 ? opts->path_capacity : nc / 16 + 4096;
  if (int64_t(set->paths.bytes / sizeof(spoly_path)) > pcap) pcap = int64_t(set->paths.bytes / sizeof(spoly_path));
  int64_t scap = nc / 64 + 1024;
  if (int64_t(set->side.bytes / sizeof(int32_t)) > scap) scap = int64_t(set->side.bytes / sizeof(int32_t));
  if (set->side.ensure(size_t(scap) * sizeof(int32_t)) != cudaSuccess ||
      set->queue.ensure(size_t(qcap) * sizeof(RootItem)) != cudaSuccess ||
      set->paths.ensure(size_t(pcap) * sizeof(spoly_path)) != cudaSuccess ||
      set->counters.ensure(C_COUNT * sizeof(unsigned long long)) != cudaSuccess)
    return bail(fail(ctx, SPOLY_ENOMEM, "solution buffers"));
  set->queue_cap = qcap;
  set->path_cap = pcap;
  set->side_cap = scap;
  set->host_valid = false;
  set->n_k2 = 0;
  // split off the 2-bounce chains
  const int64_t n2 = chains->n_k2, n1 = nc - n2;
  const int32_t* k1_list = static_cast<const int32_t*>(chains->buf.p);
  const int32_t *k1_ids = nullptr, *k2_list = nullptr, *k2_ids = nullptr;
  if (n2 > 0) {
    if (set->part.ensure(size_t(nc) * 16) != cudaSuccess || set->part_n.ensure(16) != cudaSuccess)
      return bail(fail(ctx, SPOLY_ENOMEM, "chain partition"));
    int32_t* base = static_cast<int32_t*>(set->part.p);
    int32_t* a1 = base;
    int32_t* i1 = base + 3 * n1;
    int32_t* a2 = i1 + n1;
    int32_t* i2 = a2 + 3 * n2;
    k1_list = a1;
    k1_ids = i1;
    k2_list = a2;
    k2_ids = i2;
  }
  // the split of a mixed list into its 1- and 2-bounce parts (enqueued by
  // the staged solve below, or inside the captured graph)
  auto partition = [&]() -> cudaError_t {
    if (n2 == 0) return cudaSuccess;
    cudaError_t e0 = cudaMemsetAsync(set->part_n.p, 0, 16, ctx->stream);
    if (e0 == cudaSuccess)
      e0 = launch_partition(static_cast<const int32_t*>(chains->buf.p), nc, const_cast<int32_t*>(k1_list),
                            const_cast<int32_t*>(k1_ids), const_cast<int32_t*>(k2_list), const_cast<int32_t*>(k2_ids),
                            static_cast<unsigned long long*>(set->part_n.p), ctx->num_sms, ctx->stream);
    return e0;
  };
  K1Params P{};
  P.mesh = mv;
  P.qv = qv;
  if (opts->camera) {
    const double* c = opts->camera;
    P.pix.on = 1;
    for (int i = 0; i < 3; ++i) {
      P.pix.o[i] = c[i];
      P.pix.f[i] = c[3 + i];
      P.pix.r[i] = c[6 + i];
      P.pix.u[i] = c[9 + i];
    }
    P.pix.th = c[12];
    P.pix.aspect = c[13];
    P.pix.w = int(c[14]);
    P.pix.h = int(c[15]);
    P.pix.assign = (opts->flags & SPOLY_SOLVE_PIXEL_ASSIGN) ? 1 : 0;
    if (P.pix.w < 1 || P.pix.h < 1 || int64_t(P.pix.w) * P.pix.h != qv.n)
      return bail(fail(ctx, SPOLY_EINVAL, "pixel filter: width x height must equal n_queries"));
  } else if (opts->flags & SPOLY_SOLVE_PIXEL_ASSIGN) {
    return bail(fail(ctx, SPOLY_EINVAL, "SPOLY_SOLVE_PIXEL_ASSIGN needs a camera"));
  }
  P.chains = k1_list;
  P.chain_ids = k1_ids;
  P.n_chains = n1;
  P.counters = static_cast<unsigned long long*>(set->counters.p);
  cudaError_t e;
  const bool async = (opts->flags & SPOLY_SOLVE_ASYNC) != 0;
  const bool timing = (opts->flags & SPOLY_SOLVE_TIMING) != 0;
  if (timing && !set->ev[0])
    for (auto& ev : set->ev)
      if (cudaEventCreate(&ev) != cudaSuccess) return bail(fail(ctx, SPOLY_ECUDA, "event create"));
  set->timed = timing;
  auto bind = [&]() {
    P.queue = static_cast<RootItem*>(set->queue.p);
    P.queue_cap = set->queue_cap;
    P.side = static_cast<int32_t*>(set->side.p);
    P.side_cap = set->side_cap;
    P.paths = static_cast<spoly_path*>(set->paths.p);
    P.path_cap = set->path_cap;
  };
  auto read_counters = [&]() -> cudaError_t {
    cudaError_t r = cudaMemcpyAsync(set->host, set->counters.p, sizeof(set->host), cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (r == cudaSuccess) r = cudaStreamSynchronize(ctx->stream);
    return r;
  };
  const bool persistent = (opts->flags & SPOLY_SOLVE_PERSISTENT) != 0;
  // the side chains' FP64 solve runs on the context's second stream,
  // overlapping the polish of the bracket queue
  auto finish = [&]() -> cudaError_t {
    return launch_k1_finish(P, ctx->num_sms, ctx->stream, ctx->side_stream, ctx->fork_ev, ctx->join_ev);
  };
  auto isolate = [&]() -> cudaError_t {
    return persistent ? launch_k1_isolate_persistent(P, opts->precision, ctx->num_sms, ctx->tune, ctx->stream)
                      : launch_k1_isolate(P, opts->precision, ctx->num_sms, ctx->stream);
  };
  // Graph mode: replay the captured launch sequence when everything it baked
  // in is unchanged; otherwise capture it again.  A list with 2-bounce chains
  // takes the device-driven 2-bounce pass (no host read-back), whose scratch
  // is prepared before the capture.
  const bool tt_graph = n2 > 0 && tt_device_bytes(n2) <= kDeviceDrivenBytes;
  if ((opts->flags & SPOLY_SOLVE_GRAPH) && (n2 == 0 || tt_graph) && nc > 0) {
    if (!ctx->stream) return bail(fail(ctx, SPOLY_EINVAL, "graph mode needs a non-default stream"));
    bind();
    auto run_tt_device = [&](bool enqueue) -> spoly_status {
      return solve_tt_device(ctx, set, mv, qv, k2_list, k2_ids, n2, opts,
                             static_cast<unsigned long long*>(set->counters.p) + C_ADMISSIBLE,
                             static_cast<spoly_path*>(set->paths.p), set->path_cap, enqueue);
    };
    if (n2 > 0) {
      // sizes the 2-bounce scratch (and checks the options) outside the capture
      if (opts->sqrt_table) {
        const double* t = opts->sqrt_table;
        if (t[0] != 0.0 || t[kSqrtPieces] != 1.0) return bail(fail(ctx, SPOLY_EINVAL, "sqrt_table: breaks must run from 0 to 1"));
        for (int i = 0; i < kSqrtPieces; ++i)
          if (!(t[i + 1] > t[i])) return bail(fail(ctx, SPOLY_EINVAL, "sqrt_table: breaks must increase"));
      }
      if ((opts->n_intervals > 0 ? opts->n_intervals : 4096) > 8192)
        return bail(fail(ctx, SPOLY_EINVAL, "n_intervals %d exceeds 8192", opts->n_intervals));
      st = run_tt_device(false);
      if (st != SPOLY_OK) return bail(st);
    }
    uint64_t key[48] = {0};
    const void* ptrs[] = {P.chains, P.queue, P.side, P.paths, P.counters, mv.tri, qv.x_first, qv.x_last, qv.eta,
                          qv.types, qv.k};
    for (int i = 0; i < 11; ++i) key[i] = uint64_t(reinterpret_cast<uintptr_t>(ptrs[i]));
    key[11] = uint64_t(n1);
    key[12] = uint64_t(P.queue_cap);
    key[13] = uint64_t(P.side_cap);
    key[14] = uint64_t(P.path_cap);
    key[15] = uint64_t(opts->precision) | (uint64_t(persistent) << 8) | (uint64_t(P.pix.on) << 9) |
              (uint64_t(P.pix.assign) << 10);
    key[16] = uint64_t(ctx->tune.block) | (uint64_t(ctx->tune.blocks_per_sm) << 16) | (uint64_t(ctx->tune.chunk) << 32);
    key[17] = uint64_t(mv.n_tris);
    key[18] = uint64_t(qv.n);
    std::memcpy(&key[19], &P.pix.th, sizeof(double));
    std::memcpy(&key[20], &P.pix.o[0], sizeof(double));
    key[21] = uint64_t(reinterpret_cast<uintptr_t>(ctx->stream));
    key[22] = uint64_t(n2);
    if (n2 > 0) {
      const void* tptr[] = {set->part.p, set->tt_counters.p, set->tt_sys.p, set->tt_scratch.p, set->tt_coef32.p,
                            set->tt_queue.p, set->tt_noisy.p, set->tt_active.p, set->tt_offsets.p, set->tt_chain_sys.p,
                            set->tt_masks.p};
      for (int i = 0; i < 11; ++i) key[23 + i] = uint64_t(reinterpret_cast<uintptr_t>(tptr[i]));
      key[34] = uint64_t(opts->n_intervals);
      for (int i = 0; i < 13 && opts->sqrt_table; ++i) {
        double a = opts->sqrt_table[2 * i], b = (2 * i + 1 < 25) ? opts->sqrt_table[2 * i + 1] : 0.0;
        uint64_t ua, ub;
        std::memcpy(&ua, &a, 8);
        std::memcpy(&ub, &b, 8);
        key[35 + i] = ua ^ (ub * 0x9e3779b97f4a7c15ull);
      }
    }
    if (!set->gexec || std::memcmp(key, set->gkey, sizeof(key)) != 0) {
      if (set->gexec) cudaGraphExecDestroy(set->gexec);
      set->gexec = nullptr;
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "graph capture"));
      cudaError_t ec = cudaMemsetAsync(set->counters.p, 0, C_COUNT * sizeof(unsigned long long), ctx->stream);
      if (ec == cudaSuccess) ec = partition();
      if (ec == cudaSuccess && n1 > 0) ec = isolate();
      if (ec == cudaSuccess && n1 > 0) ec = finish();
      spoly_status tst = SPOLY_OK;
      if (ec == cudaSuccess && n2 > 0) tst = run_tt_device(true);
      e = cudaStreamEndCapture(ctx->stream, &graph);
      if (tst != SPOLY_OK) {
        if (graph) cudaGraphDestroy(graph);
        return bail(tst);
      }
      if (ec != cudaSuccess) e = ec;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&set->gexec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        set->gexec = nullptr;
        return bail(cuda_fail(ctx, e, "graph capture"));
      }
      std::memcpy(set->gkey, key, sizeof(key));
    }
    if (timing) cudaEventRecord(set->ev[0], ctx->stream);
    e = cudaGraphLaunch(set->gexec, ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "graph launch"));
    if (timing) {
      cudaEventRecord(set->ev[1], ctx->stream);
      cudaEventRecord(set->ev[2], ctx->stream);
      cudaEventRecord(set->ev[3], ctx->stream);
    }
    if (async) {
      *inout = set;
      return SPOLY_OK;
    }
    e = read_counters();
    if (e == cudaSuccess && n2 > 0) {
      e = cudaMemcpyAsync(set->tt_host, set->tt_counters.p, sizeof(set->tt_host), cudaMemcpyDeviceToHost, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    }
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "graph solve"));
    if (int64_t(set->host[C_QUEUED]) <= set->queue_cap && int64_t(set->host[C_SIDE]) <= set->side_cap &&
        int64_t(set->host[C_ADMISSIBLE]) <= set->path_cap) {
      set->host_valid = true;
      *inout = set;
      return SPOLY_OK;
    }
    set->tt_device = false;
    // a queue or the path buffer overflowed: the staged solve below grows them
    // (and the next graph call captures again)
  }
  set->tt_device = false;
  e = partition();
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "chain partition"));
  // Stage 1: isolation, and Stage 2: FP64 v-polish (in place, once) and the
  // path phase.  In synchronous mode the isolation is re-run until the
  // bracket queue and the side queue hold every item; each re-run grows them
  // to the exact counts, so two passes suffice.  A synchronous solve of
  // 1-bounce chains reads the counters once, after the finish (the finish
  // kernels take the item counts from the device and stop at the capacities,
  // and an overflowed pass is solved again from the start); with 2-bounce
  // chains they are read between the stages.
  const bool check_after_finish = !async && n2 == 0;
  bool finished = false, have_counters = false;
  for (int attempt = 0; attempt < 3; ++attempt) {
    bind();
    e = cudaMemsetAsync(set->counters.p, 0, C_COUNT * sizeof(unsigned long long), ctx->stream);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "memset"));
    if (timing) cudaEventRecord(set->ev[0], ctx->stream);
    if (n1 > 0) {
      e = isolate();
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "k1_isolate"));
    }
    if (timing) cudaEventRecord(set->ev[1], ctx->stream);
    if (async && n2 == 0) break;
    if (check_after_finish) {
      if (n1 > 0) {
        e = finish();
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "k1_polish"));
      }
      if (timing) cudaEventRecord(set->ev[2], ctx->stream);
      finished = true;
    }
    e = read_counters();
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "isolation"));
    have_counters = finished;
    const int64_t queued = int64_t(set->host[C_QUEUED]);
    const int64_t side = int64_t(set->host[C_SIDE]);
    if (queued <= set->queue_cap && side <= set->side_cap) break;
    finished = have_counters = false;
    if (attempt == 2) return bail(fail(ctx, SPOLY_ECAPACITY, "bracket queue did not converge"));
    if (side > set->side_cap) {
      if (set->side.ensure(size_t(side) * sizeof(int32_t)) != cudaSuccess)
        return bail(fail(ctx, SPOLY_ENOMEM, "side queue growth"));
      set->side_cap = side;
    }
    if (queued > set->queue_cap) {
      if (set->queue.ensure(size_t(queued) * sizeof(RootItem)) != cudaSuccess)
        return bail(fail(ctx, SPOLY_ENOMEM, "queue growth"));
      set->queue_cap = queued;
    }
  }
  // Only the path phase is re-run if the path buffer overflowed: it reads the
  // polished queue and is idempotent once its counters are reset.
  if (!finished) {
    if (n1 > 0) {
      e = finish();
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "k1_polish"));
    }
    if (timing) cudaEventRecord(set->ev[2], ctx->stream);
  }
  auto run_tt = [&]() -> spoly_status {
    if (n2 == 0) return SPOLY_OK;
    return solve_tt(ctx, set, mv, qv, k2_list, k2_ids, n2, opts,
                    static_cast<unsigned long long*>(set->counters.p) + C_ADMISSIBLE,
                    static_cast<spoly_path*>(set->paths.p), set->path_cap);
  };
  st = run_tt();
  if (st != SPOLY_OK) return bail(st);
  if (timing) cudaEventRecord(set->ev[3], ctx->stream);
  if (!async || n2 > 0) {
    if (!have_counters) {
      e = read_counters();
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "solve"));
    }
    const int64_t paths = int64_t(set->host[C_ADMISSIBLE]);
    if (paths > set->path_cap) {
      if (set->paths.ensure(size_t(paths) * sizeof(spoly_path)) != cudaSuccess)
        return bail(fail(ctx, SPOLY_ENOMEM, "path growth"));
      set->path_cap = paths;
      bind();
      for (int c : {int(C_UROOTS), int(C_FLAGGED), int(C_ADMISSIBLE)}) {
        e = cudaMemsetAsync(static_cast<unsigned long long*>(set->counters.p) + c, 0, sizeof(unsigned long long),
                            ctx->stream);
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "memset"));
      }
      if (n1 > 0) {
        P.rerun = 1;
        e = finish();
        P.rerun = 0;
        if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "k1_paths"));
      }
      st = run_tt();
      if (st != SPOLY_OK) return bail(st);
      e = read_counters();
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "solve"));
      if (int64_t(set->host[C_ADMISSIBLE]) > set->path_cap)
        return bail(fail(ctx, SPOLY_ECAPACITY, "path buffer did not converge"));
    }
    set->host_valid = true;
  }
  *inout = set;
  return SPOLY_OK;
}

spoly_status spoly_stats(spoly_ctx* ctx, const spoly_solution_set* set, spoly_counters* out) {
  if (!ctx) return SPOLY_EINVAL;
  if (!set || !out) return fail(ctx, SPOLY_EINVAL, "bad arguments");
  unsigned long long h[C_COUNT];
  CK(cudaMemcpyAsync(h, set->counters.p, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "stats");
  CK(cudaStreamSynchronize(ctx->stream), "stats sync");
  std::memset(out, 0, sizeof(*out));
  out->candidates = int64_t(h[C_CANDIDATES]);
  out->degenerate = int64_t(h[C_DEGENERATE]);
  out->v_roots = int64_t(h[C_VROOTS]);
  out->queued = int64_t(h[C_QUEUED]) + int64_t(h[C_SIDE_QUEUED]);
  out->prefiltered = int64_t(h[C_PREFILTERED]);
  out->polish_lost = int64_t(h[C_POLISH_LOST]);
  out->u_roots = int64_t(h[C_UROOTS]);
  out->admissible = int64_t(h[C_ADMISSIBLE]);
  out->flagged = int64_t(h[C_FLAGGED]);
  out->fallback = int64_t(h[C_SIDE]);
  unsigned long long tdev[16];
  if (set->n_k2 > 0 && set->tt_device) {  // device-driven pass: its counters are on the device
    CK(cudaMemcpyAsync(tdev, set->tt_counters.p, sizeof(tdev), cudaMemcpyDeviceToHost, ctx->stream), "stats");
    CK(cudaStreamSynchronize(ctx->stream), "stats sync");
  }
  if (set->n_k2 > 0) {  // 2-bounce chains of the same solve (their paths are already in admissible)
    const unsigned long long* t = set->tt_device ? tdev : set->tt_host;
    out->candidates += set->n_k2;
    out->degenerate += int64_t(t[TT_DEGENERATE]);
    out->v_roots += int64_t(t[TT_BRACKETS]);
    out->queued += int64_t(t[TT_BRACKETS]);
    out->polish_lost += int64_t(t[TT_POLISH_LOST]);
    out->u_roots += int64_t(t[TT_UROOTS]);
    out->flagged += int64_t(t[TT_FLAGGED]);
    out->unsolved = int64_t(t[TT_TOO_LARGE]);
    out->fallback += int64_t(t[TT_RESAMPLED]);
    out->k2_systems = int64_t(t[TT_SYSTEMS]);
    out->k2_evals = int64_t(t[TT_EVALS]);
    out->k2_eval_n3 = int64_t(t[TT_EVAL_N3]);
    out->k2_fp64_samples = int64_t(t[TT_FP64_SAMPLES]);
    out->k2_evals32 = int64_t(t[TT_EVALS32]);
    out->k2_eval32_n3 = int64_t(t[TT_EVAL32_N3]);
  }
  return SPOLY_OK;
}

spoly_status spoly_paths(spoly_ctx* ctx, const spoly_solution_set* set, spoly_path* dst, int64_t capacity,
                         int64_t* n_total, int32_t dst_is_device) {
  if (!ctx) return SPOLY_EINVAL;
  if (!set || !n_total || (!dst && capacity > 0)) return fail(ctx, SPOLY_EINVAL, "bad arguments");
  unsigned long long cnt = 0;
  CK(cudaMemcpyAsync(&cnt, static_cast<unsigned long long*>(set->counters.p) + C_ADMISSIBLE, 8,
                     cudaMemcpyDeviceToHost, ctx->stream),
     "path count");
  CK(cudaStreamSynchronize(ctx->stream), "path count sync");
  *n_total = int64_t(cnt);
  if (int64_t(cnt) > set->path_cap)
    return fail(ctx, SPOLY_ECAPACITY, "solution set overflowed (%lld paths, buffer %lld); re-run spoly_solve "
                "without SPOLY_SOLVE_ASYNC", (long long)cnt, (long long)set->path_cap);
  int64_t m = capacity < int64_t(cnt) ? capacity : int64_t(cnt);
  if (m > 0) {
    CK(cudaMemcpyAsync(dst, set->paths.p, size_t(m) * sizeof(spoly_path),
                       dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream),
       "path copy");
    CK(cudaStreamSynchronize(ctx->stream), "path copy sync");
  }
  if (capacity < int64_t(cnt))
    return fail(ctx, SPOLY_ECAPACITY, "paths: capacity %lld < %lld", (long long)capacity, (long long)cnt);
  return SPOLY_OK;
}

spoly_status spoly_phase_ms(spoly_ctx* ctx, const spoly_solution_set* set, float* ms, int32_t n) {
  if (!ctx) return SPOLY_EINVAL;
  if (!set || !ms || n < 2) return fail(ctx, SPOLY_EINVAL, "bad arguments");
  if (!set->timed) return fail(ctx, SPOLY_EINVAL, "the last solve did not set SPOLY_SOLVE_TIMING");
  CK(cudaEventSynchronize(set->ev[2]), "phase timing");
  CK(cudaEventElapsedTime(&ms[0], set->ev[0], set->ev[1]), "phase timing");
  CK(cudaEventElapsedTime(&ms[1], set->ev[1], set->ev[2]), "phase timing");
  if (n >= 3) {
    ms[2] = 0.0f;
    if (set->n_k2 > 0) CK(cudaEventElapsedTime(&ms[2], set->ev[2], set->ev[3]), "phase timing");
  }
  if (n >= 4) ms[3] = set->n_k2 > 0 ? set->tt_sign_ms : 0.0f;
  return SPOLY_OK;
}

spoly_status spoly_measure_peak(spoly_ctx* ctx, int32_t kind, double* tflops) {
  if (!ctx) return SPOLY_EINVAL;
  if (!tflops || (kind != SPOLY_PEAK_FP32_FMA && kind != SPOLY_PEAK_FP64_FMA))
    return fail(ctx, SPOLY_EINVAL, "bad arguments");
  CK(cudaSetDevice(ctx->device), "set device");
  cudaError_t e = cudaSuccess;
  *tflops = measure_fma_peak(kind, ctx->num_sms, ctx->stream, &e);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "peak microbenchmark");
  return SPOLY_OK;
}

spoly_status spoly_autotune(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q, const spoly_chains* chains,
                            int32_t precision, spoly_tune_entry* table, int32_t cap, int32_t* n_table,
                            spoly_tune_entry* best) {
  if (!ctx) return SPOLY_EINVAL;
  if (!chains || (cap > 0 && !table)) return fail(ctx, SPOLY_EINVAL, "autotune: bad arguments");
  if (precision != SPOLY_PLAIN_FP64 && precision != SPOLY_MIXED) return fail(ctx, SPOLY_EINVAL, "autotune: precision");
  if (chains->n_k2 > 0) return fail(ctx, SPOLY_EINVAL, "autotune: the chain list holds 2-bounce chains");
  if (chains->n <= 0) return fail(ctx, SPOLY_EINVAL, "autotune: no chains");
  CK(cudaSetDevice(ctx->device), "set device");
  MeshView mv;
  QueryView qv;
  spoly_status st = stage_inputs(ctx, mesh, q, &mv, &qv);
  if (st != SPOLY_OK) return st;
  const int64_t n = chains->n;
  DevBuf counters, queue, side;
  const int64_t qcap = n / 2 + 4096, scap = n / 16 + 1024;
  CK(counters.ensure(C_COUNT * sizeof(unsigned long long)), "autotune scratch");
  CK(queue.ensure(size_t(qcap) * sizeof(RootItem)), "autotune scratch");
  CK(side.ensure(size_t(scap) * sizeof(int32_t)), "autotune scratch");
  K1Params P{};
  P.mesh = mv;
  P.qv = qv;
  P.chains = static_cast<const int32_t*>(chains->buf.p);
  P.n_chains = n;
  P.counters = static_cast<unsigned long long*>(counters.p);
  P.queue = static_cast<RootItem*>(queue.p);
  P.queue_cap = qcap;
  P.side = static_cast<int32_t*>(side.p);
  P.side_cap = scap;
  cudaEvent_t a = nullptr, b = nullptr;
  CK(cudaEventCreate(&a), "autotune events");
  CK(cudaEventCreate(&b), "autotune events");
  spoly_tune_entry top{0, 0, 0, 3.0e38f};
  int32_t k = 0;
  cudaError_t e = cudaSuccess;
  for (int block : {64, 128})
    for (int bps : {1, 2, 4, 8})
      for (int chunk : {32, 64, 128, 256}) {
        K1Launch cfg;
        cfg.block = block;
        cfg.blocks_per_sm = bps;
        cfg.chunk = chunk;
        float bestms = 3.0e38f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first run warms up
          e = cudaMemsetAsync(counters.p, 0, C_COUNT * sizeof(unsigned long long), ctx->stream);
          if (e == cudaSuccess) e = cudaEventRecord(a, ctx->stream);
          if (e == cudaSuccess) e = launch_k1_isolate_persistent(P, precision, ctx->num_sms, cfg, ctx->stream);
          if (e == cudaSuccess) e = cudaEventRecord(b, ctx->stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(b);
          float ms = 0.0f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
          if (rep > 0) bestms = std::min(bestms, ms);
        }
        if (e != cudaSuccess) break;
        const spoly_tune_entry ent{block, bps, chunk, bestms};
        if (k < cap) table[k] = ent;
        ++k;
        if (bestms < top.ms) top = ent;
      }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  counters.release();
  queue.release();
  side.release();
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
  ctx->tune.block = top.block;
  ctx->tune.blocks_per_sm = top.blocks_per_sm;
  ctx->tune.chunk = top.chunk;
  if (n_table) *n_table = k;
  if (best) *best = top;
  return SPOLY_OK;
}

spoly_status spoly_solution_free(spoly_solution_set* set) {
  if (!set) return SPOLY_EINVAL;
  for (auto& ev : set->ev)
    if (ev) cudaEventDestroy(ev);
  for (auto& ev : set->tt_ev)
    if (ev) cudaEventDestroy(ev);
  set->side.release();
  set->queue.release();
  set->paths.release();
  set->counters.release();
  for (DevBuf* b : {&set->part, &set->part_n, &set->tt_counters, &set->tt_chain_sys, &set->tt_masks, &set->tt_sys,
                    &set->tt_scratch, &set->tt_coef32, &set->tt_queue, &set->tt_noisy, &set->tt_active,
                    &set->tt_offsets})
    b->release();
  if (set->gexec) cudaGraphExecDestroy(set->gexec);
  delete set;
  return SPOLY_OK;
}

}  // extern "C"
