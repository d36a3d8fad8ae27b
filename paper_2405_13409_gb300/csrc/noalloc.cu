// spoly_solve_noalloc: the 1-bounce solve for callers that cannot allocate.
//
// Some callers are not allowed to allocate device memory at all: code that
// runs where the allocator is off limits (a host callback or a real-time
// loop that must not block on cudaMalloc's implicit synchronisation), a
// plug-in living inside a host application that owns every byte of device
// memory, or a process whose memory pool is fixed up front.  For them this
// file keeps the solve's scratch (counters, bracket queue, side queue) in one
// file-scope device array that is part of the loaded library image.  Every
// GPU that loads the library holds that array until the process exits.
//
// The array is shared by all calls: each call clears the counters that must
// start at zero and overwrites the queues, so two calls whose work overlaps
// on the GPU (different streams, or different host threads without ordering)
// race on it and corrupt each other's results.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "k1.cuh"

namespace {

// Largest chain batch one call accepts.  A chain yields at most kItemsPerChain
// brackets (resultant degree 16 plus one tangent root), so the bracket queue
// below can never overflow for an accepted batch.
constexpr int64_t kMaxChains = 4096;
constexpr int64_t kItemsPerChain = 17;
constexpr size_t kCounterBytes = 256;  // spoly::C_COUNT counters, padded
constexpr size_t kQueueBytes = size_t(kMaxChains * kItemsPerChain) * sizeof(spoly::RootItem);
constexpr size_t kSideBytes = size_t(kMaxChains) * sizeof(int32_t);
constexpr size_t kScratchBytes = kCounterBytes + kQueueBytes + kSideBytes;  // about 2.2 MiB
static_assert(spoly::C_COUNT * sizeof(unsigned long long) <= kCounterBytes, "counter block");
static_assert(kQueueBytes % 256 == 0, "queue keeps the side queue 256-byte aligned");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Offset, inside the counter block, of the validation slot: the smallest
// (chain index << 8 | reason) over the caller's chains that fail the checks
// below, or all ones when every chain passes.
constexpr size_t kBadSlot = 248;
static_assert(spoly::C_COUNT * sizeof(unsigned long long) <= kBadSlot, "validation slot after the counters");
enum BadReason : unsigned { kBadQuery = 1, kBadTriangle = 2, kBadSecond = 3, kBadBounces = 4, kBadType = 5 };

// One thread per chain: the query and triangle indices lie in range, the
// chain has one bounce (tri1 < 0 and k[query] == 1) and a known type.  The
// indices are checked before anything is read through them.
__global__ void noalloc_validate_kernel(const int32_t* __restrict__ chains, int64_t n, int64_t n_queries,
                                        int64_t n_tris, const int32_t* __restrict__ k,
                                        const int32_t* __restrict__ types, unsigned long long* bad) {
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n; c += int64_t(gridDim.x) * blockDim.x) {
    const int32_t q = chains[3 * c], t = chains[3 * c + 1], t2 = chains[3 * c + 2];
    unsigned why = 0;
    if (q < 0 || q >= n_queries) why = kBadQuery;
    else if (t < 0 || t >= n_tris) why = kBadTriangle;
    else if (t2 >= 0) why = kBadSecond;
    else if (k[q] != 1) why = kBadBounces;
    else if (types[2 * q] != SPOLY_R && types[2 * q] != SPOLY_T) why = kBadType;
    if (why) atomicMin(bad, ((unsigned long long)c << 8) | why);
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_lock;
void* g_scratch_addr[kMaxDevices] = {nullptr};

void put_msg(char* msg, int32_t len, const char* text) {
  if (msg && len > 0) snprintf(msg, size_t(len), "%s", text);
}

}  // namespace

extern "C" spoly_status spoly_solve_noalloc(int device, void* cuda_stream, const double* tri, int64_t n_tris,
                                            const double* x_first, const double* x_last, const double* eta,
                                            const int32_t* types, const int32_t* k, int64_t n_queries,
                                            const int32_t* chains, int64_t n_chains, int32_t precision,
                                            spoly_path* paths, int64_t path_capacity, int64_t* n_paths, char* msg,
                                            int32_t msg_len) {
  put_msg(msg, msg_len, "");
  if (!tri || !x_first || !x_last || !eta || !types || !k || !n_paths || (!chains && n_chains > 0) ||
      (!paths && path_capacity > 0) || n_tris <= 0 || n_queries <= 0 || n_chains < 0 || path_capacity < 0) {
    put_msg(msg, msg_len, "spoly_solve_noalloc: null pointer or negative size");
    return SPOLY_EINVAL;
  }
  if (n_chains > kMaxChains) {
    char buf[160];
    snprintf(buf, sizeof(buf), "spoly_solve_noalloc: %lld chains exceed the static scratch limit of %lld per call",
             (long long)n_chains, (long long)kMaxChains);
    put_msg(msg, msg_len, buf);
    return SPOLY_EINVAL;
  }
  if (precision != SPOLY_PLAIN_FP64 && precision != SPOLY_MIXED) {
    put_msg(msg, msg_len, "spoly_solve_noalloc: unknown precision");
    return SPOLY_EINVAL;
  }
  if (device < 0 || device >= kMaxDevices) {
    put_msg(msg, msg_len, "spoly_solve_noalloc: bad device index");
    return SPOLY_EINVAL;
  }
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
    put_msg(msg, msg_len, "spoly_solve_noalloc: cannot select the device");
    return SPOLY_ECUDA;
  }
  auto done = [&](spoly_status st, const char* text) {
    if (text) put_msg(msg, msg_len, text);
    cudaSetDevice(prev);
    return st;
  };
  // One-time set-up per device, with that device current: the device address
  // of the static scratch array (host code cannot use the symbol itself).
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_setup_lock);
    if (!g_scratch_addr[device]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p)
        return done(SPOLY_ECUDA, "spoly_solve_noalloc: cudaGetSymbolAddress failed");
      g_scratch_addr[device] = p;
    }
    base = g_scratch_addr[device];
  }
  int num_sms = 0;
  if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
    return done(SPOLY_ECUDA, "spoly_solve_noalloc: device query failed");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* b = static_cast<unsigned char*>(base);
  spoly::K1Params P{};
  P.mesh = {tri, n_tris};
  P.qv = {x_first, x_last, eta, types, k, n_queries};
  P.chains = chains;
  P.n_chains = n_chains;
  P.counters = reinterpret_cast<unsigned long long*>(b);
  P.queue = reinterpret_cast<spoly::RootItem*>(b + kCounterBytes);
  P.queue_cap = kMaxChains * kItemsPerChain;
  P.side = reinterpret_cast<int32_t*>(b + kCounterBytes + kQueueBytes);
  P.side_cap = kMaxChains;
  P.paths = paths;
  P.path_cap = path_capacity;
  // The array keeps the previous call's contents: the counters must restart
  // at zero, the validation slot at all ones.
  unsigned long long* bad = reinterpret_cast<unsigned long long*>(b + kBadSlot);
  if (cudaMemsetAsync(P.counters, 0, kBadSlot, st) != cudaSuccess ||
      cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), st) != cudaSuccess)
    return done(SPOLY_ECUDA, "spoly_solve_noalloc: memset failed");
  if (n_chains > 0) {
    // Validate the caller's list before any kernel reads through its indices.
    const int64_t g = std::min<int64_t>((n_chains + 255) / 256, int64_t(num_sms) * 4);
    noalloc_validate_kernel<<<int(g), 256, 0, st>>>(chains, n_chains, n_queries, n_tris, k, types, bad);
    unsigned long long hbad = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return done(SPOLY_ECUDA, "spoly_solve_noalloc: validation failed to run");
    if (hbad != ~0ull) {
      static const char* what[] = {"", "query index out of range", "triangle index out of range",
                                   "a second triangle (only 1-bounce chains are solved here)",
                                   "a query with k != 1 (only 1-bounce chains are solved here)",
                                   "a query whose type is neither SPOLY_R nor SPOLY_T"};
      const unsigned why = unsigned(hbad & 0xffu);
      char buf[200];
      snprintf(buf, sizeof(buf), "spoly_solve_noalloc: chain %lld has %s", (long long)(hbad >> 8),
               why < 6 ? what[why] : "an invalid entry");
      return done(SPOLY_EINVAL, buf);
    }
  }
  if (n_chains > 0) {
    if (spoly::launch_k1_isolate(P, precision, num_sms, st) != cudaSuccess ||
        spoly::launch_k1_finish(P, num_sms, st, nullptr, nullptr, nullptr) != cudaSuccess)
      return done(SPOLY_ECUDA, "spoly_solve_noalloc: kernel launch failed");
  }
  unsigned long long count = 0;
  if (cudaMemcpyAsync(&count, P.counters + spoly::C_ADMISSIBLE, sizeof(count), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return done(SPOLY_ECUDA, "spoly_solve_noalloc: solve failed");
  *n_paths = int64_t(count);
  if (int64_t(count) > path_capacity)
    return done(SPOLY_ECAPACITY, "spoly_solve_noalloc: path buffer too small; *n_paths holds the required count");
  return done(SPOLY_OK, nullptr);
}
