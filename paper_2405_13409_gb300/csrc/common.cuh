// Shared device/host definitions of the GB300 specular-polynomial library.
#pragma once
#include <stdint.h>

#include "spoly.h"

#ifdef SPOLY_HOST_BUILD
// Host build of the per-candidate numerics (used by tests to run the kernels'
// arithmetic on the CPU); kernels and warp primitives are excluded.
#include <algorithm>
#include <cmath>
#define SPOLY_HD inline
#define SPOLY_D inline
#define __constant__
using std::fabs;
using std::fma;
using std::fmax;
using std::fmin;
using std::frexp;
using std::isfinite;
using std::ldexp;
using std::log2;
using std::max;
using std::min;
using std::sqrt;
template <typename T>
inline T __ldg(const T* p) { return *p; }
inline int __double2int_rn(double x) { return int(std::nearbyint(x)); }
inline int __popc(unsigned x) { return __builtin_popcount(x); }
#include <cstring>
inline long long __double_as_longlong(double x) {
  long long b;
  std::memcpy(&b, &x, 8);
  return b;
}
inline double __longlong_as_double(long long b) {
  double x;
  std::memcpy(&x, &b, 8);
  return x;
}
inline int __float2int_rn(float x) { return int(std::nearbyint(x)); }
#else
#include <cuda_runtime.h>
#define SPOLY_HD __host__ __device__ __forceinline__
#define SPOLY_D __device__ __forceinline__
#endif

namespace spoly {

// ---------------------------------------------------------------- vectors
struct d3 {
  double x, y, z;
};
SPOLY_HD d3 mk(double x, double y, double z) { return {x, y, z}; }
SPOLY_HD d3 operator+(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
SPOLY_HD d3 operator-(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
SPOLY_HD d3 operator*(double k, d3 a) { return {k * a.x, k * a.y, k * a.z}; }
SPOLY_HD double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
SPOLY_HD d3 cross(d3 a, d3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
SPOLY_HD double norm(d3 a) { return sqrt(dot(a, a)); }

// One triangle in the library's FP64 SoA mesh: rows p0xyz, p1xyz, p2xyz,
// n0xyz, n1xyz, n2xyz, each of length n_tris (Sec. 3.1, P_i and N_i).
struct TriD {
  d3 p0, p1, p2, n0, n1, n2;
};

SPOLY_D TriD load_tri(const double* __restrict__ soa, int64_t n_tris, int t) {
  auto g = [&](int row) { return __ldg(soa + int64_t(row) * n_tris + t); };
  TriD r;
  r.p0 = mk(g(0), g(1), g(2));
  r.p1 = mk(g(3), g(4), g(5));
  r.p2 = mk(g(6), g(7), g(8));
  r.n0 = mk(g(9), g(10), g(11));
  r.n1 = mk(g(12), g(13), g(14));
  r.n2 = mk(g(15), g(16), g(17));
  return r;
}

struct QueryD {
  d3 x0, x2;
  double eta0, eta1;
  int type;
};

SPOLY_D QueryD load_query(const double* __restrict__ xf, const double* __restrict__ xl,
                          const double* __restrict__ eta, const int32_t* __restrict__ types, int q) {
  QueryD r;
  r.x0 = mk(__ldg(xf + 3 * q), __ldg(xf + 3 * q + 1), __ldg(xf + 3 * q + 2));
  r.x2 = mk(__ldg(xl + 3 * q), __ldg(xl + 3 * q + 1), __ldg(xl + 3 * q + 2));
  r.eta0 = __ldg(eta + 3 * q);
  r.eta1 = __ldg(eta + 3 * q + 1);
  r.type = __ldg(types + 2 * q);
  return r;
}

// Device views of the caller's (or the library's staged) inputs.
struct MeshView {
  const double* tri;
  int64_t n_tris;
};
struct QueryView {
  const double* x_first;
  const double* x_last;
  const double* eta;
  const int32_t* types;
  const int32_t* k;
  int64_t n;
};

// ------------------------------------------- FP64 magnitude bookkeeping
// |x| as an integer that orders like |x| (non-NaN doubles), its binary
// exponent, and exact scaling by 2^k: integer-pipe replacements for
// fabs/fmax/frexp/ldexp, which would otherwise occupy the scarce FP64 pipe.
SPOLY_D long long absbits(double x) { return __double_as_longlong(x) & 0x7fffffffffffffffLL; }
SPOLY_D int expo_bits(long long ab) { return int(ab >> 52) - 1023; }
SPOLY_D double scale2(double x, int k) {
  const long long b = __double_as_longlong(x);
  const long long ab = b & 0x7fffffffffffffffLL;
  if (ab == 0) return x;
  const int e = int(ab >> 52) + k;
  if (e <= 0) return 0.0;  // would be subnormal: negligible at these scales
  return __longlong_as_double(b + ((long long)k << 52));
}

// ------------------------------------------------------------ constants
// Readings shared with the oracle's (they are restated, not shared: the
// oracle is a separate program).
constexpr double kDelta = 1e-6;      // v and u search domain [-kDelta, 1 + kDelta]
constexpr double kTrim = 1e-13;      // negligible u-power / leading coefficient
constexpr double kIllCond = 1e-8;    // |r'(v*)| / sum|r_i| below this: ILL_COND
constexpr double kResidual = 1e-9;   // admissible path-space residual
constexpr double kEdgeEps = 1e-7;    // EDGE flag band
constexpr double kSwitch = 0.25;     // projection switch threshold (R: edge, T: b)
constexpr double kNewtonMove = 1e-5; // accepted Newton move on (a, b)
constexpr int kNewtonIters = 3;
constexpr double kPolishTol = 1e-12; // FP64 polish bracket width in v
constexpr float kIsoTol32 = 1e-6f;   // FP32 isolation bracket width in v
constexpr double kIsoTol64 = 1e-12;  // FP64 isolation bracket width in v (plain mode)
constexpr double kPrefilterMargin = 0.1;  // u-range margin of the pre-polish filter
constexpr double kPrefilterDv = 1e-3;     // side samples (in v) of the pre-polish filter
constexpr double kSideReach = 0.25;       // side search reach (in v) of a displaced FP32 root
constexpr float kTangent32 = 1e-4f;  // tangent-root test, FP32 isolation
constexpr double kTangent64 = 1e-12; // tangent-root test, FP64 isolation
// Certification of the FP32 isolation (mixed precision).  A candidate is
// re-isolated in FP64 when its FP32 resultant r
//   - has a largest coefficient below kCert32Tiny (2^-100: partial products
//     of the expansion may have left FP32's exponent range),
//   - cancels by more than kCert32Cancel: sum_c R_c Z^c > kCert32Cancel *
//     sum_c |r_c| Z^c, where R is the same expansion over |E| with every term
//     added (the scale of its rounding errors),
//   - or comes within kCert32Dip * sum_c |r_c| Z^c of zero at a critical
//     point or at an end of the domain (a near-double root or an edge root,
//     which FP32 rounding can create, remove or move across the end).
constexpr float kCert32Tiny = 7.8886091e-31f;  // 2^-100
constexpr float kCert32Cancel = 1e9f;
constexpr float kCert32Dip = 1e-3f;

// Pinhole camera of a footprint workload, for the pixel filter of the path
// phase (layout of spoly_chain_opts::camera).
struct PixelFilter {
  int on;
  int assign;  // 1: a path's query becomes the pixel its first vertex projects into
  int w, h;
  double o[3], f[3], r[3], u[3], th, aspect;
};

// Pixel of a point seen by the camera; false if behind it.
SPOLY_HD bool project_pixel(const PixelFilter& C, double x, double y, double z, int64_t* pix) {
  const double dx = x - C.o[0], dy = y - C.o[1], dz = z - C.o[2];
  const double fz = dx * C.f[0] + dy * C.f[1] + dz * C.f[2];
  if (!(fz > 0.0)) return false;
  const double sx = (dx * C.r[0] + dy * C.r[1] + dz * C.r[2]) / (fz * C.th * C.aspect);
  const double sy = (dx * C.u[0] + dy * C.u[1] + dz * C.u[2]) / (fz * C.th);
  const double fx = (sx + 1.0) * 0.5 * C.w, fy = (1.0 - sy) * 0.5 * C.h;
  if (!(fx >= 0.0 && fx < C.w && fy >= 0.0 && fy < C.h)) return false;
  *pix = int64_t(floor(fy)) * C.w + int64_t(floor(fx));
  return true;
}

// Root-bracket queue item between the isolation and polish kernels.
struct RootItem {
  double zlo, zhi;   // bracket in the scaled hidden variable z = v / t
  int32_t chain;
  uint32_t flags;    // SPOLY_FLAG_TANGENT for critical-point roots
  float rscale;      // sum_i |p_i| t^-i of the isolated polynomial
  int32_t pad;
};
static_assert(sizeof(RootItem) == 32, "RootItem layout");

// Counter slots in the solution set's device counter array.
enum Counter {
  C_CANDIDATES = 0,
  C_DEGENERATE,
  C_VROOTS,       // roots isolated in [-delta, 1 + delta]
  C_QUEUED,       // brackets passed to the FP64 polish
  C_PREFILTERED,  // brackets dropped by the u-range pre-filter
  C_POLISH_LOST,  // brackets without an FP64 sign change
  C_UROOTS,
  C_ADMISSIBLE,
  C_FLAGGED,
  C_PATHS_WRITTEN,
  C_QUEUE_OVERFLOW,
  C_SIDE,         // chains sent to the generic-size kernel
  C_TICKET,       // work-queue ticket of the persistent isolation kernel
  C_SIDE_QUEUED,  // brackets of the side chains (polished in the side kernel)
  C_COUNT
};

#ifndef SPOLY_HOST_BUILD
// --------------------------------------------------------- warp helpers
// Appends `cnt` items per lane to a global array with one atomic per warp;
// returns this lane's first slot.  All lanes of the warp must call it.
SPOLY_D unsigned long long warp_append(unsigned long long* counter, unsigned cnt) {
  const unsigned lane = threadIdx.x & 31u;
  unsigned incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= unsigned(o)) incl += y;
  }
  const unsigned total = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31 && total) base = atomicAdd(counter, (unsigned long long)total);
  base = __shfl_sync(0xffffffffu, base, 31);
  return base + incl - cnt;
}

SPOLY_D void warp_count(unsigned long long* counter, unsigned cnt) {
  unsigned s = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31u) == 0 && s) atomicAdd(counter, (unsigned long long)s);
}
#endif

}  // namespace spoly
