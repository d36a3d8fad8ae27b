// Learned candidate gate: the per-candidate features and the layout of the
// BF16 network (not part of the paper; the features restate the specular
// constraint h x n = 0 of Eq. eq_ch at the triangle's vertices).
//
// The network maps 24 features (padded to 32) through three ReLU layers of
// width 64 to one logit.  The three weight matrices and every matrix-product
// operand are BF16, accumulation is FP32; biases, the output weights w4 and
// b4 are FP32.  A candidate is solved when its logit reaches the threshold.
#pragma once
#include <stdint.h>

#include "common.cuh"

namespace spoly {

constexpr int kFeat = 24;
constexpr int kFeatMinBary = 12;      // the smallest barycentric coordinate of the mismatch zero
constexpr float kGateInside = -0.02f;  // the gate passes chains whose mismatch zero lies inside (this slack)
constexpr int kIn = 32;
constexpr int kHid = 64;

// Flat FP32 parameter vector (row-major W[in][out]).
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kIn * kHid;
constexpr int kOffW2 = kOffB1 + kHid;
constexpr int kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid;
constexpr int kOffB3 = kOffW3 + kHid * kHid;
constexpr int kOffW4 = kOffB3 + kHid;
constexpr int kOffB4 = kOffW4 + kHid;
constexpr int kParams = kOffB4 + 1;

// Packed inference weights: the B operands of mma.m16n8k16 in fragment order
// ([k tile][n tile][lane] of two 32-bit registers), then the FP32 vectors.
constexpr int kFragW1 = (kIn / 16) * (kHid / 8) * 32 * 2;   // 32-bit words
constexpr int kFragW23 = (kHid / 16) * (kHid / 8) * 32 * 2;
constexpr int kPackB = kFragW1 + 2 * kFragW23;              // word offset of b1
constexpr int kPackWords = kPackB + 4 * kHid + 4;           // b1 b2 b3 w4, b4 (+pad)
static_assert(kPackWords % 4 == 0, "packed weights are copied as 16-byte vectors");

// ----------------------------------------------------------- FP32 vectors
struct f3 {
  float x, y, z;
};
SPOLY_D f3 operator+(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
SPOLY_D f3 operator-(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
SPOLY_D f3 operator*(float k, f3 a) { return {k * a.x, k * a.y, k * a.z}; }
SPOLY_D float dotf(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
SPOLY_D f3 crossf(f3 a, f3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

#ifdef SPOLY_HOST_BUILD
inline float rsq(float x) { return 1.0f / std::sqrt(x); }
inline float d2f(double x) { return float(x); }
#else
SPOLY_D float rsq(float x) { return rsqrtf(x); }
// FP64 -> FP32 with integer instructions (round half up on the first dropped
// bit; magnitudes below 2^-126 become zero), so that the 27 conversions per
// candidate stay off the narrow FP64 pipe of this part.
SPOLY_D float d2f(double x) {
  const long long b = __double_as_longlong(x);
  const unsigned hi = unsigned((unsigned long long)b >> 32), lo = unsigned(b);
  const int e = int((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(hi & 0x80000000u);
  unsigned f = (hi & 0x80000000u) | (unsigned(e) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  f += (lo >> 28) & 1u;
  return __uint_as_float(f);
}
#endif

SPOLY_D f3 unitf(f3 v) { return rsq(fmaxf(dotf(v, v), 1e-37f)) * v; }

SPOLY_D f3 ld3(const double* p, int64_t stride, int row, int64_t t) {
  return {d2f(p[int64_t(row) * stride + t]), d2f(p[int64_t(row + 1) * stride + t]),
          d2f(p[int64_t(row + 2) * stride + t])};
}

// Generalised half vector at p, normalised: eta0 w0 + eta1 w2 with w the
// unit directions from p to the endpoints (Sec. 3.5; reflection: eta = 1).
SPOLY_D f3 half_dir(f3 x0, f3 x2, f3 p, float e0, float e1) {
  return unitf(e0 * unitf(x0 - p) + e1 * unitf(x2 - p));
}

// The 24 features of one candidate (definitions in the gate oracle):
//   0-5 mismatch d_i / S, 6-8 cross products / S^2, 9-11 barycentrics of
//   the mismatch's zero (clamped), 12 their minimum, 13 log2(S) / 8,
//   14 s n_c . h_c, 15-20 vertex offsets / L, 21 log2(L / |x0 - c|) / 8,
//   22 h_c . unit(x0 - c), 23 type.
SPOLY_D void gate_features(f3 x0, f3 x2, float e0, float e1, int type, const f3 (&P)[3], const f3 (&N)[3],
                            float (&f)[kFeat]) {
  if (type != SPOLY_T) e0 = e1 = 1.0f;
  const f3 c = (1.0f / 3.0f) * (P[0] + P[1] + P[2]);
  const f3 hc = half_dir(x0, x2, c, e0, e1);
  const f3 edge = P[1] - P[0];
  const f3 t1 = unitf(edge - dotf(edge, hc) * hc);
  const f3 t2 = crossf(hc, t1);
  f3 nh[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) nh[i] = unitf(N[i]);
  const f3 nc = unitf(nh[0] + nh[1] + nh[2]);
  const float s = dotf(nc, hc) >= 0.0f ? 1.0f : -1.0f;
  float dx[3], dy[3];
  float S2 = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const f3 d = s * nh[i] - half_dir(x0, x2, P[i], e0, e1);
    dx[i] = dotf(d, t1);
    dy[i] = dotf(d, t2);
    S2 = fmaxf(S2, dx[i] * dx[i] + dy[i] * dy[i]);
  }
  const float rS = rsq(fmaxf(S2, 1e-37f));
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dx[i] *= rS;
    dy[i] *= rS;
    f[2 * i] = dx[i];
    f[2 * i + 1] = dy[i];
  }
  const float c01 = dx[0] * dy[1] - dy[0] * dx[1];
  const float c12 = dx[1] * dy[2] - dy[1] * dx[2];
  const float c20 = dx[2] * dy[0] - dy[2] * dx[0];
  f[6] = c01;
  f[7] = c12;
  f[8] = c20;
  const float D = c01 + c12 + c20;
  float l0 = 0.0f, l1 = 0.0f, l2 = 0.0f;
  if (fabsf(D) > 1e-6f) {
    const float rD = 1.0f / D;
    l0 = fminf(fmaxf(c12 * rD, -4.0f), 4.0f);
    l1 = fminf(fmaxf(c20 * rD, -4.0f), 4.0f);
    l2 = fminf(fmaxf(c01 * rD, -4.0f), 4.0f);
  }
  f[9] = l0;
  f[10] = l1;
  f[11] = l2;
  f[12] = fminf(l0, fminf(l1, l2));
  f[13] = -0.0625f * log2f(fmaxf(rS * rS, 1e-37f));  // log2(S) / 8
  f[14] = s * dotf(nc, hc);
  const f3 e01 = P[1] - P[0], e12 = P[2] - P[1], e20 = P[0] - P[2];
  const float L2 = fmaxf(fmaxf(dotf(e01, e01), dotf(e12, e12)), fmaxf(dotf(e20, e20), 1e-37f));
  const float rL = rsq(L2);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const f3 r = P[i] - c;
    f[15 + 2 * i] = dotf(r, t1) * rL;
    f[16 + 2 * i] = dotf(r, t2) * rL;
  }
  const f3 w0 = x0 - c;
  const float W2 = fmaxf(dotf(w0, w0), 1e-37f);
  f[21] = 0.0625f * log2f(L2 / W2);  // log2(L / |x0 - c|) / 8
  f[22] = dotf(hc, rsq(W2) * w0);
  f[23] = type == SPOLY_T ? 1.0f : 0.0f;
}

// A query's endpoints, IORs and type in FP32, kept by a thread across the
// chains it takes (consecutive chains usually share their query: every chain
// of the distinct-triangle glint list does).
struct QueryF {
  int q = -1;
  f3 x0, x2;
  float e0, e1;
  int type;
};

SPOLY_D void load_query_f(const QueryView& qv, int q, QueryF& c) {
  if (q == c.q) return;
  c.q = q;
  c.x0 = {d2f(qv.x_first[3 * q]), d2f(qv.x_first[3 * q + 1]), d2f(qv.x_first[3 * q + 2])};
  c.x2 = {d2f(qv.x_last[3 * q]), d2f(qv.x_last[3 * q + 1]), d2f(qv.x_last[3 * q + 2])};
  c.e0 = d2f(qv.eta[3 * q]);
  c.e1 = d2f(qv.eta[3 * q + 1]);
  c.type = qv.types[2 * q];
}

// Features of chain `i` = (query, tri0, tri1) of a 1-bounce problem.
SPOLY_D void chain_features(const MeshView& mesh, const QueryView& qv, const int32_t* chains, int64_t i,
                             float (&f)[kFeat], QueryF& qc) {
  const int q = chains[3 * i];
  const int64_t t = chains[3 * i + 1];
  const int64_t T = mesh.n_tris;
  f3 P[3], N[3];
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    P[v] = ld3(mesh.tri, T, 3 * v, t);
    N[v] = ld3(mesh.tri, T, 9 + 3 * v, t);
  }
  load_query_f(qv, q, qc);
  gate_features(qc.x0, qc.x2, qc.e0, qc.e1, qc.type, P, N, f);
}

SPOLY_D void chain_features(const MeshView& mesh, const QueryView& qv, const int32_t* chains, int64_t i,
                             float (&f)[kFeat]) {
  QueryF qc;
  chain_features(mesh, qv, chains, i, f, qc);
}

}  // namespace spoly
