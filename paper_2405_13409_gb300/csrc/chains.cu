// Candidate chain construction: ALL, EXPLICIT and the conservative CONE cull.
//
// The paper takes its triangle tuples from an external pruning step (Sec. 3.1
// and Sec. 5 cite a path-space hierarchy with interval-arithmetic bounds).
// CONE stands in for it: a pair (query, triangle) survives only if the box of
// outgoing unit directions over the triangle (reflected or refracted per the
// query, by interval arithmetic over the triangle's bounding box and vertex
// normal range) overlaps the box of unit directions from the triangle's
// bounding box toward x_{k+1}.  Any solution x1 has its outgoing direction in
// both boxes, so the test never discards an admissible path (margin absorbs
// FP rounding).
#include "k1.cuh"

namespace spoly {

namespace {

struct Iv {
  double lo, hi;
};
SPOLY_D Iv iv(double a, double b) { return {fmin(a, b), fmax(a, b)}; }
SPOLY_D Iv operator+(Iv a, Iv b) { return {a.lo + b.lo, a.hi + b.hi}; }
SPOLY_D Iv operator-(Iv a, Iv b) { return {a.lo - b.hi, a.hi - b.lo}; }
SPOLY_D Iv operator*(Iv a, Iv b) {
  const double p1 = a.lo * b.lo, p2 = a.lo * b.hi, p3 = a.hi * b.lo, p4 = a.hi * b.hi;
  return {fmin(fmin(p1, p2), fmin(p3, p4)), fmax(fmax(p1, p2), fmax(p3, p4))};
}
SPOLY_D Iv scal(double k, Iv a) { return iv(k * a.lo, k * a.hi); }
SPOLY_D Iv sqr(Iv a) {
  if (a.lo >= 0.0) return {a.lo * a.lo, a.hi * a.hi};
  if (a.hi <= 0.0) return {a.hi * a.hi, a.lo * a.lo};
  return {0.0, fmax(a.lo * a.lo, a.hi * a.hi)};
}
// a / L with L = [llo, lhi], llo > 0.
SPOLY_D Iv divpos(Iv a, double llo, double lhi) {
  if (a.lo >= 0.0) return {a.lo / lhi, a.hi / llo};
  if (a.hi <= 0.0) return {a.lo / llo, a.hi / lhi};
  return {a.lo / llo, a.hi / llo};
}
SPOLY_D Iv widen(Iv a, double m) { return {fmax(-1.0, a.lo - m), fmin(1.0, a.hi + m)}; }

struct Iv3 {
  Iv x, y, z;
};

// Unit-vector box of a vector box (false if the box touches the origin).
SPOLY_D bool normalise(const Iv3& v, Iv3& out) {
  const Iv l2 = sqr(v.x) + sqr(v.y) + sqr(v.z);
  if (!(l2.lo > 0.0)) return false;
  const double llo = sqrt(l2.lo), lhi = sqrt(l2.hi);
  out = {divpos(v.x, llo, lhi), divpos(v.y, llo, lhi), divpos(v.z, llo, lhi)};
  return true;
}

// Outgoing-direction box of one triangle lit from x0; returns false when no
// bound is available (grazing or degenerate), true with `empty` set when no
// transmitted direction exists anywhere (total internal reflection).
SPOLY_D bool out_box(const MeshView& M, int t, d3 x0, int type, double eta0, double eta1, Iv3& o, Iv3& bb,
                     bool& empty) {
  empty = false;
  auto g = [&](int row) { return M.tri[int64_t(row) * M.n_tris + t]; };
  double p[3][3], n[3][3];
  for (int v = 0; v < 3; ++v)
    for (int c = 0; c < 3; ++c) {
      p[v][c] = g(3 * v + c);
      n[v][c] = g(9 + 3 * v + c);
    }
  Iv P[3], N[3];
  for (int c = 0; c < 3; ++c) {
    P[c] = {fmin(p[0][c], fmin(p[1][c], p[2][c])), fmax(p[0][c], fmax(p[1][c], p[2][c]))};
    N[c] = {fmin(n[0][c], fmin(n[1][c], n[2][c])), fmax(n[0][c], fmax(n[1][c], n[2][c]))};
  }
  bb = {P[0], P[1], P[2]};
  const Iv3 d = {P[0] - Iv{x0.x, x0.x}, P[1] - Iv{x0.y, x0.y}, P[2] - Iv{x0.z, x0.z}};
  Iv3 dh, nh;
  if (!normalise(d, dh)) return false;
  if (!normalise({N[0], N[1], N[2]}, nh)) return false;
  Iv c = dh.x * nh.x + dh.y * nh.y + dh.z * nh.z;
  c = {-c.hi, -c.lo};  // c = -d^ . n^
  if (c.hi < 0.0) {    // normal points away from x0: flip it
    nh = {{-nh.x.hi, -nh.x.lo}, {-nh.y.hi, -nh.y.lo}, {-nh.z.hi, -nh.z.lo}};
    c = {-c.hi, -c.lo};
  } else if (!(c.lo > 0.0)) {
    return false;  // grazing somewhere on the triangle
  }
  c.hi = fmin(c.hi, 1.0);
  if (type == SPOLY_R) {
    const Iv c2 = scal(2.0, c);
    o = {dh.x + c2 * nh.x, dh.y + c2 * nh.y, dh.z + c2 * nh.z};
  } else {
    const double eta = eta0 / eta1;
    const Iv k = {1.0 - eta * eta * (1.0 - c.lo * c.lo), 1.0 - eta * eta * (1.0 - c.hi * c.hi)};
    if (k.hi < 0.0) {
      empty = true;
      return true;
    }
    const Iv sk = {sqrt(fmax(k.lo, 0.0)), sqrt(k.hi)};
    const Iv f = scal(eta, c) - sk;
    o = {scal(eta, dh.x) + f * nh.x, scal(eta, dh.y) + f * nh.y, scal(eta, dh.z) + f * nh.z};
  }
  return true;
}

__global__ void shared_x0_kernel(QueryView Q, int32_t* flag) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < Q.n; q += stride) {
    bool same = true;
    for (int c = 0; c < 3; ++c) same &= Q.x_first[3 * q + c] == Q.x_first[c];
    same &= Q.eta[3 * q] == Q.eta[0] && Q.eta[3 * q + 1] == Q.eta[1] && Q.types[2 * q] == Q.types[0];
    same &= Q.k[q] == 1;
    if (!same) atomicExch(flag, 0);
  }
}

// Per-triangle boxes for queries sharing x0, eta and type: [t][12] floats
// (outgoing lo/hi xyz, bbox lo/hi xyz), rounded outward.  A triangle with no
// bound gets the full box; one with no transmitted direction an empty box.
__global__ void tri_boxes_kernel(ChainParams P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.tri_count) return;
  const int t = P.tri_begin + i;
  const d3 x0 = mk(P.qv.x_first[0], P.qv.x_first[1], P.qv.x_first[2]);
  Iv3 o, bb;
  bool empty = false;
  const bool ok = out_box(P.mesh, t, x0, P.qv.types[0], P.qv.eta[0], P.qv.eta[1], o, bb, empty);
  float* B = P.boxes + int64_t(i) * 12;
  const Iv comps[3] = {o.x, o.y, o.z};
  const Iv bcomp[3] = {bb.x, bb.y, bb.z};
  for (int c = 0; c < 3; ++c) {
    if (empty) {
      B[c] = 2.0f;
      B[3 + c] = -2.0f;
    } else if (!ok) {
      B[c] = -1.0f;
      B[3 + c] = 1.0f;
    } else {
      const Iv w = widen(comps[c], P.margin);
      B[c] = __double2float_rd(w.lo);
      B[3 + c] = __double2float_ru(w.hi);
    }
    B[6 + c] = __double2float_rd(bcomp[c].lo);
    B[9 + c] = __double2float_ru(bcomp[c].hi);
  }
}

// Unit-direction box from the triangle's bounding box toward a box of
// endpoints [x2l, x2h] x [y2l, y2h] x [z2l, z2h] (a point when l = h), in
// FP32 with a relative slack, tested against the outgoing-direction box.
SPOLY_D bool box_overlaps(const float* B, float x2l, float x2h, float y2l, float y2h, float z2l, float z2h) {
  const float xl = x2l - B[9], xh = x2h - B[6];
  const float yl = y2l - B[10], yh = y2h - B[7];
  const float zl = z2l - B[11], zh = z2h - B[8];
  auto s2lo = [](float lo, float hi) { return lo >= 0.f ? lo * lo : (hi <= 0.f ? hi * hi : 0.f); };
  auto s2hi = [](float lo, float hi) { return fmaxf(lo * lo, hi * hi); };
  const float l2lo = s2lo(xl, xh) + s2lo(yl, yh) + s2lo(zl, zh);
  const float l2hi = s2hi(xl, xh) + s2hi(yl, yh) + s2hi(zl, zh);
  if (!(l2lo > 0.f)) return true;
  const float ilo = rsqrtf(l2hi) * (1.f - 1e-5f), ihi = rsqrtf(l2lo) * (1.f + 1e-5f);
  auto dlo = [&](float lo, float hi) { return lo >= 0.f ? lo * ilo : lo * ihi; };
  auto dhi = [&](float lo, float hi) { return hi >= 0.f ? hi * ihi : hi * ilo; };
  const float sl = 1e-5f;
  bool ok = true;
  ok &= dlo(xl, xh) - sl <= B[3] && B[0] <= dhi(xl, xh) + sl;
  ok &= dlo(yl, yh) - sl <= B[4] && B[1] <= dhi(yl, yh) + sl;
  ok &= dlo(zl, zh) - sl <= B[5] && B[2] <= dhi(zl, zh) + sl;
  return ok;
}

SPOLY_D bool to_box_overlaps(const float* B, float x2, float y2, float z2) {
  return box_overlaps(B, x2, x2, y2, y2, z2, z2);
}

// Pair test over a tile: each thread owns one query, the block walks a chunk
// of triangles staged in shared memory.  A triangle is first tested once
// against the bounding box of the block's endpoints (a conservative superset
// of its pair tests); only triangles that pass are tested pair by pair.
// Survivors are appended with one atomic per warp per triangle.
constexpr int kConeThreads = 128;
constexpr int kConeTris = 256;

__global__ void __launch_bounds__(kConeThreads) cone_pairs_kernel(ChainParams P, int tris_per_block) {
  __shared__ float sbox[kConeTris][12];
  __shared__ int slist[kConeTris];
  __shared__ int scount;
  __shared__ float sred[6][kConeThreads / 32];
  const int64_t q = int64_t(blockIdx.x) * kConeThreads + threadIdx.x;
  const bool qok = q < P.qv.n;
  float x2 = 0.f, y2 = 0.f, z2 = 0.f;
  if (qok) {
    x2 = float(P.qv.x_last[3 * q]);
    y2 = float(P.qv.x_last[3 * q + 1]);
    z2 = float(P.qv.x_last[3 * q + 2]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // bounding box of the block's endpoints
  float v[6] = {qok ? x2 : 3e38f, qok ? -x2 : 3e38f, qok ? y2 : 3e38f, qok ? -y2 : 3e38f,
                qok ? z2 : 3e38f, qok ? -z2 : 3e38f};
#pragma unroll
  for (int c = 0; c < 6; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[c] = fminf(v[c], __shfl_xor_sync(0xffffffffu, v[c], o));
    if (lane == 0) sred[c][warp] = v[c];
  }
  __syncthreads();
  float tb[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    float m = sred[c][0];
#pragma unroll
    for (int w = 1; w < kConeThreads / 32; ++w) m = fminf(m, sred[c][w]);
    tb[c] = m;
  }
  const int t_begin = blockIdx.y * tris_per_block;
  const int t_end = min(P.tri_count, t_begin + tris_per_block);
  for (int t0 = t_begin; t0 < t_end; t0 += kConeTris) {
    const int nt = min(kConeTris, t_end - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < nt * 12; k += kConeThreads) sbox[k / 12][k % 12] = P.boxes[int64_t(t0) * 12 + k];
    if (threadIdx.x == 0) scount = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < nt; k += kConeThreads)
      if (box_overlaps(sbox[k], tb[0], -tb[1], tb[2], -tb[3], tb[4], -tb[5])) slist[atomicAdd(&scount, 1)] = k;
    __syncthreads();
    const int ns = scount;
    for (int idx = 0; idx < ns; ++idx) {
      const int k = slist[idx];
      const bool keep = qok && to_box_overlaps(sbox[k], x2, y2, z2);
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (!m) continue;
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(P.count, (unsigned long long)__popc(m));
      base = __shfl_sync(0xffffffffu, base, 0);
      if (keep) {
        const unsigned long long idx2 = base + __popc(m & ((1u << lane) - 1u));
        if (idx2 < (unsigned long long)P.cap) {
          P.out[3 * idx2] = int32_t(q);
          P.out[3 * idx2 + 1] = P.tri_begin + t0 + k;
          P.out[3 * idx2 + 2] = -1;
        }
      }
    }
  }
}

// General pair test for queries that do not share x0 / eta / type: the
// outgoing box is recomputed per pair in FP64.
__global__ void cone_pairs_general_kernel(ChainParams P) {
  const int64_t n = P.qv.n * int64_t(P.tri_count);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t c = base + lane;
    bool keep = false;
    int64_t q = 0;
    int t = 0;
    if (c < n) {
      q = c % P.qv.n;
      t = P.tri_begin + int(c / P.qv.n);
      if (P.qv.k[q] == 1) {
        Iv3 o, bb;
        bool empty = false;
        const d3 x0 = mk(P.qv.x_first[3 * q], P.qv.x_first[3 * q + 1], P.qv.x_first[3 * q + 2]);
        const bool ok = out_box(P.mesh, t, x0, P.qv.types[2 * q], P.qv.eta[3 * q], P.qv.eta[3 * q + 1], o, bb, empty);
        float B[12];
        const Iv comps[3] = {o.x, o.y, o.z};
        const Iv bcomp[3] = {bb.x, bb.y, bb.z};
        for (int k = 0; k < 3; ++k) {
          const Iv w = widen(comps[k], P.margin);
          B[k] = empty ? 2.f : (ok ? __double2float_rd(w.lo) : -1.f);
          B[3 + k] = empty ? -2.f : (ok ? __double2float_ru(w.hi) : 1.f);
          B[6 + k] = __double2float_rd(bcomp[k].lo);
          B[9 + k] = __double2float_ru(bcomp[k].hi);
        }
        keep = to_box_overlaps(B, float(P.qv.x_last[3 * q]), float(P.qv.x_last[3 * q + 1]),
                               float(P.qv.x_last[3 * q + 2]));
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) continue;
    unsigned long long b0 = 0;
    if (lane == 0) b0 = atomicAdd(P.count, (unsigned long long)__popc(m));
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (keep) {
      const unsigned long long idx = b0 + __popc(m & ((1u << lane) - 1u));
      if (idx < (unsigned long long)P.cap) {
        P.out[3 * idx] = int32_t(q);
        P.out[3 * idx + 1] = t;
        P.out[3 * idx + 2] = -1;
      }
    }
  }
}

__global__ void chains_all_kernel(ChainParams P) {
  const int64_t n = P.qv.n * int64_t(P.tri_count);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n; c += stride) {
    P.out[3 * c] = int32_t(c % P.qv.n);
    P.out[3 * c + 1] = P.tri_begin + int32_t(c / P.qv.n);
    P.out[3 * c + 2] = -1;
  }
}

__global__ void chains_explicit_kernel(ChainParams P, const int32_t* src, int64_t n) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t c = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; c < n; c += stride) {
    const int32_t q = src[3 * c], t0 = src[3 * c + 1], t1 = src[3 * c + 2];
    const bool ok = q >= 0 && q < P.qv.n && t0 >= 0 && t0 < P.mesh.n_tris && t1 >= -1 && t1 < P.mesh.n_tris;
    if (!ok) atomicCAS(P.error, 0, int32_t(c < 0x7ffffffe ? c + 1 : 0x7fffffff));
    P.out[3 * c] = ok ? q : 0;
    P.out[3 * c + 1] = ok ? t0 : 0;
    P.out[3 * c + 2] = ok ? t1 : -1;
    if (ok && t1 >= 0) atomicAdd(P.count, 1ull);  // 2-bounce chains
  }
}

}  // namespace

cudaError_t launch_chains_all(const ChainParams& P, int num_sms, cudaStream_t st) {
  chains_all_kernel<<<num_sms * 8, 256, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_chains_explicit(const ChainParams& P, const int32_t* src, int64_t n, int num_sms,
                                   cudaStream_t st) {
  chains_explicit_kernel<<<num_sms * 8, 256, 0, st>>>(P, src, n);
  return cudaGetLastError();
}

__global__ void set_flag_kernel(int32_t* flag, int32_t value) { *flag = value; }

cudaError_t launch_chains_cone(const ChainParams& P, int num_sms, cudaStream_t st) {
  // flag := 1, then cleared by any query that differs from query 0 in x0,
  // eta or type; the host reads it once to pick the pair-test variant.
  set_flag_kernel<<<1, 1, 0, st>>>(P.shared_x0, 1);
  shared_x0_kernel<<<num_sms * 4, 256, 0, st>>>(P.qv, P.shared_x0);
  int32_t h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, P.shared_x0, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return e;
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  if (h) {
    tri_boxes_kernel<<<(P.tri_count + 127) / 128, 128, 0, st>>>(P);
    const int tris_per_block = 1024;
    dim3 grid((unsigned)((P.qv.n + kConeThreads - 1) / kConeThreads),
              (unsigned)((P.tri_count + tris_per_block - 1) / tris_per_block));
    cone_pairs_kernel<<<grid, kConeThreads, 0, st>>>(P, tris_per_block);
  } else {
    cone_pairs_general_kernel<<<num_sms * 8, 256, 0, st>>>(P);
  }
  return cudaGetLastError();
}

namespace {

// ------------------------------------------- 2-bounce (TT, RR) cone cull
// For chains x0 -> T1 -> T2 -> x3 of two refractions or two reflections.
// Every path's segment direction unit(x2 - x1) lies in (i) T1's
// refracted (reflected) direction box from x0
// (forward), (ii) the unit box from T1's bounding box toward T2's, and
// (iii) the negated refracted-direction box of T2 seen from x3 with the
// indices swapped (backward: light from x3 refracted into the slab), which
// also points from T2's bounding box toward T1's.  Pairs failing any of
// these are dropped; (i) and (ii) do not depend on the receiver.

// Forward boxes of the first range: [n1][12] as tri_boxes_kernel writes.
__global__ void tt_fwd_boxes_kernel(TTConeParams P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n1) return;
  const int t = P.t1_begin + i;
  const d3 x0 = mk(P.qv.x_first[0], P.qv.x_first[1], P.qv.x_first[2]);
  Iv3 o, bb;
  bool empty = false;
  const bool ok = out_box(P.mesh, t, x0, P.qv.types[0], P.qv.eta[0], P.qv.eta[1], o, bb, empty);
  float* B = P.fwd + int64_t(i) * 12;
  const Iv comps[3] = {o.x, o.y, o.z};
  const Iv bcomp[3] = {bb.x, bb.y, bb.z};
  for (int c = 0; c < 3; ++c) {
    const Iv w = widen(comps[c], P.margin);
    B[c] = empty ? 2.f : (ok ? __double2float_rd(w.lo) : -1.f);
    B[3 + c] = empty ? -2.f : (ok ? __double2float_ru(w.hi) : 1.f);
    B[6 + c] = __double2float_rd(bcomp[c].lo);
    B[9 + c] = __double2float_ru(bcomp[c].hi);
  }
}

// Pairs (T1, T2) that pass (i) and (ii).
__global__ void tt_pairs_kernel(TTConeParams P) {
  const int64_t n = int64_t(P.n1) * P.n2;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t c = base + lane;
    bool keep = false;
    int i = 0, j = 0;
    if (c < n) {
      i = int(c / P.n2);
      j = int(c % P.n2);
      const int t2 = P.t2_begin + j;
      float lo[3], hi[3];
      for (int k = 0; k < 3; ++k) {
        const double a = P.mesh.tri[int64_t(k) * P.mesh.n_tris + t2], b = P.mesh.tri[int64_t(3 + k) * P.mesh.n_tris + t2],
                     d = P.mesh.tri[int64_t(6 + k) * P.mesh.n_tris + t2];
        lo[k] = __double2float_rd(fmin(a, fmin(b, d)));
        hi[k] = __double2float_ru(fmax(a, fmax(b, d)));
      }
      keep = box_overlaps(P.fwd + int64_t(i) * 12, lo[0], hi[0], lo[1], hi[1], lo[2], hi[2]);
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) continue;
    unsigned long long b0 = 0;
    if (lane == 0) b0 = atomicAdd(P.pair_count, (unsigned long long)__popc(m));
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (keep) {
      const unsigned long long idx = b0 + __popc(m & ((1u << lane) - 1u));
      if (idx < (unsigned long long)P.pair_cap) {
        P.pairs[2 * idx] = i;
        P.pairs[2 * idx + 1] = j;
      }
    }
  }
}

// Per (query, pair): the backward box of T2 from x3 (iii); survivors are the
// chains.  One FP64 interval evaluation per (query, T2) is recomputed per
// pair; pairs of one T2 are rare enough that this is not the bottleneck.
__global__ void tt_cone_chains_kernel(TTConeParams P, int64_t n_pairs) {
  const int64_t n = P.qv.n * n_pairs;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t c = base + lane;
    bool keep = false;
    int64_t q = 0;
    int i = 0, j = 0;
    if (c < n) {
      q = c / n_pairs;
      const int64_t f = c % n_pairs;
      i = P.pairs[2 * f];
      j = P.pairs[2 * f + 1];
      const int t2 = P.t2_begin + j;
      const d3 x3 = mk(P.qv.x_last[3 * q], P.qv.x_last[3 * q + 1], P.qv.x_last[3 * q + 2]);
      Iv3 o, bb;
      bool empty = false;
      const bool ok =
          out_box(P.mesh, t2, x3, P.qv.types[2 * q + 1], P.qv.eta[3 * q + 2], P.qv.eta[3 * q + 1], o, bb, empty);
      if (empty) {
        keep = false;
      } else if (!ok) {
        keep = true;
      } else {
        float B[12];
        const Iv comps[3] = {o.x, o.y, o.z};
        const Iv bcomp[3] = {bb.x, bb.y, bb.z};
        for (int k = 0; k < 3; ++k) {
          const Iv w = widen(comps[k], P.margin);
          B[k] = __double2float_rd(w.lo);
          B[3 + k] = __double2float_ru(w.hi);
          B[6 + k] = __double2float_rd(bcomp[k].lo);
          B[9 + k] = __double2float_ru(bcomp[k].hi);
        }
        const float* F = P.fwd + int64_t(i) * 12;
        // backward directions (from T2 toward T1) against T1's bounding box
        keep = box_overlaps(B, F[6], F[9], F[7], F[10], F[8], F[11]);
        // negated backward box against the forward box
        for (int k = 0; k < 3 && keep; ++k) keep = (-B[3 + k] <= F[3 + k]) && (F[k] <= -B[k]);
      }
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) continue;
    unsigned long long b0 = 0;
    if (lane == 0) b0 = atomicAdd(P.count, (unsigned long long)__popc(m));
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (keep) {
      const unsigned long long idx = b0 + __popc(m & ((1u << lane) - 1u));
      if (idx < (unsigned long long)P.cap) {
        P.out[3 * idx] = int32_t(q);
        P.out[3 * idx + 1] = P.t1_begin + i;
        P.out[3 * idx + 2] = P.t2_begin + j;
      }
    }
  }
}

// Queries must share x0, the IORs and the types, T T or R R (all k = 2).
__global__ void tt_shared_kernel(QueryView Q, int32_t* flag) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < Q.n; q += stride) {
    bool same = true;
    for (int c = 0; c < 3; ++c) same &= Q.x_first[3 * q + c] == Q.x_first[c] && Q.eta[3 * q + c] == Q.eta[c];
    same &= Q.types[2 * q] == Q.types[0] && Q.types[2 * q + 1] == Q.types[0] && Q.k[q] == 2;
    same &= Q.types[0] == SPOLY_T || Q.types[0] == SPOLY_R;
    if (!same) atomicExch(flag, 0);
  }
}

}  // namespace

// ------------------------------------- explicit lists, culled per chain
// The per-chain boxes use FP32 interval arithmetic with directed rounding
// (every lower end rounded down, every upper end up), so each box encloses
// the exact one like the FP64 boxes of the range-based culls, at FP32 rates.
struct IvF {
  float lo, hi;
};
SPOLY_D IvF ivf_pt(double a) { return {__double2float_rd(a), __double2float_ru(a)}; }
SPOLY_D IvF operator+(IvF a, IvF b) { return {__fadd_rd(a.lo, b.lo), __fadd_ru(a.hi, b.hi)}; }
SPOLY_D IvF operator-(IvF a, IvF b) { return {__fsub_rd(a.lo, b.hi), __fsub_ru(a.hi, b.lo)}; }
SPOLY_D IvF operator-(IvF a) { return {-a.hi, -a.lo}; }
SPOLY_D IvF operator*(IvF a, IvF b) {
  const float l = fminf(fminf(__fmul_rd(a.lo, b.lo), __fmul_rd(a.lo, b.hi)),
                        fminf(__fmul_rd(a.hi, b.lo), __fmul_rd(a.hi, b.hi)));
  const float h = fmaxf(fmaxf(__fmul_ru(a.lo, b.lo), __fmul_ru(a.lo, b.hi)),
                        fmaxf(__fmul_ru(a.hi, b.lo), __fmul_ru(a.hi, b.hi)));
  return {l, h};
}
SPOLY_D IvF sqrf(IvF a) {
  if (a.lo >= 0.f) return {__fmul_rd(a.lo, a.lo), __fmul_ru(a.hi, a.hi)};
  if (a.hi <= 0.f) return {__fmul_rd(a.hi, a.hi), __fmul_ru(a.lo, a.lo)};
  return {0.f, fmaxf(__fmul_ru(a.lo, a.lo), __fmul_ru(a.hi, a.hi))};
}
// a / L with L = [llo, lhi], llo > 0.
SPOLY_D IvF divposf(IvF a, float llo, float lhi) {
  if (a.lo >= 0.f) return {__fdiv_rd(a.lo, lhi), __fdiv_ru(a.hi, llo)};
  if (a.hi <= 0.f) return {__fdiv_rd(a.lo, llo), __fdiv_ru(a.hi, lhi)};
  return {__fdiv_rd(a.lo, llo), __fdiv_ru(a.hi, llo)};
}
struct Iv3F {
  IvF x, y, z;
};
SPOLY_D bool normalisef(const Iv3F& v, Iv3F& out) {
  const IvF l2 = sqrf(v.x) + sqrf(v.y) + sqrf(v.z);
  if (!(l2.lo > 0.f)) return false;
  const float llo = __fsqrt_rd(l2.lo), lhi = __fsqrt_ru(l2.hi);
  out = {divposf(v.x, llo, lhi), divposf(v.y, llo, lhi), divposf(v.z, llo, lhi)};
  return true;
}

// out_box in FP32 with directed rounding (the same steps).
SPOLY_D bool out_box_f(const MeshView& M, int t, d3 x0, int type, double eta0, double eta1, Iv3F& o, Iv3F& bb,
                       bool& empty) {
  empty = false;
  auto g = [&](int row) { return M.tri[int64_t(row) * M.n_tris + t]; };
  IvF P[3], N[3];
  for (int c = 0; c < 3; ++c) {
    const double p0 = g(c), p1 = g(3 + c), p2 = g(6 + c);
    const double n0 = g(9 + c), n1 = g(12 + c), n2 = g(15 + c);
    P[c] = {__double2float_rd(fmin(p0, fmin(p1, p2))), __double2float_ru(fmax(p0, fmax(p1, p2)))};
    N[c] = {__double2float_rd(fmin(n0, fmin(n1, n2))), __double2float_ru(fmax(n0, fmax(n1, n2)))};
  }
  bb = {P[0], P[1], P[2]};
  const Iv3F d = {P[0] - ivf_pt(x0.x), P[1] - ivf_pt(x0.y), P[2] - ivf_pt(x0.z)};
  Iv3F dh, nh;
  if (!normalisef(d, dh)) return false;
  if (!normalisef({N[0], N[1], N[2]}, nh)) return false;
  IvF c = -(dh.x * nh.x + dh.y * nh.y + dh.z * nh.z);  // c = -d^ . n^
  if (c.hi < 0.f) {  // normal points away from x0: flip it
    nh = {-nh.x, -nh.y, -nh.z};
    c = -c;
  } else if (!(c.lo > 0.f)) {
    return false;  // grazing somewhere on the triangle
  }
  c.hi = fminf(c.hi, 1.f);
  if (type == SPOLY_R) {
    const IvF c2 = c + c;
    o = {dh.x + c2 * nh.x, dh.y + c2 * nh.y, dh.z + c2 * nh.z};
  } else {
    const IvF eta = {__double2float_rd(__ddiv_rd(eta0, eta1)), __double2float_ru(__ddiv_ru(eta0, eta1))};
    const IvF one = {1.f, 1.f};
    const IvF k = one - sqrf(eta) * (one - sqrf(c));
    if (k.hi < 0.f) {
      empty = true;
      return true;
    }
    const IvF sk = {__fsqrt_rd(fmaxf(k.lo, 0.f)), __fsqrt_ru(k.hi)};
    const IvF f = eta * c - sk;
    o = {eta * dh.x + f * nh.x, eta * dh.y + f * nh.y, eta * dh.z + f * nh.z};
  }
  return true;
}

// Box of one triangle lit from x: [12] floats (outgoing lo/hi xyz, widened
// by the margin; bounding box lo/hi xyz).  A triangle with no bound gets
// the full box, one with no transmitted direction an empty one.
SPOLY_D void chain_box(const MeshView& M, int t, d3 x, int type, double eta_in, double eta_out, double margin,
                       float (&B)[12]) {
  Iv3F o, bb;
  bool empty = false;
  const bool ok = out_box_f(M, t, x, type, eta_in, eta_out, o, bb, empty);
  const IvF comps[3] = {o.x, o.y, o.z};
  const IvF bcomp[3] = {bb.x, bb.y, bb.z};
  const float m = __double2float_ru(margin);
  for (int k = 0; k < 3; ++k) {
    B[k] = empty ? 2.f : (ok ? fmaxf(-1.f, __fsub_rd(comps[k].lo, m)) : -1.f);
    B[3 + k] = empty ? -2.f : (ok ? fminf(1.f, __fadd_ru(comps[k].hi, m)) : 1.f);
    B[6 + k] = bcomp[k].lo;
    B[9 + k] = bcomp[k].hi;
  }
}

// The CONE test of one chain: 1 bounce as cone_pairs_general_kernel; 2
// bounces of two refractions or two reflections as tt_pairs_kernel (i, ii)
// and tt_cone_chains_kernel (iii) (for reflection the segment x1 -> x2 is
// the ray reflected from x0 and, reversed, the one reflected from x3).
// Mixed 2-bounce types are kept.
SPOLY_D bool chain_cone_keep(const MeshView& M, const QueryView& Q, int64_t q, int t0, int t1, double margin) {
  const d3 x0 = mk(Q.x_first[3 * q], Q.x_first[3 * q + 1], Q.x_first[3 * q + 2]);
  const d3 xl = mk(Q.x_last[3 * q], Q.x_last[3 * q + 1], Q.x_last[3 * q + 2]);
  const int k = Q.k[q];
  if (k == 1 || t1 < 0) {
    float B[12];
    chain_box(M, t0, x0, Q.types[2 * q], Q.eta[3 * q], Q.eta[3 * q + 1], margin, B);
    return to_box_overlaps(B, float(xl.x), float(xl.y), float(xl.z));
  }
  const int ty = Q.types[2 * q];
  if ((ty != SPOLY_T && ty != SPOLY_R) || Q.types[2 * q + 1] != ty) return true;
  float F[12], B[12];
  chain_box(M, t0, x0, ty, Q.eta[3 * q], Q.eta[3 * q + 1], margin, F);
  chain_box(M, t1, xl, ty, Q.eta[3 * q + 2], Q.eta[3 * q + 1], margin, B);
  if (!box_overlaps(F, B[6], B[9], B[7], B[10], B[8], B[11])) return false;  // (i), (ii)
  if (!box_overlaps(B, F[6], F[9], F[7], F[10], F[8], F[11])) return false;  // (iii) toward T1
  for (int c = 0; c < 3; ++c)
    if (!((-B[3 + c] <= F[3 + c]) && (F[c] <= -B[c]))) return false;  // negated backward box vs forward
  return true;
}

__global__ void explicit_cone_kernel(ChainParams P, const int32_t* src, int64_t n, unsigned long long* k2) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int lane = threadIdx.x & 31;
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t c = base + lane;
    bool keep = false;
    int32_t q = 0, t0 = 0, t1 = -1;
    if (c < n) {
      q = src[3 * c];
      t0 = src[3 * c + 1];
      t1 = src[3 * c + 2];
      keep = chain_cone_keep(P.mesh, P.qv, q, t0, t1, P.margin);
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (!m) continue;
    const unsigned m2 = __ballot_sync(0xffffffffu, keep && t1 >= 0);
    unsigned long long b0 = 0;
    if (lane == 0) {
      b0 = atomicAdd(P.count, (unsigned long long)__popc(m));
      if (m2) atomicAdd(k2, (unsigned long long)__popc(m2));
    }
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (keep) {
      const unsigned long long idx = b0 + __popc(m & ((1u << lane) - 1u));
      if (idx < (unsigned long long)P.cap) {
        P.out[3 * idx] = q;
        P.out[3 * idx + 1] = t0;
        P.out[3 * idx + 2] = t1;
      }
    }
  }
}

cudaError_t launch_tt_cone_shared(const TTConeParams& P, int32_t* flag, int num_sms, cudaStream_t st, int32_t* host) {
  set_flag_kernel<<<1, 1, 0, st>>>(flag, 1);
  tt_shared_kernel<<<num_sms * 4, 256, 0, st>>>(P.qv, flag);
  cudaError_t e = cudaMemcpyAsync(host, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t launch_tt_cone_pairs(const TTConeParams& P, int num_sms, cudaStream_t st) {
  tt_fwd_boxes_kernel<<<(P.n1 + 127) / 128, 128, 0, st>>>(P);
  tt_pairs_kernel<<<num_sms * 8, 256, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_tt_cone_chains(const TTConeParams& P, int64_t n_pairs, int num_sms, cudaStream_t st) {
  if (n_pairs <= 0) return cudaSuccess;
  tt_cone_chains_kernel<<<num_sms * 16, 256, 0, st>>>(P, n_pairs);
  return cudaGetLastError();
}


cudaError_t launch_chains_explicit_cone(const ChainParams& P, const int32_t* src, int64_t n, unsigned long long* k2,
                                        int num_sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  explicit_cone_kernel<<<num_sms * 8, 256, 0, st>>>(P, src, n, k2);
  return cudaGetLastError();
}

}  // namespace spoly
