// Pixel-footprint candidate builder (glints): a uniform grid over the mesh
// and, per pixel of a pinhole camera, the triangles whose bounding box meets
// the pixel's footprint on the mesh.
//
// The footprint of pixel (ix, iy) is the xy bounding box of its four corner
// rays between the planes z = zmin and z = zmax of the mesh's bounding box,
// so every surface point a pixel can see lies inside it.  A triangle is
// emitted once per pixel, from the first grid cell its bounding box shares
// with the footprint.  Emission is two-pass (count, exclusive scan, fill), so
// the chain list is ordered by pixel without global atomics; the count pass
// keeps each pixel's first candidates, so the fill copies them instead of
// traversing the grid again (pixels with more candidates traverse it again).
#include <algorithm>
#include <climits>
#include <cstring>

#include "k1.cuh"
#include "scan.cuh"

namespace spoly {

namespace {

using scan::kScanBlock;

// Ordered-int encoding of floats for atomicMin / atomicMax.
SPOLY_D int f2o(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
SPOLY_D float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }
float o2f_host(int i) {
  const int b = i >= 0 ? i : i ^ 0x7fffffff;
  float f;
  std::memcpy(&f, &b, 4);
  return f;
}

// Mesh bounds ([0..2] min xyz, [3..5] max xyz as ordered ints; slack added
// by the caller) and every triangle's FP32 xy box (xl, xh, yl, yh), which the
// grid and footprint passes read instead of the six FP64 coordinates.
// Ordered-int64 keys of doubles: integer min / max on them order the values,
// so the FP64 comparisons of the box run on the integer pipe (the FP64 pipe
// takes about 64 cycles per warp instruction on this part).
SPOLY_D long long d2o(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : b ^ 0x7fffffffffffffffll;
}
SPOLY_D double o2d(long long o) { return __longlong_as_double(o >= 0 ? o : o ^ 0x7fffffffffffffffll); }

// FP64 -> FP32, round to nearest even, with integer instructions where the
// result is a normal float or zero (the conversion instruction runs on the
// narrow FP64 pipe of this part); other cases take the instruction.  The
// 29 dropped mantissa bits decide the rounding; a carry out of the mantissa
// steps the exponent (up to infinity, as the rounding rule says).
SPOLY_D float f32_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = unsigned(b >> 32), lo = unsigned(b);
  const int e = int((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (e >= 1 && e <= 254) {
    unsigned f = (hi & 0x80000000u) | (unsigned(e) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned drop = lo & 0x1fffffffu;
    f += (drop > 0x10000000u || (drop == 0x10000000u && (f & 1u))) ? 1u : 0u;
    return __uint_as_float(f);
  }
  if ((b << 1) == 0ull) return __uint_as_float(hi & 0x80000000u);
  return float(x);
}

__global__ void mesh_bounds_kernel(MeshView M, int* bounds, float4* boxes) {
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  long long zlo = LLONG_MAX, zhi = LLONG_MIN;  // z range, as keys (converted once per thread)
  float wx = 0.0f, wy = 0.0f;                  // largest box width and height
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < M.n_tris; t += stride) {
    long long k[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) k[i] = d2o(__ldg(M.tri + int64_t(i) * M.n_tris + t));
    // float(min) = min(float): rounding to nearest is monotone
    const float xl = f32_rn(o2d(min(k[0], min(k[3], k[6])))), xh = f32_rn(o2d(max(k[0], max(k[3], k[6]))));
    const float yl = f32_rn(o2d(min(k[1], min(k[4], k[7])))), yh = f32_rn(o2d(max(k[1], max(k[4], k[7]))));
    zlo = min(zlo, min(k[2], min(k[5], k[8])));
    zhi = max(zhi, max(k[2], max(k[5], k[8])));
    boxes[t] = make_float4(xl, xh, yl, yh);
    lo[0] = fminf(lo[0], xl);
    hi[0] = fmaxf(hi[0], xh);
    lo[1] = fminf(lo[1], yl);
    hi[1] = fmaxf(hi[1], yh);
    wx = fmaxf(wx, xh - xl);
    wy = fmaxf(wy, yh - yl);
  }
  if (zlo <= zhi) {
    lo[2] = f32_rn(o2d(zlo));
    hi[2] = f32_rn(o2d(zhi));
  }
  for (int o = 16; o > 0; o >>= 1) {
    wx = fmaxf(wx, __shfl_xor_sync(0xffffffffu, wx, o));
    wy = fmaxf(wy, __shfl_xor_sync(0xffffffffu, wy, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(bounds + 6, f2o(wx));
    atomicMax(bounds + 7, f2o(wy));
  }
  for (int c = 0; c < 3; ++c) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
      hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(bounds + c, f2o(lo[c]));
      atomicMax(bounds + 3 + c, f2o(hi[c]));
    }
  }
}

// One wave of a grid-stride kernel of `Block` threads per block: every
// resident block on every SM, so no block starts late and leaves a tail.  The
// count is taken once per kernel.
template <auto Kernel, int Block>
int resident_grid(int num_sms) {
  static int per_sm = 0;
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, Kernel, Block, 0) != cudaSuccess || b < 1) {
      (void)cudaGetLastError();
      b = 4;
    }
    per_sm = b;
  }
  return num_sms * per_sm;
}

__global__ void init_bounds_kernel(int* bounds) {
  if (threadIdx.x < 3) bounds[threadIdx.x] = f2o(3e38f);
  else if (threadIdx.x < 6) bounds[threadIdx.x] = f2o(-3e38f);
  else if (threadIdx.x < 8) bounds[threadIdx.x] = f2o(0.0f);
}

struct GridGeom {
  float x0, y0, inv;  // origin and 1 / cell size
  int gx, gy;
};

SPOLY_D void cell_range(const GridGeom& G, float xl, float xh, float yl, float yh, int& cx0, int& cx1, int& cy0,
                        int& cy1) {
  cx0 = max(0, min(G.gx - 1, int(floorf((xl - G.x0) * G.inv))));
  cx1 = max(0, min(G.gx - 1, int(floorf((xh - G.x0) * G.inv))));
  cy0 = max(0, min(G.gy - 1, int(floorf((yl - G.y0) * G.inv))));
  cy1 = max(0, min(G.gy - 1, int(floorf((yh - G.y0) * G.inv))));
}

SPOLY_D void tri_bbox(const float4* __restrict__ boxes, int64_t t, float& xl, float& xh, float& yl, float& yh) {
  const float4 b = __ldg(boxes + t);
  xl = b.x;
  xh = b.y;
  yl = b.z;
  yh = b.w;
}

// pass 0: count entries per cell; pass 1: fill (cursor = count copy)
__global__ void grid_insert_kernel(MeshView M, const float4* boxes, GridGeom G, int* cell_count,
                                   const int64_t* cell_off, int32_t* entries, int pass) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < M.n_tris; t += stride) {
    float xl, xh, yl, yh;
    tri_bbox(boxes, t, xl, xh, yl, yh);
    int cx0, cx1, cy0, cy1;
    cell_range(G, xl, xh, yl, yh, cx0, cx1, cy0, cy1);
    for (int cy = cy0; cy <= cy1; ++cy)
      for (int cx = cx0; cx <= cx1; ++cx) {
        const int64_t cell = int64_t(cy) * G.gx + cx;
        const int slot = atomicAdd(cell_count + cell, 1);
        if (pass == 1) entries[cell_off[cell] + slot] = int32_t(t);
      }
  }
}

struct CamF {
  float ox, oy, oz, fx, fy, fz, rx, ry, rz, ux, uy, uz;
  float sx_scale, sy_scale;  // 2 tan aspect / w, 2 tan / h
  float tha, th;             // tan aspect, tan
  int w, h;
};

CamF make_cam(const double* c) {  // host: c is the caller's 16-double camera
  CamF k;
  k.ox = float(c[0]);
  k.oy = float(c[1]);
  k.oz = float(c[2]);
  k.fx = float(c[3]);
  k.fy = float(c[4]);
  k.fz = float(c[5]);
  k.rx = float(c[6]);
  k.ry = float(c[7]);
  k.rz = float(c[8]);
  k.ux = float(c[9]);
  k.uy = float(c[10]);
  k.uz = float(c[11]);
  k.w = int(c[14]);
  k.h = int(c[15]);
  k.tha = float(c[12] * c[13]);
  k.th = float(c[12]);
  k.sx_scale = float(2.0 * c[12] * c[13] / c[14]);
  k.sy_scale = float(2.0 * c[12] / c[15]);
  return k;
}

// Footprint of a pixel: xy box of its corner rays between z = zlo and z = zhi,
// in FP32 (coordinates are O(1); the 1e-5 relative margin covers rounding).
SPOLY_D bool pixel_footprint(const CamF& C, int64_t q, float zlo, float zhi, float& xl, float& xh, float& yl,
                             float& yh) {
  const int qi = int(q);  // n_pixels < 2^31
  const int iy = qi / C.w, ix = qi - iy * C.w;
  xl = yl = 3e38f;
  xh = yh = -3e38f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float a = float(ix + (k & 1)) * C.sx_scale - C.tha;  // sx tan aspect
    const float b = C.th - float(iy + (k >> 1)) * C.sy_scale;  // sy tan
    const float dx = C.fx + a * C.rx + b * C.ux, dy = C.fy + a * C.ry + b * C.uy, dz = C.fz + a * C.rz + b * C.uz;
    if (!(dz < 0.0f)) return false;  // a corner ray never reaches the surface slab
    const float rdz = 1.0f / dz;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const float tt = ((p ? zhi : zlo) - C.oz) * rdz;
      const float x = C.ox + tt * dx, y = C.oy + tt * dy;
      xl = fminf(xl, x);
      xh = fmaxf(xh, x);
      yl = fminf(yl, y);
      yh = fmaxf(yh, y);
    }
  }
  const float m = 1e-5f * (1.f + fmaxf(fmaxf(fabsf(xl), fabsf(xh)), fmaxf(fabsf(yl), fabsf(yh))));
  xl -= m;
  yl -= m;
  xh += m;
  yh += m;
  return true;
}

constexpr int kPixCand = 128;  // candidates per pixel kept by the count pass for the fill

// Candidates of pixel q in emission order: each one goes to emit(t); returns
// their number.
// ext < 0: every triangle sits in every cell its box meets, and a triangle
// is emitted from the first cell it shares with the footprint.  ext >= 0
// (single-cell grid): every triangle sits in its box's lower-corner cell
// only, and the traversal starts ext cells lower in x and y.
template <typename Emit>
SPOLY_D int64_t pixel_candidates(const float4* boxes, const GridGeom& G, const CamF& C, float zlo, float zhi,
                                 int64_t q, const int* cell_count, const int64_t* cell_off, const int32_t* entries,
                                 Emit emit, int64_t cap = INT64_MAX, int ext = -1) {
  float xl, xh, yl, yh;
  int64_t n = 0;
  if (!pixel_footprint(C, q, zlo, zhi, xl, xh, yl, yh)) return 0;
  int fx0, fx1, fy0, fy1;
  cell_range(G, xl, xh, yl, yh, fx0, fx1, fy0, fy1);
  const bool single = ext >= 0;
  const int sx0 = single ? max(0, fx0 - ext) : fx0, sy0 = single ? max(0, fy0 - ext) : fy0;
  for (int cy = sy0; cy <= fy1; ++cy)
    for (int cx = sx0; cx <= fx1; ++cx) {
      const int64_t cell = int64_t(cy) * G.gx + cx;
      const int64_t b = cell_off[cell], e = min(b + cell_count[cell], cap);
      // four entries at a time: their index loads, then their box gathers,
      // are independent, so each group waits for two memory round trips
      for (int64_t k0 = b; k0 < e; k0 += 4) {
        int32_t t[4];
        float4 bx[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) t[u] = (k0 + u < e) ? __ldg(entries + k0 + u) : -1;
#pragma unroll
        for (int u = 0; u < 4; ++u) bx[u] = (t[u] >= 0) ? __ldg(boxes + t[u]) : make_float4(1.f, -1.f, 1.f, -1.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float txl = bx[u].x, txh = bx[u].y, tyl = bx[u].z, tyh = bx[u].w;
          if (t[u] < 0 || txh < xl || txl > xh || tyh < yl || tyl > yh) continue;
          if (!single) {
            int tx0, tx1, ty0, ty1;
            cell_range(G, txl, txh, tyl, tyh, tx0, tx1, ty0, ty1);
            if (cx != max(tx0, fx0) || cy != max(ty0, fy0)) continue;  // emitted from its first shared cell
          }
          emit(n, t[u]);
          ++n;
        }
      }
    }
  return n;
}

// Count pass: candidates per pixel, the first kPixCand of them kept in
// `cand` ([n_pixels][kPixCand]) so that the fill needs no second traversal.
__global__ void footprint_count_kernel(const float4* boxes, GridGeom G, const int* bounds, CamF C, int64_t n_pixels,
                                       const int* cell_count, const int64_t* cell_off, const int32_t* entries,
                                       int64_t* pix_count, int32_t* cand) {
  const float zlo = o2f(bounds[2]), zhi = o2f(bounds[5]);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < n_pixels; q += stride) {
    int32_t* mine = cand + q * kPixCand;
    pix_count[q] = pixel_candidates(boxes, G, C, zlo, zhi, q, cell_count, cell_off, entries,
                                    [&](int64_t k, int32_t t) {
                                      if (k < kPixCand) mine[k] = t;
                                    });
  }
}

// ---- distinct-triangle mode without host round trips: the grid geometry
// is derived on the device from the mesh bounds, the grid fill checks its
// capacity, and the counts the host needs land in one record read once.
struct FpUniqueDev {
  GridGeom G;
  unsigned long long n_entries, pairs, n_unique;
  int32_t differ;  // some query differs from query 0
  int32_t single;  // 1: each triangle sits in the cell of its box's lower corner only
  int32_t ext;     // single: the most cells a box spans beyond its lower corner's (set by pass 0)
  int32_t pad;
};

// Single-cell insertion is used while the widest triangle box is narrower
// than kSingleCellSpan cells: a pixel's traversal then reaches `ext` cells
// further down in x and y (ext = the largest span of a box beyond its lower
// corner's cell), and no triangle is met twice.
constexpr float kSingleCellSpan = 2.0f;

// Square cells over the bounds' larger extent, g x g of them.
__global__ void grid_setup_kernel(const int* bounds, int g, FpUniqueDev* info) {
  const float xl = o2f(bounds[0]), yl = o2f(bounds[1]), xh = o2f(bounds[3]), yh = o2f(bounds[4]);
  const float w = fmaxf(fmaxf(xh - xl, yh - yl), 1e-20f) * (1.0f + 1e-5f);
  info->G.x0 = xl;
  info->G.y0 = yl;
  info->G.inv = float(g) / w;
  info->G.gx = g;
  info->G.gy = g;
  const float span = fmaxf(o2f(bounds[6]), o2f(bounds[7])) * info->G.inv;
  info->single = (span < kSingleCellSpan) ? 1 : 0;
  info->ext = 0;
}

// pass 0: count entries per cell (single-cell mode: also the largest span
// beyond the lower corner's cell); pass 1: fill, writing only below cap.
__global__ void grid_insert_dev_kernel(MeshView M, const float4* boxes, FpUniqueDev* info, int* cell_count,
                                       const int64_t* cell_off, int32_t* entries, int64_t cap, int pass) {
  const GridGeom G = info->G;
  const bool single = info->single != 0;
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  int span = 0;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < M.n_tris; t += stride) {
    float xl, xh, yl, yh;
    tri_bbox(boxes, t, xl, xh, yl, yh);
    int cx0, cx1, cy0, cy1;
    cell_range(G, xl, xh, yl, yh, cx0, cx1, cy0, cy1);
    if (single) {
      span = max(span, max(cx1 - cx0, cy1 - cy0));
      cx1 = cx0;
      cy1 = cy0;
    }
    for (int cy = cy0; cy <= cy1; ++cy)
      for (int cx = cx0; cx <= cx1; ++cx) {
        const int64_t cell = int64_t(cy) * G.gx + cx;
        const int slot = atomicAdd(cell_count + cell, 1);
        if (pass == 1 && cell_off[cell] + slot < cap) entries[cell_off[cell] + slot] = int32_t(t);
      }
  }
  if (single && pass == 0) {
    span = __reduce_max_sync(0xffffffffu, span);
    if ((threadIdx.x & 31) == 0 && span > 0) atomicMax(&info->ext, span);
  }
}

__global__ void grid_total_kernel(const int* cell_count, const int64_t* cell_off, int64_t n_cells, FpUniqueDev* info) {
  info->n_entries = (unsigned long long)(cell_off[n_cells - 1] + cell_count[n_cells - 1]);
}

// Marks the candidate triangles of every pixel and sums the (pixel,
// triangle) pairs (one atomic per warp).
__global__ void footprint_mark_kernel(const float4* boxes, FpUniqueDev* info, const int* bounds, CamF C,
                                      int64_t n_pixels, const int* cell_count, const int64_t* cell_off,
                                      const int32_t* entries, int64_t cap, uint8_t* mark) {
  const GridGeom G = info->G;
  const int ext = info->single ? info->ext : -1;
  const float zlo = o2f(bounds[2]), zhi = o2f(bounds[5]);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q0 = int64_t(blockIdx.x) * blockDim.x; q0 < n_pixels; q0 += stride) {
    const int64_t q = q0 + threadIdx.x;
    unsigned n = 0;
    if (q < n_pixels)
      n = unsigned(pixel_candidates(boxes, G, C, zlo, zhi, q, cell_count, cell_off, entries,
                                    [&](int64_t, int32_t t) { mark[t] = 1; }, cap, ext));
    warp_count(&info->pairs, n);
  }
}

// Distinct-triangle list: the marked triangles as chains (query, t, -1).
// Each block compacts a chunk of 256 consecutive triangles in order and
// takes its output range with one atomic, so the list is ordered by
// triangle within chunks (chunks land in completion order).
__global__ void __launch_bounds__(256) unique_fill_kernel(const uint8_t* __restrict__ mark, int64_t n_tris,
                                                          int32_t query, unsigned long long* count, int32_t* out) {
  __shared__ unsigned warp_n[8];
  __shared__ unsigned long long base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t c0 = int64_t(blockIdx.x) * 256; c0 < n_tris; c0 += int64_t(gridDim.x) * 256) {
    const int64_t t = c0 + threadIdx.x;
    const bool on = t < n_tris && mark[t] != 0;
    const unsigned b = __ballot_sync(0xffffffffu, on);
    if (lane == 0) warp_n[warp] = __popc(b);
    __syncthreads();
    unsigned before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      before += (w < warp) ? warp_n[w] : 0u;
      total += warp_n[w];
    }
    if (threadIdx.x == 0) base = total ? atomicAdd(count, (unsigned long long)total) : 0ull;
    __syncthreads();
    if (on) {
      const unsigned long long slot = base + before + __popc(b & ((1u << lane) - 1u));
      out[3 * slot] = query;
      out[3 * slot + 1] = int32_t(t);
      out[3 * slot + 2] = -1;
    }
    __syncthreads();
  }
}

// flag[0] = 1 when some query differs from query 0 in x_first, x_last, eta,
// types or k (bitwise).
__global__ void queries_shared_kernel(QueryView qv, int32_t* flag) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < qv.n; q += stride) {
    // every field compared without short-circuit, so all loads issue at once
    bool same = (qv.k[q] == qv.k[0]) & (qv.types[2 * q] == qv.types[0]) & (qv.types[2 * q + 1] == qv.types[1]);
#pragma unroll
    for (int c = 0; c < 3; ++c)
      same &= (__double_as_longlong(qv.x_first[3 * q + c]) == __double_as_longlong(qv.x_first[c])) &
              (__double_as_longlong(qv.x_last[3 * q + c]) == __double_as_longlong(qv.x_last[c])) &
              (__double_as_longlong(qv.eta[3 * q + c]) == __double_as_longlong(qv.eta[c]));
    if (!same) flag[0] = 1;
  }
}

// Fill: one warp per pixel copies its kept candidates to out[pix_off[q]..]
// (coalesced); pixels with more than kPixCand are left to the overflow pass.
__global__ void footprint_fill_kernel(int64_t n_pixels, const int64_t* pix_count, const int64_t* pix_off,
                                      const int32_t* cand, int32_t* out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t q = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; q < n_pixels; q += nw) {
    const int64_t n = pix_count[q], o = pix_off[q];
    if (n > kPixCand) continue;
    for (int64_t k = lane; k < n; k += 32) {
      out[3 * (o + k)] = int32_t(q);
      out[3 * (o + k) + 1] = cand[q * kPixCand + k];
      out[3 * (o + k) + 2] = -1;
    }
  }
}

// Overflow pass: a pixel with more than kPixCand candidates traverses the
// grid again (one pixel per thread) and writes all of them.
__global__ void footprint_overflow_kernel(const float4* boxes, GridGeom G, const int* bounds, CamF C,
                                          int64_t n_pixels, const int* cell_count, const int64_t* cell_off,
                                          const int32_t* entries, const int64_t* pix_count, const int64_t* pix_off,
                                          int32_t* out) {
  const float zlo = o2f(bounds[2]), zhi = o2f(bounds[5]);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < n_pixels; q += stride) {
    const int64_t n = pix_count[q], o = pix_off[q];
    if (n <= kPixCand) continue;
    pixel_candidates(boxes, G, C, zlo, zhi, q, cell_count, cell_off, entries, [&](int64_t k, int32_t t) {
      if (k < n) {
        out[3 * (o + k)] = int32_t(q);
        out[3 * (o + k) + 1] = t;
        out[3 * (o + k) + 2] = -1;
      }
    });
  }
}

}  // namespace

// Scratch layout of the footprint builder (bytes, library-owned).
struct FpLayout {
  int* cell_count;
  int64_t* cell_off;
  int64_t* pix_count;
  int64_t* pix_off;
  int64_t *sums1, *sums1_off, *sums2;
  int32_t* pix_cand;  // [n_pixels][kPixCand]
};

static size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

size_t footprint_scratch_bytes(int64_t n_cells, int64_t n_pixels) {
  const int64_t nb = (std::max(n_cells, n_pixels) + kScanBlock - 1) / kScanBlock;
  return up256(n_cells * 4) + up256(n_cells * 8) + 2 * up256(n_pixels * 8) + 2 * up256(nb * 8 + 64) +
         up256(3 * kScanBlock * 8) + up256(size_t(n_pixels) * kPixCand * 4);
}

static FpLayout fp_layout(void* scratch, int64_t n_cells, int64_t n_pixels) {
  const int64_t nb = (std::max(n_cells, n_pixels) + kScanBlock - 1) / kScanBlock;
  char* p = static_cast<char*>(scratch);
  FpLayout L;
  L.cell_count = reinterpret_cast<int*>(p);
  p += up256(n_cells * 4);
  L.cell_off = reinterpret_cast<int64_t*>(p);
  p += up256(n_cells * 8);
  L.pix_count = reinterpret_cast<int64_t*>(p);
  p += up256(n_pixels * 8);
  L.pix_off = reinterpret_cast<int64_t*>(p);
  p += up256(n_pixels * 8);
  L.sums1 = reinterpret_cast<int64_t*>(p);
  p += up256(nb * 8 + 64);
  L.sums1_off = reinterpret_cast<int64_t*>(p);
  p += up256(nb * 8 + 64);
  L.sums2 = reinterpret_cast<int64_t*>(p);
  p += up256(3 * kScanBlock * 8);
  L.pix_cand = reinterpret_cast<int32_t*>(p);
  return L;
}

template <typename In>
static cudaError_t exclusive_scan(const In* in, int64_t* out, int64_t n, const FpLayout& L, cudaStream_t st) {
  return scan::exclusive_scan<In>(in, out, n, L.sums1, L.sums1_off, L.sums2, st);
}

static cudaError_t read_total(const int64_t* off, const void* count, bool count64, int64_t n, int64_t* total,
                              cudaStream_t st) {
  int64_t a = 0, b64 = 0;
  int b32 = 0;
  cudaError_t e = cudaMemcpyAsync(&a, off + n - 1, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = count64 ? cudaMemcpyAsync(&b64, static_cast<const int64_t*>(count) + n - 1, 8, cudaMemcpyDeviceToHost, st)
                : cudaMemcpyAsync(&b32, static_cast<const int*>(count) + n - 1, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *total = a + (count64 ? b64 : b32);
  return e;
}

// Stage 1: grid cell counts and offsets; returns the number of cell entries.
cudaError_t fp_grid_count(const MeshView& M, const float4* boxes, const FpGrid& g, void* scratch, int64_t n_pixels,
                          int64_t* n_entries, int num_sms, cudaStream_t st) {
  const int64_t n_cells = int64_t(g.gx) * g.gy;
  FpLayout L = fp_layout(scratch, n_cells, n_pixels);
  GridGeom G{float(g.x0), float(g.y0), float(1.0 / g.cell), g.gx, g.gy};
  cudaError_t e = cudaMemsetAsync(L.cell_count, 0, size_t(n_cells) * 4, st);
  if (e != cudaSuccess) return e;
  grid_insert_kernel<<<num_sms * 8, 256, 0, st>>>(M, boxes, G, L.cell_count, L.cell_off, nullptr, 0);
  if ((e = exclusive_scan<int>(L.cell_count, L.cell_off, n_cells, L, st)) != cudaSuccess) return e;
  return read_total(L.cell_off, L.cell_count, false, n_cells, n_entries, st);
}

// Stage 2: fills the grid and counts candidates per pixel; returns the total.
cudaError_t fp_grid_fill_and_count(const MeshView& M, const float4* boxes, const FpGrid& g, void* scratch,
                                   int32_t* entries, const double* cam_host, const int* bounds_dev, int64_t n_pixels,
                                   int64_t* total, int num_sms, cudaStream_t st) {
  const int64_t n_cells = int64_t(g.gx) * g.gy;
  FpLayout L = fp_layout(scratch, n_cells, n_pixels);
  GridGeom G{float(g.x0), float(g.y0), float(1.0 / g.cell), g.gx, g.gy};
  cudaError_t e = cudaMemsetAsync(L.cell_count, 0, size_t(n_cells) * 4, st);
  if (e != cudaSuccess) return e;
  grid_insert_kernel<<<num_sms * 8, 256, 0, st>>>(M, boxes, G, L.cell_count, L.cell_off, entries, 1);
  footprint_count_kernel<<<num_sms * 8, 128, 0, st>>>(boxes, G, bounds_dev, make_cam(cam_host), n_pixels,
                                                      L.cell_count, L.cell_off, entries, L.pix_count, L.pix_cand);
  if ((e = exclusive_scan<int64_t>(L.pix_count, L.pix_off, n_pixels, L, st)) != cudaSuccess) return e;
  return read_total(L.pix_off, L.pix_count, true, n_pixels, total, st);
}

cudaError_t fp_unique_build(const MeshView& M, const QueryView& qv, float4* boxes, int* bounds_dev, int g,
                            void* scratch, int64_t n_pixels, int32_t* entries, int64_t entries_cap,
                            const double* cam_host, uint8_t* mark, int32_t* out, void* info_dev,
                            FpUniqueCounts* counts, int num_sms, cudaStream_t st) {
  const int64_t n_cells = int64_t(g) * g;
  FpLayout L = fp_layout(scratch, n_cells, n_pixels);
  FpUniqueDev* info = static_cast<FpUniqueDev*>(info_dev);
  cudaError_t e = cudaMemsetAsync(info, 0, sizeof(FpUniqueDev), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(L.cell_count, 0, size_t(n_cells) * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(mark, 0, size_t(M.n_tris), st);
  if (e != cudaSuccess) return e;
  init_bounds_kernel<<<1, 32, 0, st>>>(bounds_dev);
  mesh_bounds_kernel<<<resident_grid<mesh_bounds_kernel, 256>(num_sms), 256, 0, st>>>(M, bounds_dev, boxes);
  grid_setup_kernel<<<1, 1, 0, st>>>(bounds_dev, g, info);
  const int gi = resident_grid<grid_insert_dev_kernel, 256>(num_sms);
  grid_insert_dev_kernel<<<gi, 256, 0, st>>>(M, boxes, info, L.cell_count, L.cell_off, entries, entries_cap, 0);
  if ((e = exclusive_scan<int>(L.cell_count, L.cell_off, n_cells, L, st)) != cudaSuccess) return e;
  grid_total_kernel<<<1, 1, 0, st>>>(L.cell_count, L.cell_off, n_cells, info);
  if ((e = cudaMemsetAsync(L.cell_count, 0, size_t(n_cells) * 4, st)) != cudaSuccess) return e;
  grid_insert_dev_kernel<<<gi, 256, 0, st>>>(M, boxes, info, L.cell_count, L.cell_off, entries, entries_cap, 1);
  // One block of 128 pixels each (up to 64 per SM): footprints differ in
  // size, and the block scheduler balances them better than a fixed share.
  const int64_t gm = std::max<int64_t>(1, std::min<int64_t>((n_pixels + 127) / 128, int64_t(num_sms) * 64));
  footprint_mark_kernel<<<unsigned(gm), 128, 0, st>>>(boxes, info, bounds_dev, make_cam(cam_host), n_pixels,
                                                      L.cell_count, L.cell_off, entries, entries_cap, mark);
  const int64_t gq = std::max<int64_t>(1, std::min<int64_t>((qv.n + 255) / 256, int64_t(num_sms) * 16));
  queries_shared_kernel<<<unsigned(gq), 256, 0, st>>>(qv, &info->differ);
  const int64_t gu = std::min<int64_t>((M.n_tris + 255) / 256, int64_t(num_sms) * 8);
  unique_fill_kernel<<<unsigned(gu), 256, 0, st>>>(mark, M.n_tris, 0, &info->n_unique, out);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  FpUniqueDev h;
  if ((e = cudaMemcpyAsync(&h, info, sizeof(h), cudaMemcpyDeviceToHost, st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  counts->n_entries = int64_t(h.n_entries);
  counts->pairs = int64_t(h.pairs);
  counts->n_unique = int64_t(h.n_unique);
  counts->shared = h.differ == 0;
  return cudaSuccess;
}

size_t fp_unique_info_bytes() { return sizeof(FpUniqueDev); }

// Stage 3: writes the candidates ([total][3] int32, ordered by pixel).
cudaError_t fp_fill(const float4* boxes, const FpGrid& g, void* scratch, const int32_t* entries, const double* cam_host,
                    const int* bounds_dev, int64_t n_pixels, int32_t* out, int num_sms, cudaStream_t st) {
  const int64_t n_cells = int64_t(g.gx) * g.gy;
  FpLayout L = fp_layout(scratch, n_cells, n_pixels);
  GridGeom G{float(g.x0), float(g.y0), float(1.0 / g.cell), g.gx, g.gy};
  footprint_fill_kernel<<<num_sms * 16, 256, 0, st>>>(n_pixels, L.pix_count, L.pix_off, L.pix_cand, out);
  footprint_overflow_kernel<<<num_sms * 8, 128, 0, st>>>(boxes, G, bounds_dev, make_cam(cam_host), n_pixels,
                                                         L.cell_count, L.cell_off, entries, L.pix_count, L.pix_off,
                                                         out);
  return cudaGetLastError();
}

cudaError_t compute_mesh_bounds(const MeshView& M, int* bounds_dev, float* bounds_host, float4* boxes, int num_sms,
                                cudaStream_t st) {
  init_bounds_kernel<<<1, 32, 0, st>>>(bounds_dev);
  mesh_bounds_kernel<<<resident_grid<mesh_bounds_kernel, 256>(num_sms), 256, 0, st>>>(M, bounds_dev, boxes);
  int b[6];
  cudaError_t e = cudaMemcpyAsync(b, bounds_dev, sizeof(b), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 6; ++i) bounds_host[i] = o2f_host(b[i]);
  return cudaSuccess;
}

}  // namespace spoly
