// Pixel-footprint candidate builder (glints): a uniform grid over the mesh
// and, per pixel of a pinhole camera, the triangles whose bounding box meets
// the pixel's footprint on the mesh.
//
// The footprint of pixel (ix, iy) is the xy bounding box of its four corner
// rays between the planes z = zmin and z = zmax of the mesh's bounding box,
// so every surface point a pixel can see lies inside it.  A triangle is
// emitted once per pixel, from the first grid cell its bounding box shares
// with the footprint.  Emission is two-pass (count, exclusive scan, fill), so
// the chain list is ordered by pixel without global atomics.
#include <algorithm>
#include <cstring>

#include "k1.cuh"

namespace spoly {

namespace {

constexpr int kScanBlock = 1024;

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

// mesh bounds: [0..2] min xyz, [3..5] max xyz as ordered ints (slack added by the caller)
__global__ void mesh_bounds_kernel(MeshView M, int* bounds) {
  float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < M.n_tris; t += stride)
    for (int v = 0; v < 3; ++v)
      for (int c = 0; c < 3; ++c) {
        const float x = float(M.tri[int64_t(3 * v + c) * M.n_tris + t]);
        lo[c] = fminf(lo[c], x);
        hi[c] = fmaxf(hi[c], x);
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

__global__ void init_bounds_kernel(int* bounds) {
  if (threadIdx.x < 3) bounds[threadIdx.x] = f2o(3e38f);
  else if (threadIdx.x < 6) bounds[threadIdx.x] = f2o(-3e38f);
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

SPOLY_D void tri_bbox(const MeshView& M, int64_t t, float& xl, float& xh, float& yl, float& yh) {
  const float a = float(M.tri[0 * M.n_tris + t]), b = float(M.tri[3 * M.n_tris + t]), c = float(M.tri[6 * M.n_tris + t]);
  const float d = float(M.tri[1 * M.n_tris + t]), e = float(M.tri[4 * M.n_tris + t]), f = float(M.tri[7 * M.n_tris + t]);
  xl = fminf(a, fminf(b, c));
  xh = fmaxf(a, fmaxf(b, c));
  yl = fminf(d, fminf(e, f));
  yh = fmaxf(d, fmaxf(e, f));
}

// pass 0: count entries per cell; pass 1: fill (cursor = count copy)
__global__ void grid_insert_kernel(MeshView M, GridGeom G, int* cell_count, const int64_t* cell_off,
                                   int32_t* entries, int pass) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < M.n_tris; t += stride) {
    float xl, xh, yl, yh;
    tri_bbox(M, t, xl, xh, yl, yh);
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

struct CamD {
  d3 o, f, r, u;
  double th, aspect;
  int w, h;
};

SPOLY_D CamD load_cam(const double* c) {
  CamD k;
  k.o = mk(c[0], c[1], c[2]);
  k.f = mk(c[3], c[4], c[5]);
  k.r = mk(c[6], c[7], c[8]);
  k.u = mk(c[9], c[10], c[11]);
  k.th = c[12];
  k.aspect = c[13];
  k.w = int(c[14]);
  k.h = int(c[15]);
  return k;
}

// Footprint of a pixel: xy box of its corner rays between z = zlo and z = zhi.
SPOLY_D bool pixel_footprint(const CamD& C, int64_t q, float zlo, float zhi, float& xl, float& xh, float& yl,
                             float& yh) {
  const int ix = int(q % C.w), iy = int(q / C.w);
  xl = yl = 3e38f;
  xh = yh = -3e38f;
  for (int k = 0; k < 4; ++k) {
    const double sx = -1.0 + 2.0 * (ix + (k & 1)) / C.w;
    const double sy = 1.0 - 2.0 * (iy + (k >> 1)) / C.h;
    const d3 d = C.f + (sx * C.th * C.aspect) * C.r + (sy * C.th) * C.u;
    if (!(d.z < 0.0)) return false;  // a corner ray never reaches the surface slab
    for (int p = 0; p < 2; ++p) {
      const double z = p ? zhi : zlo;
      const double tt = (z - C.o.z) / d.z;
      const float x = float(C.o.x + tt * d.x), y = float(C.o.y + tt * d.y);
      xl = fminf(xl, x);
      xh = fmaxf(xh, x);
      yl = fminf(yl, y);
      yh = fmaxf(yh, y);
    }
  }
  const float m = 1e-5f * (1.f + fmaxf(fabsf(xl), fabsf(yh)));
  xl -= m;
  yl -= m;
  xh += m;
  yh += m;
  return true;
}

// pass 0: count candidates per pixel; pass 1: write them at out_off[q]
__global__ void footprint_kernel(MeshView M, GridGeom G, const int* bounds, const double* cam, int64_t n_pixels,
                                 const int* cell_count, const int64_t* cell_off, const int32_t* entries,
                                 int64_t* pix_count, const int64_t* pix_off, int32_t* out, int pass) {
  const CamD C = load_cam(cam);
  const float zlo = o2f(bounds[2]), zhi = o2f(bounds[5]);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < n_pixels; q += stride) {
    float xl, xh, yl, yh;
    int64_t n = 0, o = pass ? pix_off[q] : 0;
    if (pixel_footprint(C, q, zlo, zhi, xl, xh, yl, yh)) {
      int fx0, fx1, fy0, fy1;
      cell_range(G, xl, xh, yl, yh, fx0, fx1, fy0, fy1);
      for (int cy = fy0; cy <= fy1; ++cy)
        for (int cx = fx0; cx <= fx1; ++cx) {
          const int64_t cell = int64_t(cy) * G.gx + cx;
          const int64_t b = cell_off[cell], e = b + cell_count[cell];
          for (int64_t k = b; k < e; ++k) {
            const int32_t t = entries[k];
            float txl, txh, tyl, tyh;
            tri_bbox(M, t, txl, txh, tyl, tyh);
            if (txh < xl || txl > xh || tyh < yl || tyl > yh) continue;
            int tx0, tx1, ty0, ty1;
            cell_range(G, txl, txh, tyl, tyh, tx0, tx1, ty0, ty1);
            if (cx != max(tx0, fx0) || cy != max(ty0, fy0)) continue;  // emitted from its first shared cell
            if (pass) {
              out[3 * (o + n)] = int32_t(q);
              out[3 * (o + n) + 1] = t;
              out[3 * (o + n) + 2] = -1;
            }
            ++n;
          }
        }
    }
    if (!pass) pix_count[q] = n;
  }
}

// Exclusive scan of int64 (or int32 widened) values, in blocks of kScanBlock.
template <typename In>
__global__ void scan_block_kernel(const In* in, int64_t* out, int64_t* block_sums, int64_t n) {
  __shared__ int64_t s[kScanBlock / 32];
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  const int64_t v = i < n ? int64_t(in[i]) : 0;
  int64_t x = v;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = s[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s[lane] = w;
  }
  __syncthreads();
  const int64_t incl = x + (warp ? s[warp - 1] : 0);
  if (i < n) out[i] = incl - v;
  if (threadIdx.x == kScanBlock - 1) block_sums[blockIdx.x] = incl;
}

__global__ void scan_add_kernel(int64_t* out, const int64_t* block_off, int64_t n) {
  const int64_t i = int64_t(blockIdx.x) * kScanBlock + threadIdx.x;
  if (i < n) out[i] += block_off[blockIdx.x];
}

}  // namespace

// Scratch layout of the footprint builder (bytes, library-owned).
struct FpLayout {
  int* cell_count;
  int64_t* cell_off;
  int64_t* pix_count;
  int64_t* pix_off;
  int64_t *sums1, *sums1_off, *sums2;
};

static size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

size_t footprint_scratch_bytes(int64_t n_cells, int64_t n_pixels) {
  const int64_t nb = (std::max(n_cells, n_pixels) + kScanBlock - 1) / kScanBlock;
  return up256(n_cells * 4) + up256(n_cells * 8) + 2 * up256(n_pixels * 8) + 2 * up256(nb * 8 + 64) +
         up256(3 * kScanBlock * 8);
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
  return L;
}

// Exclusive scan with up to three levels of block sums (n <= 2^30).
template <typename In>
static cudaError_t exclusive_scan(const In* in, int64_t* out, int64_t n, const FpLayout& L, cudaStream_t st) {
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  scan_block_kernel<In><<<unsigned(nb), kScanBlock, 0, st>>>(in, out, L.sums1, n);
  if (nb > 1) {
    const int64_t nb2 = (nb + kScanBlock - 1) / kScanBlock;
    scan_block_kernel<int64_t><<<unsigned(nb2), kScanBlock, 0, st>>>(L.sums1, L.sums1_off, L.sums2, nb);
    if (nb2 > 1) {
      int64_t* s2off = L.sums2 + kScanBlock;
      scan_block_kernel<int64_t><<<1, kScanBlock, 0, st>>>(L.sums2, s2off, L.sums2 + 2 * kScanBlock, nb2);
      scan_add_kernel<<<unsigned(nb2), kScanBlock, 0, st>>>(L.sums1_off, s2off, nb);
    }
    scan_add_kernel<<<unsigned(nb), kScanBlock, 0, st>>>(out, L.sums1_off, n);
  }
  return cudaGetLastError();
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
cudaError_t fp_grid_count(const MeshView& M, const FpGrid& g, void* scratch, int64_t n_pixels, int64_t* n_entries,
                          int num_sms, cudaStream_t st) {
  const int64_t n_cells = int64_t(g.gx) * g.gy;
  FpLayout L = fp_layout(scratch, n_cells, n_pixels);
  GridGeom G{float(g.x0), float(g.y0), float(1.0 / g.cell), g.gx, g.gy};
  cudaError_t e = cudaMemsetAsync(L.cell_count, 0, size_t(n_cells) * 4, st);
  if (e != cudaSuccess) return e;
  grid_insert_kernel<<<num_sms * 8, 256, 0, st>>>(M, G, L.cell_count, L.cell_off, nullptr, 0);
  if ((e = exclusive_scan<int>(L.cell_count, L.cell_off, n_cells, L, st)) != cudaSuccess) return e;
  return read_total(L.cell_off, L.cell_count, false, n_cells, n_entries, st);
}

// Stage 2: fills the grid and counts candidates per pixel; returns the total.
cudaError_t fp_grid_fill_and_count(const MeshView& M, const FpGrid& g, void* scratch, int32_t* entries,
                                   const double* cam_dev, const int* bounds_dev, int64_t n_pixels, int64_t* total,
                                   int num_sms, cudaStream_t st) {
  const int64_t n_cells = int64_t(g.gx) * g.gy;
  FpLayout L = fp_layout(scratch, n_cells, n_pixels);
  GridGeom G{float(g.x0), float(g.y0), float(1.0 / g.cell), g.gx, g.gy};
  cudaError_t e = cudaMemsetAsync(L.cell_count, 0, size_t(n_cells) * 4, st);
  if (e != cudaSuccess) return e;
  grid_insert_kernel<<<num_sms * 8, 256, 0, st>>>(M, G, L.cell_count, L.cell_off, entries, 1);
  footprint_kernel<<<num_sms * 8, 128, 0, st>>>(M, G, bounds_dev, cam_dev, n_pixels, L.cell_count, L.cell_off, entries,
                                                L.pix_count, nullptr, nullptr, 0);
  if ((e = exclusive_scan<int64_t>(L.pix_count, L.pix_off, n_pixels, L, st)) != cudaSuccess) return e;
  return read_total(L.pix_off, L.pix_count, true, n_pixels, total, st);
}

// Stage 3: writes the candidates ([total][3] int32, ordered by pixel).
cudaError_t fp_fill(const MeshView& M, const FpGrid& g, void* scratch, const int32_t* entries, const double* cam_dev,
                    const int* bounds_dev, int64_t n_pixels, int32_t* out, int num_sms, cudaStream_t st) {
  const int64_t n_cells = int64_t(g.gx) * g.gy;
  FpLayout L = fp_layout(scratch, n_cells, n_pixels);
  GridGeom G{float(g.x0), float(g.y0), float(1.0 / g.cell), g.gx, g.gy};
  footprint_kernel<<<num_sms * 8, 128, 0, st>>>(M, G, bounds_dev, cam_dev, n_pixels, L.cell_count, L.cell_off, entries,
                                                nullptr, L.pix_off, out, 1);
  return cudaGetLastError();
}

cudaError_t compute_mesh_bounds(const MeshView& M, int* bounds_dev, float* bounds_host, int num_sms, cudaStream_t st) {
  init_bounds_kernel<<<1, 32, 0, st>>>(bounds_dev);
  mesh_bounds_kernel<<<num_sms * 4, 256, 0, st>>>(M, bounds_dev);
  int b[6];
  cudaError_t e = cudaMemcpyAsync(b, bounds_dev, sizeof(b), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < 6; ++i) bounds_host[i] = o2f_host(b[i]);
  return cudaSuccess;
}

}  // namespace spoly
