// The last steps of the path phase (Sec. 4.3): the visibility test of every
// admissible path and its contribution, accumulated per pixel into a glint
// image (Sec. 5.1).
//
// Visibility.  A path x0 -> x1 (-> x2) -> x_last is rejected when a segment
// between consecutive vertices meets a triangle strictly inside it (ray
// parameter in (1e-9, 1 - 1e-9); the segment's own end triangles are
// excluded).  Segments walk a uniform grid over the mesh's xy extent (2D
// DDA, one cell at a time); a cell whose z range misses the segment's z
// range over the cell is skipped, the others test their triangles with an
// FP64 Moller-Trumbore intersection.  One thread per path: the paths of a
// step are few and each walk is short.
//
// Contribution.  The irradiance at the camera point x0 of the point light
// (intensity I) at x_last carried through the chain: a ray leaving the light
// toward the last vertex is perturbed by eps in two directions perpendicular
// to it and traced back through the planes of the chain's triangles
// (interpolated normals; mirror reflection or Snell refraction); J is the
// derivative of the two components of (outgoing direction - direction from
// the traced first vertex y to x0) perpendicular to the path's direction,
// by central differences in FP64, and f = I / (|y - x0|^2 |det J|).  For a
// flat mirror this is the inverse square law of the light's mirror image.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctx.cuh"
#include "scan.cuh"

namespace spoly {
namespace {

constexpr double kVisEps = 1e-9;    // ray parameter band excluded at both ends of a segment
constexpr double kFdStep = 1e-6;    // central-difference step of the contribution's Jacobian
constexpr float kBoxPad = 1e-6f;    // relative padding of FP32 triangle boxes and cell z ranges

SPOLY_D int f2o(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
SPOLY_D float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }
int f2o_host(float f) {
  int i;
  std::memcpy(&i, &f, 4);
  return i >= 0 ? i : i ^ 0x7fffffff;
}

struct Grid {
  double x0, y0, cell, inv;
  int gx, gy;
};

SPOLY_D void cell_span(const Grid& G, float lo, float hi, double o, int n, int& c0, int& c1) {
  c0 = max(0, min(n - 1, int(floor((double(lo) - o) * G.inv))));
  c1 = max(0, min(n - 1, int(floor((double(hi) - o) * G.inv))));
}

// Padded FP32 box of triangle t: x, y and z ranges (outward rounding plus a
// relative pad, so that the box holds the FP64 triangle).
SPOLY_D void tri_box(const MeshView& M, int64_t t, float (&lo)[3], float (&hi)[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    double a = M.tri[int64_t(c) * M.n_tris + t], b = a;
#pragma unroll
    for (int v = 1; v < 3; ++v) {
      const double x = M.tri[int64_t(3 * v + c) * M.n_tris + t];
      a = fmin(a, x);
      b = fmax(b, x);
    }
    const float fa = __double2float_rd(a), fb = __double2float_ru(b);
    const float pad = kBoxPad * (1.0f + fmaxf(fabsf(fa), fabsf(fb)));
    lo[c] = fa - pad;
    hi[c] = fb + pad;
  }
}

// pass 0: per-cell counts and z ranges; pass 1: the cell entries.
__global__ void vis_grid_kernel(MeshView M, Grid G, int* count, int* zlo, int* zhi, const int64_t* off, int* cursor,
                                int32_t* entries, int pass) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < M.n_tris; t += stride) {
    float lo[3], hi[3];
    tri_box(M, t, lo, hi);
    int cx0, cx1, cy0, cy1;
    cell_span(G, lo[0], hi[0], G.x0, G.gx, cx0, cx1);
    cell_span(G, lo[1], hi[1], G.y0, G.gy, cy0, cy1);
    for (int cy = cy0; cy <= cy1; ++cy)
      for (int cx = cx0; cx <= cx1; ++cx) {
        const int64_t c = int64_t(cy) * G.gx + cx;
        if (pass == 0) {
          atomicAdd(count + c, 1);
          atomicMin(zlo + c, f2o(lo[2]));
          atomicMax(zhi + c, f2o(hi[2]));
        } else {
          entries[off[c] + atomicAdd(cursor + c, 1)] = int32_t(t);
        }
      }
  }
}

__global__ void fill_int_kernel(int* a, int64_t n, int v) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    a[i] = v;
}

struct VisView {
  MeshView M;
  Grid G;
  const int* count;
  const int64_t* off;
  const int32_t* entries;
  const int* zlo;
  const int* zhi;
  double zmin, zmax;  // the mesh's z range, padded: a segment outside it meets no triangle
};

// Segment a -> b against triangle t (FP64 Moller-Trumbore): a hit strictly
// inside (kVisEps, 1 - kVisEps).
SPOLY_D bool seg_hits_tri(const MeshView& M, int t, d3 a, d3 d) {
  auto g = [&](int row) { return __ldg(M.tri + int64_t(row) * M.n_tris + t); };
  const d3 p0 = mk(g(0), g(1), g(2));
  const d3 e1 = mk(g(3), g(4), g(5)) - p0, e2 = mk(g(6), g(7), g(8)) - p0;
  const d3 pv = cross(d, e2);
  const double det = dot(e1, pv);
  if (!(fabs(det) > 1e-300)) return false;
  const double inv = 1.0 / det;
  const d3 s = a - p0;
  const double u = dot(s, pv) * inv;
  if (u < 0.0 || u > 1.0) return false;
  const d3 qv = cross(s, e1);
  const double v = dot(d, qv) * inv;
  if (v < 0.0 || u + v > 1.0) return false;
  const double tt = dot(e2, qv) * inv;
  return tt > kVisEps && tt < 1.0 - kVisEps;
}

// True when the segment a -> b is blocked (excluding triangles ea, eb).
SPOLY_D bool segment_blocked(const VisView& V, d3 a, d3 b, int ea, int eb) {
  const Grid& G = V.G;
  const d3 d = b - a;
  // clip the xy projection to the grid's extent
  const double X0 = G.x0, X1 = G.x0 + G.gx * G.cell, Y0 = G.y0, Y1 = G.y0 + G.gy * G.cell;
  double t0 = 0.0, t1 = 1.0;
  auto clip = [&](double p, double dp, double lo, double hi) {
    if (fabs(dp) < 1e-300) return p >= lo && p <= hi;
    double ta = (lo - p) / dp, tb = (hi - p) / dp;
    if (ta > tb) {
      const double tmp = ta;
      ta = tb;
      tb = tmp;
    }
    t0 = fmax(t0, ta);
    t1 = fmin(t1, tb);
    return t0 <= t1;
  };
  // and to the mesh's z slab: from a camera or a light above a heightfield,
  // only the segment's end near the surface needs the walk
  if (!clip(a.x, d.x, X0, X1) || !clip(a.y, d.y, Y0, Y1) || !clip(a.z, d.z, V.zmin, V.zmax)) return false;
  // 2D DDA from the entry cell
  const double px = a.x + t0 * d.x, py = a.y + t0 * d.y;
  int cx = max(0, min(G.gx - 1, int(floor((px - G.x0) * G.inv))));
  int cy = max(0, min(G.gy - 1, int(floor((py - G.y0) * G.inv))));
  const int sx = d.x > 0 ? 1 : -1, sy = d.y > 0 ? 1 : -1;
  const double inf = 1e300;
  const double dtx = fabs(d.x) > 1e-300 ? G.cell / fabs(d.x) : inf;
  const double dty = fabs(d.y) > 1e-300 ? G.cell / fabs(d.y) : inf;
  double tx = fabs(d.x) > 1e-300 ? (G.x0 + (cx + (sx > 0 ? 1 : 0)) * G.cell - a.x) / d.x : inf;
  double ty = fabs(d.y) > 1e-300 ? (G.y0 + (cy + (sy > 0 ? 1 : 0)) * G.cell - a.y) / d.y : inf;
  double tc = t0;
  const int max_steps = G.gx + G.gy + 4;
  for (int step = 0; step < max_steps; ++step) {
    const double tn = fmin(fmin(tx, ty), t1);
    const int64_t c = int64_t(cy) * G.gx + cx;
    const int n = V.count[c];
    if (n > 0) {
      const double za = a.z + tc * d.z, zb = a.z + tn * d.z;
      const float zl = o2f(V.zlo[c]), zh = o2f(V.zhi[c]);
      if (fmin(za, zb) <= double(zh) && fmax(za, zb) >= double(zl)) {
        const int64_t o = V.off[c];
        for (int k = 0; k < n; ++k) {
          const int t = V.entries[o + k];
          if (t == ea || t == eb) continue;
          if (seg_hits_tri(V.M, t, a, d)) return true;
        }
      }
    }
    if (tn >= t1) break;
    tc = tn;
    if (tx <= ty) {
      cx += sx;
      tx += dtx;
    } else {
      cy += sy;
      ty += dty;
    }
    if (cx < 0 || cx >= G.gx || cy < 0 || cy >= G.gy) break;
  }
  return false;
}

// Paths in the set's buffer: the device count, capped by the capacity.
SPOLY_D int64_t path_count(const unsigned long long* counters, int64_t cap) {
  const unsigned long long n = *(volatile unsigned long long*)(counters + C_ADMISSIBLE);
  return int64_t(n < (unsigned long long)cap ? n : cap);
}

__global__ void visibility_kernel(VisView V, QueryView qv, spoly_path* paths, unsigned long long* counters,
                                  int64_t cap, unsigned long long* n_visible) {
  const int64_t n = path_count(counters, cap);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    spoly_path& p = paths[i];
    const int q = p.query;
    const int k2 = p.tri[1] >= 0;
    // the chain's query: x_first and x_last of the path's query (with the
    // pixel assignment every pixel shares them)
    const d3 x0 = mk(qv.x_first[3 * q], qv.x_first[3 * q + 1], qv.x_first[3 * q + 2]);
    const d3 xl = mk(qv.x_last[3 * q], qv.x_last[3 * q + 1], qv.x_last[3 * q + 2]);
    const d3 x1 = mk(p.x[0][0], p.x[0][1], p.x[0][2]);
    bool blocked = segment_blocked(V, x0, x1, -1, p.tri[0]);
    if (k2) {
      const d3 x2 = mk(p.x[1][0], p.x[1][1], p.x[1][2]);
      blocked = blocked || segment_blocked(V, x1, x2, p.tri[0], p.tri[1]) || segment_blocked(V, x2, xl, p.tri[1], -1);
    } else {
      blocked = blocked || segment_blocked(V, x1, xl, p.tri[0], -1);
    }
    if (blocked) p.flags |= SPOLY_FLAG_OCCLUDED;
    else atomicAdd(n_visible, 1ull);
  }
}

SPOLY_D d3 unit(d3 a) { return (1.0 / norm(a)) * a; }

SPOLY_D void perp_basis(d3 w, d3& a, d3& b) {
  a = unit(cross(w, fabs(w.x) < 0.9 ? mk(1.0, 0.0, 0.0) : mk(0.0, 1.0, 0.0)));
  b = cross(w, a);
}

// Outgoing direction at a vertex of unit normal n; false on total internal
// reflection.
SPOLY_D bool scatter(d3& w, d3 n, int type, double eta_in, double eta_out) {
  if (type == SPOLY_R) {
    w = w - (2.0 * dot(w, n)) * n;
    return true;
  }
  if (dot(w, n) > 0.0) n = -1.0 * n;
  const double c = -dot(w, n), r = eta_in / eta_out;
  const double k = 1.0 - r * r * (1.0 - c * c);
  if (k < 0.0) return false;
  w = r * w + (r * c - sqrt(k)) * n;
  return true;
}

// Traces y + s w through the planes of triangles tris[0..k) (interpolated
// normals at the barycentric point of each plane hit).
SPOLY_D bool trace(const MeshView& M, d3& y, d3& w, const int (&tris)[2], const int (&types)[2],
                   const double (&etas)[3], int k) {
  w = unit(w);
  for (int i = 0; i < k; ++i) {
    const TriD T = load_tri(M.tri, M.n_tris, tris[i]);
    const d3 e1 = T.p1 - T.p0, e2 = T.p2 - T.p0;
    const d3 nrm = cross(e1, e2);
    const double den = dot(w, nrm);
    if (!(fabs(den) > 1e-300)) return false;
    y = y + (dot(T.p0 - y, nrm) / den) * w;
    const double g11 = dot(e1, e1), g12 = dot(e1, e2), g22 = dot(e2, e2);
    const double r1 = dot(y - T.p0, e1), r2 = dot(y - T.p0, e2);
    const double det = g11 * g22 - g12 * g12;
    const double u = (r1 * g22 - r2 * g12) / det, v = (g11 * r2 - g12 * r1) / det;
    const d3 n = unit(T.n0 + u * (T.n1 - T.n0) + v * (T.n2 - T.n0));
    if (!scatter(w, n, types[i], etas[i], etas[i + 1])) return false;
    w = unit(w);
  }
  return true;
}

__global__ void contribution_kernel(MeshView M, QueryView qv, const spoly_path* paths, unsigned long long* counters,
                                    int64_t cap, double intensity, double* per_path, double* image,
                                    int64_t image_size) {
  const int64_t n = path_count(counters, cap);
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
    const spoly_path p = paths[i];
    double f = 0.0;
    if (!(p.flags & SPOLY_FLAG_OCCLUDED)) {
      const int q = p.query, k = p.tri[1] >= 0 ? 2 : 1;
      const d3 x0 = mk(qv.x_first[3 * q], qv.x_first[3 * q + 1], qv.x_first[3 * q + 2]);
      const d3 xl = mk(qv.x_last[3 * q], qv.x_last[3 * q + 1], qv.x_last[3 * q + 2]);
      // the chain traced from the light: triangles, types and IORs reversed
      int tris[2], types[2];
      double etas[3];
      for (int j = 0; j < k; ++j) {
        tris[j] = p.tri[k - 1 - j];
        types[j] = qv.types[2 * q + (k - 1 - j)];
      }
      for (int j = 0; j <= k; ++j) etas[j] = qv.eta[3 * q + (k - j)];
      const d3 ylast = mk(p.x[k - 1][0], p.x[k - 1][1], p.x[k - 1][2]);
      const d3 y1 = mk(p.x[0][0], p.x[0][1], p.x[0][2]);
      const d3 wl = unit(ylast - xl);
      d3 ea, eb, pa, pb;
      perp_basis(wl, ea, eb);
      const d3 psi = unit(x0 - y1);
      perp_basis(psi, pa, pb);
      double J[2][2];
      bool ok = true;
      for (int col = 0; col < 2 && ok; ++col) {
        double F[2][2];
        for (int sgn = 0; sgn < 2 && ok; ++sgn) {
          const double h = sgn ? -kFdStep : kFdStep;
          d3 w = wl + (col == 0 ? h : 0.0) * ea + (col == 1 ? h : 0.0) * eb;
          d3 y = xl;
          ok = trace(M, y, w, tris, types, etas, k);
          const d3 diff = w - unit(x0 - y);
          F[sgn][0] = dot(diff, pa);
          F[sgn][1] = dot(diff, pb);
        }
        J[0][col] = (F[0][0] - F[1][0]) / (2.0 * kFdStep);
        J[1][col] = (F[0][1] - F[1][1]) / (2.0 * kFdStep);
      }
      const double det = fabs(J[0][0] * J[1][1] - J[0][1] * J[1][0]);
      const d3 dy = y1 - x0;
      if (ok && det > 0.0) f = intensity / (dot(dy, dy) * det);
      if (image && q >= 0 && q < image_size && f > 0.0) atomicAdd(image + q, f);
    }
    if (per_path) per_path[i] = f;
  }
}

}  // namespace
}  // namespace spoly

using namespace spoly;

extern "C" {

spoly_status spoly_visibility(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q, spoly_solution_set* set,
                              int64_t* n_visible) {
  if (!ctx) return SPOLY_EINVAL;
  if (!set || !n_visible) return fail(ctx, SPOLY_EINVAL, "visibility: set and n_visible are required");
  CK(cudaSetDevice(ctx->device), "set device");
  MeshView mv;
  QueryView qv;
  spoly_status st = stage_inputs(ctx, mesh, q, &mv, &qv);
  if (st != SPOLY_OK) return st;
  cudaStream_t s = ctx->stream;
  // grid over the mesh's xy extent, about two triangles per cell
  CK(ctx->bounds.ensure(64), "visibility bounds");
  CK(ctx->fp_boxes.ensure(size_t(mv.n_tris) * sizeof(float4)), "visibility boxes");
  float bh[6];
  CK(compute_mesh_bounds(mv, static_cast<int*>(ctx->bounds.p), bh, static_cast<float4*>(ctx->fp_boxes.p), ctx->num_sms,
                         s),
     "visibility bounds");
  const double pad = 1e-5 * (1.0 + std::max({std::fabs(bh[0]), std::fabs(bh[1]), std::fabs(bh[3]), std::fabs(bh[4])}));
  const double wx = double(bh[3]) - bh[0] + 2 * pad, wy = double(bh[4]) - bh[1] + 2 * pad;
  Grid G;
  G.cell = std::sqrt(std::max(wx * wy, 1e-30) / std::max<double>(1.0, double(mv.n_tris) / 2.0));
  G.gx = int(std::min(8192.0, std::max(1.0, std::ceil(wx / G.cell))));
  G.gy = int(std::min(8192.0, std::max(1.0, std::ceil(wy / G.cell))));
  G.cell = std::max(wx / G.gx, wy / G.gy);
  G.inv = 1.0 / G.cell;
  G.x0 = double(bh[0]) - pad;
  G.y0 = double(bh[1]) - pad;
  const int64_t nc = int64_t(G.gx) * G.gy;
  const int64_t nb = nc / scan::kScanBlock + 2;
  const size_t bytes = size_t(nc) * (4 * 4 + 8) + size_t(2 * nb + 3 * scan::kScanBlock) * 8 + 256;
  CK(ctx->vis_grid.ensure(bytes), "visibility grid");
  char* b = static_cast<char*>(ctx->vis_grid.p);
  int* count = reinterpret_cast<int*>(b);
  int* zlo = count + nc;
  int* zhi = zlo + nc;
  int* cursor = zhi + nc;
  int64_t* off = reinterpret_cast<int64_t*>(b + ((size_t(nc) * 16 + 255) & ~size_t(255)));
  int64_t* sums = off + nc;
  CK(cudaMemsetAsync(count, 0, size_t(nc) * 4, s), "visibility grid");
  CK(cudaMemsetAsync(cursor, 0, size_t(nc) * 4, s), "visibility grid");
  const int g = ctx->num_sms * 8;
  fill_int_kernel<<<g, 256, 0, s>>>(zlo, nc, f2o_host(3e38f));
  fill_int_kernel<<<g, 256, 0, s>>>(zhi, nc, f2o_host(-3e38f));
  vis_grid_kernel<<<g, 256, 0, s>>>(mv, G, count, zlo, zhi, nullptr, nullptr, nullptr, 0);
  CK(cudaGetLastError(), "visibility grid");
  CK(scan::exclusive_scan<int>(count, off, nc, sums, sums + nb, sums + 2 * nb, s), "visibility scan");
  int64_t last_off = 0;
  int last_count = 0;
  CK(cudaMemcpyAsync(&last_off, off + nc - 1, 8, cudaMemcpyDeviceToHost, s), "visibility grid");
  CK(cudaMemcpyAsync(&last_count, count + nc - 1, 4, cudaMemcpyDeviceToHost, s), "visibility grid");
  CK(cudaStreamSynchronize(s), "visibility grid");
  const int64_t n_entries = last_off + last_count;
  CK(ctx->vis_entries.ensure(size_t(std::max<int64_t>(n_entries, 1)) * 4), "visibility grid entries");
  vis_grid_kernel<<<g, 256, 0, s>>>(mv, G, count, zlo, zhi, off, cursor, static_cast<int32_t*>(ctx->vis_entries.p), 1);
  CK(cudaGetLastError(), "visibility grid");
  const double zpad = 1e-5 * (1.0 + std::max(std::fabs(bh[2]), std::fabs(bh[5])));
  VisView V{mv, G, count, off, static_cast<const int32_t*>(ctx->vis_entries.p), zlo, zhi, double(bh[2]) - zpad,
            double(bh[5]) + zpad};
  CK(ctx->flag.ensure(16), "visibility count");
  unsigned long long* nv = static_cast<unsigned long long*>(ctx->flag.p);
  CK(cudaMemsetAsync(nv, 0, 8, s), "visibility count");
  visibility_kernel<<<ctx->num_sms * 4, 64, 0, s>>>(V, qv, static_cast<spoly_path*>(set->paths.p),
                                                    static_cast<unsigned long long*>(set->counters.p), set->path_cap,
                                                    nv);
  CK(cudaGetLastError(), "visibility");
  unsigned long long h = 0;
  CK(cudaMemcpyAsync(&h, nv, 8, cudaMemcpyDeviceToHost, s), "visibility count");
  CK(cudaStreamSynchronize(s), "visibility");
  *n_visible = int64_t(h);
  return SPOLY_OK;
}

spoly_status spoly_contributions(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q,
                                 const spoly_solution_set* set, double intensity, double* per_path, double* image,
                                 int64_t image_size) {
  if (!ctx) return SPOLY_EINVAL;
  if (!set || !(intensity >= 0.0) || (image && image_size <= 0))
    return fail(ctx, SPOLY_EINVAL, "contributions: bad arguments");
  CK(cudaSetDevice(ctx->device), "set device");
  MeshView mv;
  QueryView qv;
  spoly_status st = stage_inputs(ctx, mesh, q, &mv, &qv);
  if (st != SPOLY_OK) return st;
  contribution_kernel<<<ctx->num_sms * 4, 64, 0, ctx->stream>>>(
      mv, qv, static_cast<const spoly_path*>(set->paths.p), static_cast<unsigned long long*>(set->counters.p),
      set->path_cap, intensity, per_path, image, image_size);
  CK(cudaGetLastError(), "contributions");
  CK(cudaStreamSynchronize(ctx->stream), "contributions");
  return SPOLY_OK;
}

}  // extern "C"
