// 2-bounce chains (TT, RR), path phase per chain (after the FP64 polish in
// tt_sign.cuh):
// u1 from a(u1, v1*) = 0, u2 from the rational mapping (Eq. eq_rct),
// path-space Newton on h x n = 0 at both vertices (Eq. eq_ch), sidedness,
// in-triangle tests and de-duplication of the chain's paths.
#include "tt_kernels.cuh"

namespace spoly {

// ------------------------------------------------------------- path phase
struct TTPath {
  double w[4];
  d3 x1, x2;
  double res;
  uint32_t flags;
};

SPOLY_D d3 unit3(d3 a) { return (1.0 / norm(a)) * a; }

// h x n / (|h| |n|) with h = eta_out d1_hat - eta_in d0_hat (Eq. eq_ch;
// reflection: both IORs 1), and the sidedness test: refraction crosses the
// surface (d0 . n and d1 . n of one sign), reflection stays on its side
// (opposite signs).
SPOLY_D d3 vertex_residual(d3 xp, d3 x, d3 xn, d3 n, double ein, double eout, bool refl, bool* side) {
  const d3 d0 = x - xp, d1 = xn - x;
  const d3 h = eout * unit3(d1) - ein * unit3(d0);
  const double s0 = dot(d0, n), s1 = dot(d1, n);
  *side = (refl ? ((s0 < 0.0) != (s1 < 0.0)) : ((s0 < 0.0) == (s1 < 0.0))) && s0 != 0.0 && s1 != 0.0;
  return (1.0 / (norm(h) * norm(n))) * cross(h, n);
}

struct TTGeom {
  TriD t1, t2;
  d3 x0, x3;
  double e0, e1, e2;
  bool refl;  // two reflections (RR); else two refractions (TT)
};

SPOLY_D void tt_points(const TTGeom& G, const double (&w)[4], d3& x1, d3& n1, d3& x2, d3& n2) {
  x1 = G.t1.p0 + w[0] * (G.t1.p1 - G.t1.p0) + w[1] * (G.t1.p2 - G.t1.p0);
  n1 = G.t1.n0 + w[0] * (G.t1.n1 - G.t1.n0) + w[1] * (G.t1.n2 - G.t1.n0);
  x2 = G.t2.p0 + w[2] * (G.t2.p1 - G.t2.p0) + w[3] * (G.t2.p2 - G.t2.p0);
  n2 = G.t2.n0 + w[2] * (G.t2.n1 - G.t2.n0) + w[3] * (G.t2.n2 - G.t2.n0);
}

SPOLY_D void tangent_basis(d3 n, d3& a, d3& b) {
  n = unit3(n);
  const double ax = fabs(n.x), ay = fabs(n.y), az = fabs(n.z);
  const d3 e = (ax <= ay && ax <= az) ? mk(1, 0, 0) : (ay <= az ? mk(0, 1, 0) : mk(0, 0, 1));
  a = unit3(cross(n, e));
  b = cross(n, a);
}

SPOLY_D void tt_F(const TTGeom& G, const double (&w)[4], d3 a1, d3 b1, d3 a2, d3 b2, double (&f)[4]) {
  d3 x1, n1, x2, n2;
  tt_points(G, w, x1, n1, x2, n2);
  bool s;
  const d3 r1 = vertex_residual(G.x0, x1, x2, n1, G.e0, G.e1, G.refl, &s);
  const d3 r2 = vertex_residual(x1, x2, G.x3, n2, G.e1, G.e2, G.refl, &s);
  f[0] = dot(r1, a1);
  f[1] = dot(r1, b1);
  f[2] = dot(r2, a2);
  f[3] = dot(r2, b2);
}

// Newton on the four tangential components (bases fixed at the start),
// Jacobian by central differences, at most kTTNewtonIters steps.
SPOLY_D void tt_newton(const TTGeom& G, double (&w)[4]) {
  d3 x1, n1, x2, n2, a1, b1, a2, b2;
  tt_points(G, w, x1, n1, x2, n2);
  tangent_basis(n1, a1, b1);
  tangent_basis(n2, a2, b2);
  for (int it = 0; it < kTTNewtonIters; ++it) {
    double f[4];
    tt_F(G, w, a1, b1, a2, b2, f);
    if (fmax(fmax(fabs(f[0]), fabs(f[1])), fmax(fabs(f[2]), fabs(f[3]))) < 1e-15) break;
    double J[4][5];
    for (int k = 0; k < 4; ++k) {
      double wp[4] = {w[0], w[1], w[2], w[3]}, wm[4] = {w[0], w[1], w[2], w[3]};
      wp[k] += 1e-7;
      wm[k] -= 1e-7;
      double fp[4], fm[4];
      tt_F(G, wp, a1, b1, a2, b2, fp);
      tt_F(G, wm, a1, b1, a2, b2, fm);
      for (int r = 0; r < 4; ++r) J[r][k] = (fp[r] - fm[r]) / 2e-7;
    }
    for (int r = 0; r < 4; ++r) J[r][4] = -f[r];
    // Gaussian elimination with partial pivoting on the 4 x 5 system
    bool sing = false;
    for (int c = 0; c < 4; ++c) {
      int p = c;
      for (int r = c + 1; r < 4; ++r)
        if (fabs(J[r][c]) > fabs(J[p][c])) p = r;
      if (J[p][c] == 0.0) {
        sing = true;
        break;
      }
      if (p != c)
        for (int k = 0; k < 5; ++k) {
          const double t = J[c][k];
          J[c][k] = J[p][k];
          J[p][k] = t;
        }
      for (int r = c + 1; r < 4; ++r) {
        const double m = J[r][c] / J[c][c];
        for (int k = c; k < 5; ++k) J[r][k] -= m * J[c][k];
      }
    }
    if (sing) break;
    double dx[4];
    for (int r = 3; r >= 0; --r) {
      double s = J[r][4];
      for (int k = r + 1; k < 4; ++k) s -= J[r][k] * dx[k];
      dx[r] = s / J[r][r];
    }
    for (int k = 0; k < 4; ++k) w[k] += dx[k];
  }
}

// The chains of this batch with at least one polished root, listed so that
// the path kernel's warps are full of chains with work (a few percent of
// the chains have one).
__global__ void tt_active_kernel(TTParams P, int64_t chain_begin, int64_t chain_end) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t base = chain_begin + int64_t(blockIdx.x) * blockDim.x; base < chain_end; base += stride) {
    const int64_t c = base + threadIdx.x;
    bool has = false;
    if (c < chain_end) {
      const int s0 = P.chain_sys[2 * c], ns = P.chain_sys[2 * c + 1];
      for (int si = s0; si < s0 + ns && !has; ++si) {
        const TTSys sy = P.sys[si];
        if (sy.n < 1) continue;
        for (int k = 0; k < sy.n_items && !has && sy.first_item + k < P.queue_cap; ++k)
          has = (P.queue[sy.first_item + k].flags & kTTValid) != 0;
      }
    }
    const unsigned long long slot = warp_append(P.active_n, has ? 1u : 0u);
    if (has) P.active[slot] = int32_t(c);
  }
}

// The path phase of the listed chains (one thread per chain).
__global__ void __launch_bounds__(64) tt_path_kernel(TTParams P) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  const int64_t n_active = int64_t(*P.active_n);
  for (int64_t base = int64_t(blockIdx.x) * blockDim.x; base < n_active; base += stride) {
    const int64_t idx = base + threadIdx.x;
    const int64_t c = idx < n_active ? int64_t(P.active[idx]) : 0;
    TTPath out[6];
    int np = 0;
    unsigned n_u = 0;
    if (idx < n_active) {
      const int q = P.chains[3 * c], t1i = P.chains[3 * c + 1], t2i = P.chains[3 * c + 2];
      TTGeom G;
      G.t1 = load_tri(P.mesh.tri, P.mesh.n_tris, t1i);
      G.t2 = load_tri(P.mesh.tri, P.mesh.n_tris, t2i);
      const QueryD qd = load_query(P.qv.x_first, P.qv.x_last, P.qv.eta, P.qv.types, q);
      G.x0 = qd.x0;
      G.x3 = qd.x2;
      G.refl = chain_kind(P.qv.types, q) == kChainRR;
      G.e0 = G.refl ? 1.0 : qd.eta0;
      G.e1 = G.refl ? 1.0 : qd.eta1;
      G.e2 = G.refl ? 1.0 : P.qv.eta[3 * q + 2];
      const int s0 = P.chain_sys[2 * c], ns = P.chain_sys[2 * c + 1];
      const d3 c1 = (1.0 / 3.0) * (G.t1.p0 + G.t1.p1 + G.t1.p2);
      const d3 ncen = (1.0 / 3.0) * (G.t1.n0 + G.t1.n1 + G.t1.n2);
      const double s_arg = dot(ncen, ncen) * dot(c1 - G.x0, c1 - G.x0);
      const double er = G.e0 / G.e1;
      for (int si = s0; si < s0 + ns; ++si) {
        const TTSys sy = P.sys[si];
        if (sy.n < 1) continue;
        const int64_t col = si - P.sys_offset;
        const double* sc = P.scratch + col * kTTKeep;
        const int64_t st = 1;
        const GP A{const_cast<double*>(sc) + int64_t(kOffA) * st, st, kTTDa};
        const GP B{const_cast<double*>(sc) + int64_t(kOffB) * st, st, kTTDb};
        const GP UT{const_cast<double*>(sc) + int64_t(kOffUt) * st, st, kTTDmap};
        const GP VT{const_cast<double*>(sc) + int64_t(kOffVt) * st, st, kTTDmap};
        const GP KA{const_cast<double*>(sc) + int64_t(kOffKap) * st, st, kTTDmap};
        for (int k = 0; k < sy.n_items; ++k) {
          if (sy.first_item + k >= P.queue_cap) break;  // brackets past an overflowed queue were not kept
          const RootItem item = P.queue[sy.first_item + k];
          if (!(item.flags & kTTValid)) continue;
          const double v = item.zlo;
          // u1 from a(u1, v*) = 0 on [-delta, 1 - v* + delta]
          double ac[kTTDa + 1];
          double am = 0.0;
          for (int i = 0; i <= kTTDa; ++i) {
            double r = 0.0;
            if (i <= sy.da)
              for (int j = kTTDa - i; j >= 0; --j) r = fma(r, v, A.at(i, j));
            ac[i] = r;
            am = fmax(am, fabs(r));
          }
          int deg = -1;
          for (int i = 0; i <= kTTDa; ++i)
            if (fabs(ac[i]) > kTrim * am) deg = i;
          if (deg < 1) continue;
          double rs = 0.0;
          for (int i = 0; i <= deg; ++i) rs += fabs(ac[i]);
          double blo[kTTDa + 1], bhi[kTTDa + 1];
          uint32_t bfl[kTTDa + 1];
          const int nr = isolate<double, kTTDa>(ac, deg, -kDelta, 1.0 - v + kDelta, 1e-14, kTangent64, rs, blo, bhi,
                                                bfl);
          for (int r = 0; r < nr; ++r) {
            const double u = 0.5 * (blo[r] + bhi[r]);
            // b(u, v*) must vanish with a, measured against the magnitude
            // bound of evaluating b there, sum_ij |b_ij| |u|^i |v*|^j (the
            // coefficients of b(., v*) alone all vanish when b does not
            // depend on u, as for two flat mirrors)
            double bv = 0.0, bs = 0.0;
            const double au = fmax(1.0, fabs(u)), av = fabs(v);
            for (int i = sy.db; i >= 0; --i) {
              double row = 0.0, rabs = 0.0;
              for (int j = kTTDb - i; j >= 0; --j) {
                row = fma(row, v, B.at(i, j));
                rabs = fma(rabs, av, fabs(B.at(i, j)));
              }
              bv = fma(bv, u, row);
              bs = fma(bs, au, rabs);
            }
            if (fabs(bv) > 1e-6 * bs) continue;
            const double kap = gp_eval(KA, u, v);
            if (kap == 0.0) continue;
            double w[4] = {u, v, gp_eval(UT, u, v) / kap, gp_eval(VT, u, v) / kap};
            if (sy.flags & SPOLY_FLAG_SQRT_SPLIT) {
              // keep the root only in the piece its approximant argument falls in
              d3 x1, n1, x2, n2;
              tt_points(G, w, x1, n1, x2, n2);
              const d3 d = x1 - G.x0;
              const double nd = dot(n1, n1) * dot(d, d), dn = dot(d, n1);
              double x = (nd - er * er * (nd - dn * dn)) / s_arg;
              x = fmin(fmax(x, 0.0), 1.0);
              int pc = 0;
              while (pc < kSqrtPieces - 1 && x >= P.sqrt_tab.breaks[pc + 1]) ++pc;
              if (pc != sy.piece) continue;
            }
            ++n_u;
            tt_newton(G, w);
            d3 x1, n1, x2, n2;
            tt_points(G, w, x1, n1, x2, n2);
            bool sd1, sd2;
            const d3 r1 = vertex_residual(G.x0, x1, x2, n1, G.e0, G.e1, G.refl, &sd1);
            const d3 r2 = vertex_residual(x1, x2, G.x3, n2, G.e1, G.e2, G.refl, &sd2);
            const double res = fmax(norm(r1), norm(r2));
            if (!sd1 || !sd2 || !(res < kResidual)) continue;
            const double m1 = fmin(fmin(w[0], w[1]), 1.0 - w[0] - w[1]);
            const double m2 = fmin(fmin(w[2], w[3]), 1.0 - w[2] - w[3]);
            if (m1 < 0.0 || m2 < 0.0) continue;
            uint32_t flags = (item.flags & SPOLY_FLAG_ILL_COND) | SPOLY_FLAG_NEWTON | (sy.flags & SPOLY_FLAG_SQRT_SPLIT);
            if (fmin(m1, m2) < kEdgeEps) flags |= SPOLY_FLAG_EDGE;
            bool dup = false;
            for (int o = 0; o < np; ++o)
              if (fabs(out[o].w[0] - w[0]) <= 1e-9 && fabs(out[o].w[1] - w[1]) <= 1e-9 &&
                  fabs(out[o].w[2] - w[2]) <= 1e-9 && fabs(out[o].w[3] - w[3]) <= 1e-9) {
                out[o].flags |= flags;
                dup = true;
              }
            if (dup || np >= 6) continue;
            TTPath& pth = out[np++];
            for (int k2 = 0; k2 < 4; ++k2) pth.w[k2] = w[k2];
            pth.x1 = x1;
            pth.x2 = x2;
            pth.res = res;
            pth.flags = flags;
          }
        }
      }
    }
    warp_count(P.counters + TT_UROOTS, n_u);
    unsigned n_flag = 0;
    for (int k = 0; k < np; ++k) n_flag += (out[k].flags & SPOLY_FLAG_ILL_COND) ? 1u : 0u;
    warp_count(P.counters + TT_FLAGGED, n_flag);
    warp_count(P.counters + TT_ADMISSIBLE, unsigned(np));
    const unsigned long long slot = warp_append(P.path_counter, unsigned(np));
    for (int k = 0; k < np; ++k) {
      const unsigned long long idx = slot + k;
      if (idx >= (unsigned long long)P.path_cap) continue;
      spoly_path p;
      p.query = P.chains[3 * c];
      p.tri[0] = P.chains[3 * c + 1];
      p.tri[1] = P.chains[3 * c + 2];
      p.chain = P.chain_ids ? P.chain_ids[c] : int32_t(c);
      p.uv[0][0] = out[k].w[0];
      p.uv[0][1] = out[k].w[1];
      p.uv[1][0] = out[k].w[2];
      p.uv[1][1] = out[k].w[3];
      p.x[0][0] = out[k].x1.x;
      p.x[0][1] = out[k].x1.y;
      p.x[0][2] = out[k].x1.z;
      p.x[1][0] = out[k].x2.x;
      p.x[1][1] = out[k].x2.y;
      p.x[1][2] = out[k].x2.z;
      p.residual = float(out[k].res);
      p.flags = out[k].flags;
      P.paths[idx] = p;
    }
  }
}

cudaError_t launch_tt_paths(const TTParams& P, int64_t chain_begin, int64_t chain_end, int num_sms, cudaStream_t st) {
  if (chain_end <= chain_begin) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(P.active_n, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int64_t ga = std::min<int64_t>((chain_end - chain_begin + 255) / 256, int64_t(num_sms) * 8);
  tt_active_kernel<<<int(ga), 256, 0, st>>>(P, chain_begin, chain_end);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t g = std::min<int64_t>((chain_end - chain_begin + 63) / 64, int64_t(num_sms) * 8);
  tt_path_kernel<<<int(g), 64, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace spoly
