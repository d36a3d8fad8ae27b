// Host build of the CUDA path's per-candidate numerics (test infrastructure).
// Runs the same device functions as the kernels, one candidate at a time on
// the CPU, so tests can exercise kernel arithmetic without a GPU.  It is not
// a product path and it makes no parity claim: the GPU tests do.
#define SPOLY_HOST_BUILD 1
#include "k1_polish.cuh"

using namespace spoly;

namespace {

template <int DB>
int isolate_one(const TriD& tr, const K1Sys<DB>& s, int precision, RootItem (&items)[kRD + 1], unsigned& nv,
                unsigned& np, int* status) {
  int r = -2;
  if (precision == 1 && !flat_shaded(tr)) r = k1_isolate_dispatch<float, DB>(s, items, 0, nv, np);
  status[0] = r;
  if (r != -2) return r;
  r = k1_isolate_dispatch<double, DB>(s, items, 0, nv, np);
  if (r != -2) return r;
  return k1_generic_one<DB>(s, items, 0, nv, np);
}

template <int DB>
int run(const TriD& tr, const QueryD& qd, int precision, double* out, int cap, int* status) {
  K1Sys<DB> s;
  if (!k1_system<DB>(tr, qd, s)) {
    status[0] = -1;
    return 0;
  }
  RootItem items[kRD + 1];
  unsigned nv = 0, npref = 0, lost = 0, nu = 0;
  const int nq = isolate_one<DB>(tr, s, precision, items, nv, npref, status);
  status[1] = int(nv);
  status[2] = nq;
  int ntang = 0;
  for (int i = 0; i < nq; ++i) ntang += (items[i].flags & SPOLY_FLAG_TANGENT) ? 1 : 0;
  status[4] = ntang;
  int total = 0;
  PixelFilter nofilter{};
  k1_chain_solve<DB>(s, true, tr, qd, items, nq, 0, 0, nofilter, lost, nu, [&](const spoly_path& p) {
    if (total < cap) {
      out[3 * total] = p.uv[0][0];
      out[3 * total + 1] = p.uv[0][1];
      out[3 * total + 2] = double(p.flags);
      ++total;
    }
  });
  status[3] = int(lost);
  return total;
}

}  // namespace

// status[0]: first isolation result (-2: sent to the FP64 side path, -1:
// degenerate, >= 0 brackets); status[1]: roots isolated; status[2]: brackets
// queued; status[3]: brackets lost in the polish; status[4]: tangent brackets.  out: (u, v, flags) rows.
extern "C" int host_k1_candidate(const double* tri18, const double* x0, const double* x2, int type, double eta0,
                                 double eta1, int precision, double* out, int cap, int* status) {
  TriD tr = load_tri(tri18, 1, 0);
  QueryD qd;
  qd.x0 = mk(x0[0], x0[1], x0[2]);
  qd.x2 = mk(x2[0], x2[1], x2[2]);
  qd.eta0 = eta0;
  qd.eta1 = eta1;
  qd.type = type;
  return type == SPOLY_R ? run<4>(tr, qd, precision, out, cap, status) : run<6>(tr, qd, precision, out, cap, status);
}
