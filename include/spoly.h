/* spoly.h -- C ABI of the GB300-native specular-polynomial solver.
 *
 * The library finds every admissible specular path between two fixed
 * endpoints (separators x0 and x_{k+1}) through a candidate chain of k
 * triangles with barycentrically interpolated vertex normals, following
 * "Specular Polynomials" (Fan et al. 2024):
 *   - problem statement: Sec. 3.1 (Eq. eq_xi, eq_ni, eq_ch);
 *   - bivariate systems: Sec. 3.5 (R: Eq. eq_coplane + eq_pf_result,
 *     T: Eq. eq_coplane + eq_cpf_result);
 *   - elimination: Sec. 4.1 (Bezout matrix, Eq. eq_bezout);
 *   - univariate phase: Sec. 4.2 (Laplace expansion + recursive-derivative
 *     isolation for one bounce; determinant bisection for k bounces);
 *   - path phase: Sec. 4.3 (u recovery, path-space check, in-triangle test).
 *
 * Conventions for every entry point
 *   - All inputs are plain pointers plus sizes.  Each input struct says
 *     whether its pointers are host or device memory (`on_device`).  The
 *     caller owns every input buffer and keeps it valid until the call
 *     returns (or, with SPOLY_SOLVE_ASYNC, until the context's stream has
 *     passed the enqueued work).
 *   - The library owns its handles (spoly_ctx, spoly_chains,
 *     spoly_solution_set) and the device memory behind them; free them with
 *     the matching *_destroy / *_free call.  Handles may be reused across
 *     calls, which keeps allocation out of steady-state loops.
 *   - All device work is enqueued on the context's CUDA stream.
 *   - Every call returns a spoly_status; nothing throws across the ABI.  On
 *     an error the context keeps a message (spoly_last_error).  Errors:
 *       SPOLY_EINVAL       bad pointer, shape or value (message names it)
 *       SPOLY_ENOMEM       device allocation failed
 *       SPOLY_ECUDA        a CUDA call failed (message has the CUDA error)
 *       SPOLY_ECAPACITY    the caller's output buffer is too small;
 *                          *n_total holds the required count and nothing is
 *                          silently truncated
 *       SPOLY_ETIMEOUT     a bounded device-side wait gave up
 *       SPOLY_EUNSUPPORTED bounce count or scattering type not built
 */
#ifndef SPOLY_H_
#define SPOLY_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t spoly_status;
#define SPOLY_OK 0
#define SPOLY_EINVAL (-1)
#define SPOLY_ENOMEM (-2)
#define SPOLY_ECUDA (-3)
#define SPOLY_ECAPACITY (-4)
#define SPOLY_ETIMEOUT (-5)
#define SPOLY_EUNSUPPORTED (-6)

/* Scattering type per bounce (Sec. 3.5, Heckbert notation). */
#define SPOLY_R 0 /* reflection */
#define SPOLY_T 1 /* refraction */

/* Path flags. */
#define SPOLY_FLAG_ILL_COND 1u      /* |r'(v*)| / sum|r_i| < 1e-8, or a tangent root */
#define SPOLY_FLAG_EDGE 2u          /* min(u, v, 1-u-v) within 1e-7 of the edge */
#define SPOLY_FLAG_BACKFACE 4u      /* (x0 - x1) . n < 0 */
#define SPOLY_FLAG_NEWTON 8u        /* refined by path-space Newton (k = 2) */
#define SPOLY_FLAG_SQRT_SPLIT 16u   /* rational sqrt piece split (k = 2, T) */
#define SPOLY_FLAG_TANGENT 32u      /* root found at a critical point of r */
#define SPOLY_FLAG_OCCLUDED 64u     /* a segment of the path is blocked (spoly_visibility) */

typedef struct spoly_ctx spoly_ctx;
typedef struct spoly_chains spoly_chains;
typedef struct spoly_solution_set spoly_solution_set;

/* Triangles (Sec. 3.1, D1): FP64 SoA of shape [18][n_tris], rows
 * p0x p0y p0z p1x p1y p1z p2x p2y p2z n0x n0y n0z n1x n1y n1z n2x n2y n2z,
 * row-major, n_tris contiguous doubles per row.  Normals need not be unit
 * length; they are interpolated unnormalised (Eq. eq_ni). */
typedef struct {
  const double* tri;
  int64_t n_tris;
  int32_t on_device; /* 1: device pointer, 0: host pointer (copied in) */
  int32_t reserved;
} spoly_mesh;

/* Endpoint queries (Sec. 3.1, D2): one row per query q.
 *   x_first[q][3] = x0, x_last[q][3] = x_{k+1} (FP64)
 *   eta[q][3]     = eta_0 .. eta_k, IOR of the outgoing side of each vertex
 *                   (Sec. 3.1); reflection ignores it
 *   types[q][2]   = SPOLY_R / SPOLY_T per bounce
 *   k[q]          = bounce count: 1, or 2 for chains with two triangles:
 *                   two refractions (types T T; eta_0 .. eta_2 used) or
 *                   two reflections (types R R) */
typedef struct {
  const double* x_first;
  const double* x_last;
  const double* eta;
  const int32_t* types;
  const int32_t* k;
  int64_t n_queries;
  int32_t on_device;
  int32_t reserved;
} spoly_queries;

/* Candidate construction (stands in for the tuple pruning of Sec. 3.1 and Sec. 5). */
#define SPOLY_CHAINS_ALL 0      /* every (query, triangle) pair */
#define SPOLY_CHAINS_CONE 1     /* pairs passing a conservative direction-box test */
#define SPOLY_CHAINS_EXPLICIT 2 /* caller's list */
#define SPOLY_CHAINS_FOOTPRINT 3 /* pixel footprints of a pinhole camera (query q = pixel q) */
#define SPOLY_CHAINS_EXPLICIT_CONE 4 /* caller's list, each chain kept only if it passes the CONE test */
#define SPOLY_CHAINS_FOOTPRINT_UNIQUE 5 /* the distinct triangles of all pixel footprints, one chain each */

typedef struct {
  int32_t mode;
  /* CONE with second_end > 0: 2-bounce chains (all queries k = 2, all of
   * types T T or all of types R R, sharing x0 and the IORs) whose second
   * triangle lies in [second_begin, second_end); the first lies in
   * [tri_begin, tri_end).  A chain survives when its segment direction can
   * lie in the first triangle's refracted (reflected) direction box from
   * x0, in the direction box from the first triangle's bounding box to the
   * second's, and in the negated refracted (reflected) direction box of the
   * second triangle lit from x_last. */
  int32_t second_begin;
  int32_t tri_begin; /* triangle range [tri_begin, tri_end); tri_end <= 0: all */
  int32_t tri_end;
  double margin;     /* CONE: slack added to every unit-direction box (>= 0) */
  const int32_t* explicit_chains; /* EXPLICIT: [n][3] (query, tri0, tri1) */
  int64_t n_explicit;
  int32_t explicit_on_device;
  int32_t second_end;
  /* FOOTPRINT: host array of 16 doubles: camera origin xyz, forward xyz,
   * right xyz, up xyz (unit, orthogonal), tan(vertical fov / 2), aspect
   * (width / height), width, height.  Pixel (ix, iy) = query iy * width + ix
   * covers screen x in [-1 + 2 ix / w, -1 + 2 (ix + 1) / w] and screen y in
   * [1 - 2 (iy + 1) / h, 1 - 2 iy / h]; its ray through screen (sx, sy) is
   * forward + sx tan aspect right + sy tan up. */
  const double* camera;
  double cell; /* FOOTPRINT: grid cell size; <= 0 picks one cell per ~2 triangles */
} spoly_chain_opts;

/* Solve options. */
#define SPOLY_PLAIN_FP64 0 /* every step in FP64 */
#define SPOLY_MIXED 1      /* FP64 construction of a, b and the Bezout entries;
                              FP32 Laplace + isolation; FP64 polish and checks */
#define SPOLY_SOLVE_ASYNC 1  /* do not synchronise or read counters back */
#define SPOLY_SOLVE_TIMING 2 /* record CUDA events around the solve's phases */
#define SPOLY_SOLVE_PERSISTENT 4 /* 1-bounce isolation as one persistent grid whose warps take chunks of
                                    chains from a global ticket counter (launch shape: spoly_autotune's
                                    choice, else 128 threads, 4 blocks per SM, 64 chains per ticket) */
#define SPOLY_SOLVE_PIXEL_ASSIGN 16 /* with a camera: a path's query becomes the pixel its first vertex
                                       projects into (paths outside the image are dropped) instead of
                                       being kept only when that pixel equals its query */
#define SPOLY_SOLVE_GRAPH 8  /* lists without 2-bounce chains: the solve's launches are captured once
                                into a CUDA graph and replayed while the chain list, buffers and
                                options stay the same (needs a non-default stream); a replay whose
                                queues or path buffer overflow falls back to the staged solve */

typedef struct {
  int32_t precision;       /* SPOLY_PLAIN_FP64 or SPOLY_MIXED */
  int32_t flags;           /* SPOLY_SOLVE_* flags */
  int64_t path_capacity;   /* initial path buffer size (0: automatic) */
  /* Optional pixel filter (host array of 16 doubles, camera layout of
   * spoly_chain_opts): a path of query q is kept only if its first vertex
   * projects into pixel q, so each path of a footprint workload is counted
   * once.  NULL: no filter. */
  const double* camera;
  /* 2-bounce chains: the rational pieces replacing sqrt(beta) in the
   * refraction mapping (Sec. 3.4), host array of 25 doubles: breaks[7]
   * (0 = b0 < ... < b6 = 1), then (c0, c1, d1) of (c0 + c1 x) / (1 + d1 x)
   * for each of the six pieces.  NULL: the library's default fit (maximum
   * error 9.4e-4 on [0, 1]). */
  const double* sqrt_table;
  int32_t n_intervals; /* 2-bounce: uniform v1 intervals on [0, 1] (0: 4096; at most 8192) */
  int32_t reserved3;
} spoly_solve_opts;

/* One admissible path (104 bytes).  For k = 1, tri[1] = -1 and the second
 * vertex entries are zero. */
typedef struct {
  int32_t query;
  int32_t tri[2];
  int32_t chain;   /* index of the producing candidate in the solved chain list */
  double uv[2][2]; /* (u_i, v_i) of each specular vertex */
  double x[2][3];  /* world position of each specular vertex */
  float residual;  /* max_i |h_i x n_i| / (|h_i| |n_i|) */
  uint32_t flags;  /* SPOLY_FLAG_* */
} spoly_path;

/* Counters of one solve. */
typedef struct {
  int64_t candidates;   /* chains solved */
  int64_t degenerate;   /* r(v) vanished identically or no u-degree */
  int64_t v_roots;      /* roots of r(v) isolated on [-1e-6, 1 + 1e-6] */
  int64_t queued;       /* brackets sent to the FP64 polish */
  int64_t prefiltered;  /* brackets whose u lies far outside the triangle */
  int64_t polish_lost;  /* brackets with no FP64 sign change */
  int64_t u_roots;      /* (u, v) pairs checked in path space */
  int64_t admissible;   /* paths returned */
  int64_t flagged;      /* returned paths with SPOLY_FLAG_ILL_COND */
  int64_t fallback;     /* chains re-isolated in FP64: FP32 signs not certified,
                           a Bezout size without an unrolled kernel, a
                           flat-shaded triangle, or (2-bounce) FP32 signs that
                           change sign too often */
  int64_t unsolved;     /* 2-bounce systems whose Bezout size exceeds 31 (not solved) */
  int64_t k2_systems;   /* 2-bounce (chain, sqrt piece) systems */
  int64_t k2_evals;     /* 2-bounce Bezout determinant evaluations */
  int64_t k2_eval_n3;   /* sum of n^3 over those evaluations (work of the sign phase) */
  int64_t k2_fp64_samples; /* samples evaluated again in FP64 (re-sampled 2-bounce systems) */
  int64_t k2_evals32;   /* 2-bounce evaluations of the FP32 sign pass (mixed mode) */
  int64_t k2_eval32_n3; /* sum of n^3 over them */
} spoly_counters;

/* Creates a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Errors: EINVAL (out NULL), ECUDA (bad device). */
spoly_status spoly_ctx_create(int device, void* cuda_stream, spoly_ctx** out);

/* Synchronises the stream and frees the context and its scratch.  Handles
 * created from it must be freed before. */
spoly_status spoly_ctx_destroy(spoly_ctx* ctx);

/* Message of the last failed call on this context ("" if none). */
const char* spoly_last_error(const spoly_ctx* ctx);

/* Copies host-resident inputs (on_device = 0; pinned host memory makes the
 * copies asynchronous DMA) into the context's staging buffers on its stream,
 * checks them on the device (non-finite values; k and types on the host),
 * and writes device views of them to *mesh_out and *q_out for the calls that
 * follow.  Device-resident inputs pass through unchanged.  The views stay
 * valid until the next call that stages host inputs on this context, or its
 * destruction.  One upload per step copies each input once, where passing
 * host inputs to every call would copy them into the same buffers again.
 * Synchronises once (to read the check).  Errors: EINVAL (bad shape,
 * non-finite value: the message names the row and triangle or query),
 * ENOMEM, ECUDA. */
spoly_status spoly_upload(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q, spoly_mesh* mesh_out,
                          spoly_queries* q_out);

/* Builds the candidate chain list (query, tri0, tri1) on the device.
 * ALL enumerates every (query, triangle) pair with the query index fastest
 * (consecutive chains share a triangle); CONE keeps the pairs whose conservative box of outgoing unit
 * directions over the triangle (reflected or refracted per the query,
 * interval arithmetic over the triangle's bounding box and normal range)
 * overlaps the box of unit directions from the triangle toward x_{k+1};
 * FOOTPRINT lists every (pixel, triangle) pair whose boxes overlap, ordered
 * by pixel (query q = pixel q); FOOTPRINT_UNIQUE builds the same pairs but
 * keeps only their distinct triangles, one chain (0, t, -1) each, ordered by
 * triangle within chunks of 256: every pixel of a pinhole camera shares its
 * endpoints (the camera origin and one light), so a triangle's solutions
 * do not depend on the pixel, and a solve with SPOLY_SOLVE_PIXEL_ASSIGN
 * hands each path to the pixel its first vertex projects into (that pixel's
 * footprint holds the triangle, so every (pixel, triangle) pair's paths are
 * produced once); it requires every query to equal query 0 (EINVAL
 * otherwise), and spoly_chains_footprint_pairs returns the number of pairs;
 * EXPLICIT copies the caller's list after a bounds check; EXPLICIT_CONE
 * keeps the chains of the caller's list (any mix of queries, bounce counts
 * and triangles) that pass the CONE test of their own bounce count, per
 * query x0, IORs and types (1 bounce: as CONE; 2 bounces of two refractions
 * or two reflections: the three tests of the 2-bounce CONE; mixed 2-bounce
 * types are kept),
 * in no particular order (its boxes use FP32 intervals with directed
 * rounding, so they enclose the FP64 boxes of CONE up to rounding).
 * *inout: NULL to
 * allocate a new handle, or a handle to reuse.  The call synchronises once
 * to read the chain count.  EXPLICIT lists may hold 2-bounce chains
 * (tri1 >= 0).  Errors: EINVAL, ENOMEM, ECUDA, EUNSUPPORTED (CONE with
 * k != 1). */
spoly_status spoly_build_chains(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q,
                                const spoly_chain_opts* opts, spoly_chains** inout);

/* Number of chains in a chain list. */
spoly_status spoly_chains_count(const spoly_chains* chains, int64_t* n);

/* Number of (pixel, triangle) candidate pairs of a list built in a
 * FOOTPRINT mode (0 for other modes). */
spoly_status spoly_chains_footprint_pairs(const spoly_chains* chains, int64_t* n);

/* Copies the chain list [n][3] int32 into dst (host or device).  Errors:
 * ECAPACITY (capacity < count; *n_total = count). */
spoly_status spoly_chains_copy(spoly_ctx* ctx, const spoly_chains* chains, int32_t* dst, int64_t capacity,
                               int64_t* n_total, int32_t dst_is_device);

/* Frees a chain list. */
spoly_status spoly_chains_free(spoly_chains* chains);

/* Solves every chain (Sec. 4.3 pipeline) and keeps the admissible paths in
 * a library-owned solution set.  mesh and q must be the ones the chains were
 * built from.  *inout: NULL for a new set or a set to reuse.  Unless
 * SPOLY_SOLVE_ASYNC is set, the call synchronises, grows the path buffer and
 * re-runs the path phase if it overflowed, and returns with counters valid.
 * Chains with a second triangle (tri1 >= 0, explicit lists) are solved as
 * 2-bounce chains x0 -> tri0 -> tri1 -> x_last of two refractions (TT:
 * the rational sqrt pieces of Sec. 3.4) or two reflections (RR: the exact
 * reflected direction of Eq. eq_431_di and the system of Eq. eq_rr1), by
 * the same solver (Sec. 3.4-3.5,
 * Sec. 4.2 bisection: the Bezout determinant's sign at n_intervals + 1
 * uniform v1, 10 FP32 bisection steps per sign change, FP64 bisection to
 * 1e-10, u1 from a(u1, v1) = 0, u2 from the rational mapping, then
 * path-space Newton on h x n = 0 at both vertices); their paths carry
 * SPOLY_FLAG_NEWTON.  A list with such chains is always solved
 * synchronously, in batches.  Errors: EINVAL, ENOMEM, ECUDA, EUNSUPPORTED
 * (a 2-bounce chain whose query is not of types T T or R R; on device
 * queries such chains are not checked and return no paths). */
spoly_status spoly_solve(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q,
                         const spoly_chains* chains, const spoly_solve_opts* opts,
                         spoly_solution_set** inout);

/* Copies up to `capacity` paths to dst (host or device) in the device's
 * completion order; *n_total receives the path count.  Errors: ECAPACITY
 * when capacity < *n_total (the first `capacity` paths are still copied). */
spoly_status spoly_paths(spoly_ctx* ctx, const spoly_solution_set* set, spoly_path* dst, int64_t capacity,
                         int64_t* n_total, int32_t dst_is_device);

/* Counters of the last solve into `set` (synchronises the context stream). */
spoly_status spoly_stats(spoly_ctx* ctx, const spoly_solution_set* set, spoly_counters* out);

/* Visibility test of the path phase (Sec. 4.3: a path is rejected when the
 * segment from a vertex to the next is blocked): every path of `set` whose
 * segments x0 -> x1 (-> x2) -> x_last meet a triangle of `mesh` strictly
 * inside (ray parameter in (1e-9, 1 - 1e-9); each segment's own end
 * triangles excluded) gets SPOLY_FLAG_OCCLUDED, in place; *n_visible (host)
 * receives the number of the others.  mesh and q must be the solve's (with
 * SPOLY_SOLVE_PIXEL_ASSIGN every pixel shares the endpoints, which the test
 * takes from the path's query).  Builds a uniform xy grid over the mesh
 * (library scratch, FP64 triangle tests).  Synchronises.  Errors: EINVAL,
 * ENOMEM, ECUDA. */
spoly_status spoly_visibility(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q, spoly_solution_set* set,
                              int64_t* n_visible);

/* Contribution of every path of `set` (Sec. 4.3; the paper cites the
 * generalised geometric term of specular chains without printing it, so the
 * library states its own reading): the irradiance at the camera point
 * x_first of a point light of intensity `intensity` at x_last carried
 * through the chain, f = I / (|x1 - x_first|^2 |det J|), where J is the
 * 2 x 2 derivative (central differences in FP64) of where a ray leaving the
 * light toward the last vertex, traced back through the planes of the
 * chain's triangles with their interpolated normals, passes the camera, per
 * unit solid angle of emission.  Occluded paths (SPOLY_FLAG_OCCLUDED)
 * contribute 0.  per_path (device FP64 [number of paths], may be NULL)
 * receives f in the set's path order; image (device FP64 [image_size], may
 * be NULL) is accumulated: image[query] += f (a pixel, with
 * SPOLY_SOLVE_PIXEL_ASSIGN).  Synchronises.  Errors: EINVAL (intensity < 0,
 * image_size <= 0 with an image), ECUDA. */
spoly_status spoly_contributions(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q,
                                 const spoly_solution_set* set, double intensity, double* per_path, double* image,
                                 int64_t image_size);

/* Device time of the last solve's phases, measured with CUDA events on the
 * context stream when the solve set SPOLY_SOLVE_TIMING: ms[0] = isolation
 * (coefficient, elimination and univariate phases, both isolation kernels),
 * ms[1] = FP64 polish and path phase, ms[2] (n >= 3) = the whole 2-bounce
 * pipeline, ms[3] (n >= 4) = its sign passes in the solve's precision (the
 * FP32 pass in mixed mode), summed over batches.  n >= 2.  Synchronises on
 * the last event.  Errors: EINVAL if the solve was not timed. */
spoly_status spoly_phase_ms(spoly_ctx* ctx, const spoly_solution_set* set, float* ms, int32_t n);

/* Peak-throughput microbenchmark of a scalar pipe on the context's device:
 * SPOLY_PEAK_FP32_FMA or SPOLY_PEAK_FP64_FMA.  *tflops receives the best
 * TFLOP/s (2 flop per FMA) over timed launches of independent FMA chains on
 * every SM.  Allocates and frees a small device buffer.  The roofline
 * fractions the project reports use these numbers as denominators. */
#define SPOLY_PEAK_FP32_FMA 0
#define SPOLY_PEAK_FP64_FMA 1
spoly_status spoly_measure_peak(spoly_ctx* ctx, int32_t kind, double* tflops);

/* One measured launch shape of the persistent 1-bounce isolation kernel. */
typedef struct {
  int32_t block;         /* threads per block (64 or 128) */
  int32_t blocks_per_sm; /* requested resident blocks per SM (capped by occupancy) */
  int32_t chunk;         /* chains per work-queue ticket */
  float ms;              /* best of three timed launches on the given chains */
} spoly_tune_entry;

/* Autotuner of the persistent isolation kernel (north star (2)): times
 * every shape of block in {64, 128} x blocks per SM in {1, 2, 4, 8} x chunk
 * in {32, 64, 128, 256} on the 1-bounce chains of `chains` (precision
 * SPOLY_MIXED or SPOLY_PLAIN_FP64), keeps the fastest in the context for
 * later SPOLY_SOLVE_PERSISTENT solves, and writes it to *best (may be NULL)
 * and up to `cap` entries to table (host, may be NULL; *n_table receives
 * the number of shapes).  Allocates and frees its scratch.  Errors: EINVAL
 * (no 1-bounce chains), ENOMEM, ECUDA. */
spoly_status spoly_autotune(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q,
                            const spoly_chains* chains, int32_t precision, spoly_tune_entry* table, int32_t cap,
                            int32_t* n_table, spoly_tune_entry* best);

/* Frees a solution set. */
spoly_status spoly_solution_free(spoly_solution_set* set);

/* The 1-bounce solve for callers that cannot allocate device memory.  (The
 * paper has no counterpart: this is a deployment variant of spoly_solve.)
 *
 * Some callers may not allocate at all: code running where the allocator is
 * off limits (a host callback, a real-time loop that must not block on an
 * allocation), a plug-in whose host application owns all device memory, or
 * a process with a fixed memory pool.  This entry point allocates nothing:
 * the solve's scratch (counters and root-bracket queues) lives in one static
 * device array of about 2.2 MiB inside the library, which every GPU that
 * loads the library keeps until the process exits.
 *
 * Inputs are device pointers with the layouts of spoly_mesh, spoly_queries
 * and the chain list (int32 [n_chains][3]); `paths` is a device buffer of
 * `path_capacity` records that receives the admissible paths; *n_paths (host)
 * receives their count.  precision is SPOLY_PLAIN_FP64 or SPOLY_MIXED.  Only
 * 1-bounce chains are solved here: every chain must have tri1 < 0, a query
 * in [0, n_queries) with k = 1 and type SPOLY_R or SPOLY_T, and a triangle in
 * [0, n_tris); a device-side pass checks this before the solve reads through
 * any index, and the first failing chain is reported by SPOLY_EINVAL.
 *
 * The call is synchronous: it selects `device`, enqueues on `cuda_stream`,
 * waits on that stream twice (after the validation pass and at the end),
 * restores the caller's current device and returns.  `msg` (host buffer of
 * msg_len bytes, may be NULL) receives a message on failure.
 *
 * Limits and sharing: at most 4096 chains per call (more is rejected with
 * SPOLY_EINVAL and a message).  All calls share the static array; each call
 * clears its counters and overwrites its queues, so calls whose GPU work
 * overlaps (other streams, unordered host threads) race and corrupt each
 * other.  The first call on a device performs a one-time set-up (it looks up
 * the array's device address); make that first call before any stream
 * capture begins.
 * Errors: EINVAL (null pointer, negative size, too many chains, bad
 * precision or device, or a chain failing the checks above: the message
 * names its index and the reason), ECUDA (a CUDA call failed), ECAPACITY
 * (more paths than path_capacity: *n_paths holds the required count and the
 * first path_capacity paths, in completion order, were written). */
spoly_status spoly_solve_noalloc(int device, void* cuda_stream, const double* tri, int64_t n_tris,
                                 const double* x_first, const double* x_last, const double* eta,
                                 const int32_t* types, const int32_t* k, int64_t n_queries, const int32_t* chains,
                                 int64_t n_chains, int32_t precision, spoly_path* paths, int64_t path_capacity,
                                 int64_t* n_paths, char* msg, int32_t msg_len);

/* ------------------------------------------------------------------------
 * Learned candidate gate.  (The paper has no counterpart: the gate predicts,
 * from a candidate's geometry, whether its solve returns any admissible path,
 * so that candidates predicted empty are not solved.)
 *
 * Features: 24 FP32 values per 1-bounce chain, computed from the triangle's
 * vertices and normals relative to the endpoints: the tangential mismatch
 * between the unit normal and the generalised half vector (the constraint
 * h x n = 0 of Eq. eq_ch) at the three vertices, in a frame perpendicular to
 * the half vector at the centroid; the barycentric coordinates of the zero
 * of its affine interpolant; shape, distance and type terms.
 *
 * Network: 24 (padded to 32) -> 64 -> 64 -> 64 -> 1 with ReLU hidden layers
 * and a sigmoid output.  The three weight matrices and every matrix-product
 * operand are BF16 (round to nearest even) with FP32 accumulation on the
 * tensor cores; biases, the output weights and bias are FP32.  Parameters
 * form one FP32 vector of SPOLY_MLP_PARAMS values: W1[32][64] (rows 24..31
 * unused and kept zero), b1[64], W2[64][64], b2[64], W3[64][64], b3[64],
 * w4[64], b4, each row-major W[in][out].
 * ---------------------------------------------------------------------- */
#define SPOLY_MLP_FEATURES 24
#define SPOLY_MLP_PARAMS 10497

typedef struct spoly_mlp spoly_mlp;

typedef struct {
  int64_t steps;        /* Adam steps (> 0) */
  int32_t batch;        /* rows per step, 32 .. 2^20 */
  float lr;             /* initial learning rate (> 0) */
  float lr_final;       /* learning rate of the last step, geometric decay; 0: constant */
  float pos_weight;     /* loss weight of a positive row (> 0) */
  float pos_fraction;   /* share of positives in every batch, in (0, 1) */
  int32_t reserved;
  uint64_t seed;        /* batch sampler seed */
} spoly_mlp_train_opts;

/* A network with He-uniform weights from `seed` (splitmix64) and zero
 * biases, resident on the context's device.  Free with spoly_mlp_free. */
spoly_status spoly_mlp_create(spoly_ctx* ctx, uint64_t seed, spoly_mlp** out);
spoly_status spoly_mlp_free(spoly_mlp* mlp);

/* Limit, in SM clock cycles, of each wait of the gate's inference kernel
 * (spoly_gate, spoly_mlp_forward, spoly_mlp_calibrate) for a layer's
 * tensor-core products to complete; 0 restores the default (2^31 cycles,
 * about a second).  A wait that gives up makes the call return
 * SPOLY_ETIMEOUT with incomplete outputs; the kernel then waits for the
 * product still in flight with the default limit before it frees its tensor
 * memory, so the context stays usable.  Errors: EINVAL (mlp NULL or
 * cycles < 0). */
spoly_status spoly_mlp_set_wait_limit(spoly_mlp* mlp, int64_t cycles);

/* Copy the FP32 parameter vector (SPOLY_MLP_PARAMS values, host memory) out
 * of or into the network.  set rejects non-finite values (EINVAL). */
spoly_status spoly_mlp_get_params(spoly_ctx* ctx, const spoly_mlp* mlp, float* dst);
spoly_status spoly_mlp_set_params(spoly_ctx* ctx, spoly_mlp* mlp, const float* src);

/* Checkpoint file: magic "SPOLYMLP", int32 version 1, int32 parameter count,
 * int64 Adam step, then the parameters and both Adam moment vectors (FP32,
 * little-endian).  load returns a new network; EINVAL on a bad file. */
spoly_status spoly_mlp_save(spoly_ctx* ctx, const spoly_mlp* mlp, const char* path);
spoly_status spoly_mlp_load(spoly_ctx* ctx, const char* path, spoly_mlp** out);

/* Features of every chain of `chains` into dst (device, FP32 [n][24],
 * 16-byte aligned).  Synchronises. */
spoly_status spoly_mlp_features(spoly_ctx* ctx, const spoly_mesh* mesh, const spoly_queries* q,
                                const spoly_chains* chains, float* dst);

/* Training labels from a finished (synchronous) solve of a chain list:
 * dst[c] = 1 if chain c produced a returned path, else 0 (device uint8
 * [n_chains]).  Solve without a pixel filter to label each chain's own
 * solution set.  Synchronises. */
spoly_status spoly_chain_labels(spoly_ctx* ctx, const spoly_solution_set* set, int64_t n_chains, uint8_t* dst);

/* Logits of n feature rows (device FP32 [n][24] -> device FP32 [n]) by the
 * gate's inference kernel.  Synchronises. */
spoly_status spoly_mlp_forward(spoly_ctx* ctx, const spoly_mlp* mlp, const float* feat, int64_t n, float* logits);

/* Gradient of the mean weighted binary cross-entropy of n rows (device
 * features and uint8 labels; n <= 2^24) with respect to the parameter
 * vector, into grad (host, SPOLY_MLP_PARAMS FP32), by the training kernels;
 * *loss (host, may be NULL) receives the loss.  The parameters are unchanged. */
spoly_status spoly_mlp_grad(spoly_ctx* ctx, spoly_mlp* mlp, const float* feat, const uint8_t* labels, int64_t n,
                            float pos_weight, float* grad, float* loss);

/* Trains on n labelled rows (device features and uint8 labels, both classes
 * present) with Adam on stratified batches sampled with replacement.
 * *final_loss (host, may be NULL) receives the mean batch loss of the last
 * min(steps, 64) steps.  Synchronises. */
spoly_status spoly_mlp_train(spoly_ctx* ctx, spoly_mlp* mlp, const float* feat, const uint8_t* labels, int64_t n,
                             const spoly_mlp_train_opts* opts, float* final_loss);

/* The largest logit threshold that keeps at least target_recall of the
 * positive rows of a labelled set (device features and labels), into
 * *tau_logit; *pass_fraction (may be NULL) receives the share of all rows at
 * or above it. */
spoly_status spoly_mlp_calibrate(spoly_ctx* ctx, spoly_mlp* mlp, const float* feat, const uint8_t* labels,
                                 int64_t n, double target_recall, float* tau_logit, double* pass_fraction);

/* Gates a chain list: features, network and compaction in one kernel.  A
 * 1-bounce chain passes if its logit is >= tau_logit or if the zero of its
 * tangential mismatch (the features' barycentric coordinates) lies inside
 * the triangle (smallest coordinate >= -0.02): the network only rejects
 * chains whose zero lies outside.  Every 2-bounce chain (tri1 >= 0: outside
 * the network's domain) passes.  The survivors are written to *inout
 * (created when NULL, else reused and grown; it must not be `in`).  Their
 * order is not preserved.  Synchronises (reads the count back). */
spoly_status spoly_gate(spoly_ctx* ctx, const spoly_mlp* mlp, const spoly_mesh* mesh, const spoly_queries* q,
                        const spoly_chains* in, float tau_logit, spoly_chains** inout);

/* The library's default rational pieces of sqrt on [0, 1] (Sec. 3.4: six
 * pieces (c0 + c1 x) / (1 + d1 x); the paper's own coefficients are in its
 * missing supplement, so the library fits its own), in the 25-double layout
 * of spoly_solve_opts::sqrt_table, into dst (host, n >= 25).  A comparison
 * with another implementation of the method passes this table to both sides:
 * the pieces are a parameter of the approximation, like the IORs.  Errors:
 * EINVAL (dst NULL or n < 25). */
spoly_status spoly_default_sqrt_table(double* dst, int32_t n);

/* Library version string. */
const char* spoly_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPOLY_H_ */
