"""Per-workload error of the CUDA path against the FP64 oracles (needs a GPU).

For each workload, at its stated size and in the launch configuration the
benchmark times, the GPU's paths are paired with the oracle's on a sample of
candidates the oracle can solve (|delta(u, v)| <= 1e-5 within a candidate),
and the script prints one table row: compared candidates, paths on each
side, unmatched paths (flagged / unflagged), max and p99 |delta(u, v)|.

    python tests/parity_table.py [--precision mixed|plain]

Rows: reflection (all 524,288 pairs), refraction caustics (every triangle
for 48 seeded receivers of the full cone-culled solve), the 2-bounce slab
(64x64 receivers, cone cull, the library's sqrt pieces; every culled chain
with a GPU path plus seeded culled chains), glints (distinct-triangle
footprint with pixel assignment, no gate, against the oracle's
pixel-filtered solve of the footprints of seeded 16x16-pixel blocks), and
the batched mixed workload at its full 4096 queries (every chain of seeded
1-bounce queries, a sample of the culled 2-bounce chains; no gate).
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _pair(gpu_rows, ref_rows, tol=1e-5):
    """gpu_rows, ref_rows: lists of (key, uv vector, flags).  Returns counts
    and the matched distances."""
    from collections import defaultdict
    G, R = defaultdict(list), defaultdict(list)
    for k, x, f in gpu_rows:
        G[k].append((np.asarray(x, float), int(f)))
    for k, x, f in ref_rows:
        R[k].append((np.asarray(x, float), int(f)))
    from tests.parity import ALLOWED
    d_all, un_f, un_u = [], 0, 0
    for key in set(G) | set(R):
        a, b = G.get(key, []), R.get(key, [])
        pairs = sorted((float(np.max(np.abs(x - y))), i, j) for i, (x, _) in enumerate(a) for j, (y, _) in enumerate(b))
        ua, ub = set(range(len(a))), set(range(len(b)))
        for d, i, j in pairs:
            if d > tol:
                break
            if i in ua and j in ub:
                ua.discard(i)
                ub.discard(j)
                d_all.append(d)
        for i in ua:
            un_f, un_u = (un_f + 1, un_u) if a[i][1] & ALLOWED else (un_f, un_u + 1)
        for j in ub:
            un_f, un_u = (un_f + 1, un_u) if b[j][1] & ALLOWED else (un_f, un_u + 1)
    d = np.array(d_all) if d_all else np.zeros(1)
    return len(d_all), un_f, un_u, float(d.max()), float(np.quantile(d, 0.99))


def _block_footprint(s, cam, origins, side=16):
    """(pixel, triangle, -1) candidates of the 16x16-pixel blocks at the given
    origins: the triangles whose xy box meets the pixel's footprint box (its
    four corner rays between the mesh's z bounds)."""
    from tests.parity import footprint_boxes
    T = s.tri
    xs, ys = T[[0, 3, 6]], T[[1, 4, 7]]
    txl, txh, tyl, tyh = xs.min(0), xs.max(0), ys.min(0), ys.max(0)
    w = int(cam[14])
    rows = []
    for x0, y0 in origins:
        qs = np.array([iy * w + ix for iy in range(y0, y0 + side) for ix in range(x0, x0 + side)])
        for q, b in zip(qs, footprint_boxes(s, cam, qs)):
            if b is None:
                continue
            bx0, bx1, by0, by1 = b
            t = np.where(~((txh < bx0) | (txl > bx1) | (tyh < by0) | (tyl > by1)))[0]
            rows.append(np.stack([np.full(t.size, q), t, -np.ones(t.size, np.int64)], -1))
    return np.ascontiguousarray(np.unique(np.concatenate(rows), axis=0).astype(np.int32))


def _rows1(paths, gpu):
    if gpu:
        return [((int(p["query"]), int(p["tri"][0])), p["uv"][:2], p["flags"]) for p in paths]
    return [((int(p["query"]), int(p["tri0"])), p["uv"][:2], p["flags"]) for p in paths]


def _rows2(paths, gpu):
    if gpu:
        return [((int(p["query"]), int(p["tri"][0]), int(p["tri"][1])), p["uv"].ravel(), p["flags"]) for p in paths]
    return [((int(p["query"]), int(p["tri0"]), int(p["tri1"])), p["uv"], p["flags"]) for p in paths]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", choices=["mixed", "plain"], default="mixed")
    args = ap.parse_args()
    from tests import oracle_pool
    oracle_pool.pool()  # worker processes before the first CUDA call
    import torch

    import __graft_entry__
    import oracle
    from paper_2405_13409_gb300 import binding, scenes
    __graft_entry__.build()
    prec = binding.MIXED if args.precision == "mixed" else binding.PLAIN_FP64
    ctx = binding.Context(0, torch.cuda.current_stream().cuda_stream)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = []

    def solve(s, mode, chains=None, camera=None, flags=0, table=None, **kw):
        d = [dev(a) for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
        mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
        ch = ctx.spoly_build_chains(mesh, q, mode, explicit=None if chains is None else dev(chains), camera=camera,
                                    margin=1e-3, **kw)
        sol = ctx.spoly_solve(mesh, q, ch, precision=prec, camera=camera, flags=flags, sqrt_table=table)
        p = ctx.spoly_paths(sol)
        kept = ctx.spoly_chains_copy(ch)
        ctx.spoly_solution_free(sol)
        ctx.spoly_chains_free(ch)
        return p, kept

    # reflection: every pair
    s = scenes.reflect_scene()
    every = scenes.all_pairs(s.n_queries, s.n_tris)
    p, _ = solve(s, binding.CHAINS_ALL)
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, every)
    out.append(("reflection 16x16 cells x 32x32 receivers (all pairs)", every.shape[0], p.size, ref.size,
                *_pair(_rows1(p, True), _rows1(ref, False))))
    # refraction: the full cone-culled solve, 48 receivers against every triangle
    s = scenes.refract_scene()
    p, _ = solve(s, binding.CHAINS_CONE)
    rng = np.random.default_rng(5)
    qs = np.sort(rng.choice(s.n_queries, 48, replace=False)).astype(np.int32)
    every = np.stack([np.repeat(qs, s.n_tris), np.tile(np.arange(s.n_tris, dtype=np.int32), qs.size),
                      -np.ones(qs.size * s.n_tris, np.int32)], -1).astype(np.int32)
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, every)
    mine = p[np.isin(p["query"], qs)]
    out.append(("refraction 64x64 cells x 256x256 receivers (48 receivers x all triangles)", every.shape[0],
                mine.size, ref.size, *_pair(_rows1(mine, True), _rows1(ref, False))))
    # slab: 64x64 receivers, cone cull, the library's sqrt pieces
    s = scenes.slab_scene(seed=0, n_cells=16, n_recv=64)
    half = s.n_tris // 2
    table = binding.spoly_default_sqrt_table()
    p, kept = solve(s, binding.CHAINS_CONE, table=table, tri_range=(0, half), second_range=(half, s.n_tris))
    with_p = {(int(a), int(b), int(c)) for a, b, c in zip(p["query"], p["tri"][:, 0], p["tri"][:, 1])}
    rng = np.random.default_rng(7)
    rows = set(with_p) | {tuple(r) for r in kept[rng.choice(kept.shape[0], 300, replace=False)].tolist()}
    sample = np.array(sorted(rows), np.int32)
    ref, _ = oracle_pool.tt_solve(s.tri, s.x_first, s.x_last, s.eta, sample, table[1])
    mine = p[[(int(a), int(b), int(c)) in rows for a, b, c in zip(p["query"], p["tri"][:, 0], p["tri"][:, 1])]]
    out.append(("TT slab 16x16+16x16 cells x 64x64 receivers (culled chains with paths + 300 seeded)",
                sample.shape[0], mine.size, ref.size, *_pair(_rows2(mine, True), _rows2(ref, False))))
    # glints: distinct triangles + pixel assignment; the oracle solves every
    # footprint candidate of 16x16-pixel blocks, 6 around seeded lit pixels
    # of the GPU image and 2 at seeded positions
    s = scenes.glint_scene()
    cam = s.meta["camera"].as_array()
    p, _ = solve(s, binding.CHAINS_FOOTPRINT_UNIQUE, camera=cam, flags=binding.SOLVE_PIXEL_ASSIGN)
    w, h = int(cam[14]), int(cam[15])
    rng = np.random.default_rng(11)
    lit = rng.choice(np.unique(p["query"]), 6, replace=False)
    origins = [(int(min(max(q % w - 8, 0), w - 16)), int(min(max(q // w - 8, 0), h - 16))) for q in lit]
    origins += [(int(rng.integers(0, w - 15)), int(rng.integers(0, h - 15))) for _ in range(2)]
    fp = _block_footprint(s, cam, origins)
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, fp)
    from tests.parity import project_pixels
    ref = ref[project_pixels(cam, ref["x"][:, :3]) == ref["query"]]
    pix = np.unique(fp[:, 0])
    mine = p[np.isin(p["query"], pix)]
    out.append((f"glints 1024x1024 cells, 512x512 px (8 16x16-pixel blocks: 6 around lit pixels, 2 seeded)",
                fp.shape[0], mine.size, ref.size, *_pair(_rows1(mine, True), _rows1(ref, False))))
    # batched mixed workload at its full size (4096 queries); the oracle
    # solves every chain of 24 seeded 1-bounce queries and a sample of the
    # culled 2-bounce chains
    s = scenes.batched_scene(seed=0, n_queries=4096)
    d = [dev(a) for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, s.chains)]
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:6])
    cut = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT_CONE, margin=1e-3, explicit=d[6])
    sol = ctx.spoly_solve(mesh, q, cut, precision=prec, flags=binding.SOLVE_PERSISTENT, sqrt_table=table)
    p = ctx.spoly_paths(sol)
    kept = ctx.spoly_chains_copy(cut)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(cut)
    del d, mesh, q
    one_q = np.where(s.k == 1)[0]
    qs = np.sort(rng.choice(one_q, 24, replace=False))
    ex1 = np.ascontiguousarray(s.chains[np.isin(s.chains[:, 0], qs) & (s.chains[:, 2] < 0)])
    ref1, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, ex1)
    g1 = p[(p["tri"][:, 1] < 0) & np.isin(p["query"], qs)]
    out.append(("batched 4096 queries (no gate): every chain of 24 seeded 1-bounce queries", ex1.shape[0],
                g1.size, ref1.size, *_pair(_rows1(g1, True), _rows1(ref1, False))))
    k2 = kept[kept[:, 2] >= 0]
    g2 = p[p["tri"][:, 1] >= 0]
    with_p = {(int(a), int(b), int(c)) for a, b, c in zip(g2["query"], g2["tri"][:, 0], g2["tri"][:, 1])}
    rows = set(with_p) | {tuple(r) for r in k2[rng.choice(k2.shape[0], min(300, k2.shape[0]), replace=False)].tolist()}
    sample = np.array(sorted(rows), np.int32)
    ref2, _ = oracle_pool.tt_solve(s.tri, s.x_first, s.x_last, s.eta, sample, table[1])
    mine = g2[[(int(a), int(b), int(c)) in rows for a, b, c in zip(g2["query"], g2["tri"][:, 0], g2["tri"][:, 1])]]
    out.append(("batched 4096 queries (no gate): 2-bounce culled chains with a GPU path + 300 seeded",
                sample.shape[0], mine.size, ref2.size, *_pair(_rows2(mine, True), _rows2(ref2, False))))
    ctx.close()
    print(f"| workload ({args.precision}) | candidates compared | GPU paths | oracle paths | matched | "
          f"unmatched flagged | unmatched unflagged | max abs d(u,v) | p99 abs d(u,v) |")
    print("|---|---|---|---|---|---|---|---|---|")
    for name, nc, ng, nr, m, uf, uu, mx, p99 in out:
        print(f"| {name} | {nc:,} | {ng:,} | {nr:,} | {m:,} | {uf} | {uu} | {mx:.1e} | {p99:.1e} |", flush=True)


if __name__ == "__main__":
    main()
