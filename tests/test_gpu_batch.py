"""GPU tests of the batched mixed workload's pieces: the per-chain cone test
of explicit lists (EXPLICIT_CONE) is conservative for both bounce counts,
the learned gate passes 2-bounce chains through, and the whole batch solved
in one call equals the unculled solve."""
import numpy as np
import pytest

from paper_2405_13409_gb300 import binding, scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bctx():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    stream = torch.cuda.Stream()
    c = binding.Context(0, stream.cuda_stream)
    yield c, stream
    c.close()


@pytest.fixture(scope="module")
def batch(bctx):
    """48 queries; every triangle of each 1-bounce query's mesh (so their
    paths are all present) and 512 of the (top, bottom) pairs of each
    2-bounce query (the unculled 2-bounce solve stays short)."""
    ctx, stream = bctx
    s = scenes.batched_scene(seed=3, n_queries=48, c_min=8192, c_max=8192)
    two = s.chains[:, 2] >= 0
    keep = ~two
    for qq in np.unique(s.chains[two, 0]):
        idx = np.where(s.chains[:, 0] == qq)[0]
        keep[idx[:512]] = True
    s.chains = np.ascontiguousarray(s.chains[keep])
    with torch.cuda.stream(stream):
        d = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
             for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, s.chains)]
    stream.synchronize()
    return s, d, ctx.mesh(d[0]), ctx.queries(*d[1:6])


def _keys(p):
    return sorted(zip(p["query"].tolist(), p["tri"][:, 0].tolist(), p["tri"][:, 1].tolist(),
                      np.round(p["uv"].reshape(-1, 4), 8).tolist()))


def test_batched_scene_shape():
    s = scenes.batched_scene(seed=1, n_queries=16, c_min=100, c_max=1000)
    counts = s.meta["counts"]
    assert s.chains.shape[0] == counts.sum()
    q = s.chains[:, 0]
    assert np.all(np.diff(q) >= 0)  # grouped by query
    for i in range(16):
        ch = s.chains[q == i]
        assert ch.shape[0] == counts[i]
        assert np.all((ch[:, 2] >= 0) == (s.k[i] == 2))
        assert np.unique(ch[:, 1:], axis=0).shape[0] == ch.shape[0]  # distinct candidates
    assert s.chains[:, 1:].max() < s.n_tris


@pytest.mark.parametrize("precision", [binding.MIXED, binding.PLAIN_FP64])
def test_explicit_cone_is_conservative(bctx, batch, precision):
    ctx, stream = bctx
    s, d, mesh, q = batch
    full = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=d[6])
    cut = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT_CONE, margin=1e-3, explicit=d[6])
    n_full, n_cut = ctx.spoly_chains_count(full), ctx.spoly_chains_count(cut)
    assert n_full == s.chains.shape[0]
    assert 0 < n_cut < n_full // 10
    kept = ctx.spoly_chains_copy(cut)
    src = {tuple(r) for r in s.chains.tolist()}
    assert all(tuple(r) in src for r in kept.tolist())
    a = ctx.spoly_solve(mesh, q, full, precision=precision)
    b = ctx.spoly_solve(mesh, q, cut, precision=precision, flags=binding.SOLVE_PERSISTENT)
    pa, pb = ctx.spoly_paths(a), ctx.spoly_paths(b)
    ctx.spoly_solution_free(a)
    ctx.spoly_solution_free(b)
    ctx.spoly_chains_free(full)
    ctx.spoly_chains_free(cut)
    assert pa.size > 10
    assert _keys(pa) == _keys(pb)


def _rows(a):
    return sorted(map(tuple, a.tolist()))


def test_explicit_cone_equals_range_cone(bctx):
    """On every (receiver, triangle) pair, or every (receiver, top, bottom)
    tuple of a slab, the per-chain test (FP32 intervals with directed
    rounding) keeps every chain of the range-based cone cull (the same
    predicates on FP64 intervals) and at most a few more."""
    ctx, stream = bctx
    r = scenes.refract_scene(seed=2, n_cells=32, n_recv=12)
    sl = scenes.slab_scene(seed=0, n_cells=16, n_recv=2)
    half = sl.n_tris // 2
    for s, ranges in ((r, None), (sl, ((0, half), (half, sl.n_tris)))):
        with torch.cuda.stream(stream):
            d = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
                 for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
        stream.synchronize()
        mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
        if ranges is None:
            ref = ctx.spoly_build_chains(mesh, q, binding.CHAINS_CONE, margin=1e-3)
            allc = scenes.all_pairs(s.n_queries, s.n_tris)
        else:
            ref = ctx.spoly_build_chains(mesh, q, binding.CHAINS_CONE, margin=1e-3, tri_range=ranges[0],
                                         second_range=ranges[1])
            qq, t1, t2 = np.meshgrid(np.arange(s.n_queries), np.arange(half), np.arange(half, s.n_tris),
                                     indexing="ij")
            allc = np.stack([qq.ravel(), t1.ravel(), t2.ravel()], -1).astype(np.int32)
        exp = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT_CONE, margin=1e-3,
                                     explicit=torch.from_numpy(allc).cuda())
        a, b = ctx.spoly_chains_copy(ref), ctx.spoly_chains_copy(exp)
        ctx.spoly_chains_free(ref)
        ctx.spoly_chains_free(exp)
        assert 0 < a.shape[0] < allc.shape[0] // 20
        ra, rb = set(_rows(a)), set(_rows(b))
        assert ra <= rb
        assert len(rb) <= 1.02 * len(ra) + 4


def test_gate_passes_two_bounce_chains(bctx, batch):
    ctx, stream = bctx
    s, d, mesh, q = batch
    cut = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT_CONE, margin=1e-3, explicit=d[6])
    mlp = ctx.spoly_mlp_create(seed=5)
    # a threshold no logit reaches: only the 2-bounce chains and the 1-bounce
    # chains whose mismatch zero lies inside the triangle pass
    gated = ctx.spoly_gate(mlp, mesh, q, cut, 3e38)
    kept = ctx.spoly_chains_copy(gated)
    all_cut = ctx.spoly_chains_copy(cut)
    f = torch.empty((all_cut.shape[0], 24), dtype=torch.float32, device="cuda")
    ctx.spoly_mlp_features(mesh, q, cut, f)
    inside = f[:, 12].cpu().numpy() >= -0.02
    want = all_cut[(all_cut[:, 2] >= 0) | inside]
    assert int((all_cut[:, 2] >= 0).sum()) > 0
    assert _rows(kept) == _rows(want)
    ctx.spoly_chains_free(gated)
    ctx.spoly_chains_free(cut)
    ctx.spoly_mlp_free(mlp)


def test_batch_pipeline_matches_oracles(bctx):
    """A batch shaped like the batched mixed workload (160 independent
    queries, bounce count uniform in {1, 2}, candidate counts log-uniform in
    1e2..2e4) through the workload's whole pipeline: the per-chain cone
    test, the gate (its threshold below every logit, so every chain it
    keeps is compared), the persistent isolation with the autotuner's launch
    shape, and the 2-bounce pipeline with the library's default sqrt pieces;
    then the same solve captured into one CUDA graph and replayed.
    Every 1-bounce chain of the explicit (unculled) list is solved by the
    C++ oracle; a sample of 2-bounce chains (every culled chain with a GPU
    path, culled chains at random and unculled chains at random) by the
    numpy TT oracle with the same sqrt pieces.  Paths are paired at 1e-5."""
    import oracle
    from tests import oracle_pool
    from .parity import assert_parity
    from .test_gpu_tt import _compare
    ctx, stream = bctx
    s = scenes.batched_scene(seed=11, n_queries=160, c_min=1e2, c_max=2e4)
    # random receivers rarely see a 2-bounce path: eight more 2-bounce queries
    # receive paths planted through the 16x16-cell slab (appended to the
    # mesh), with their chains and neighbouring pairs
    from .test_tt_oracle import planted_slab_cases
    slab = scenes.slab_scene(seed=0, n_cells=16, n_recv=4)
    half, off, q0 = slab.n_tris // 2, s.n_tris, s.n_queries
    cases = planted_slab_cases(17, 8)
    rows = []
    for i, c in enumerate(cases):
        for d2 in (-2, 0, 2):
            if half <= c[3] + d2 < slab.n_tris:
                rows.append([q0 + i, off + c[2], off + c[3] + d2])
    s.tri = np.ascontiguousarray(np.concatenate([s.tri, slab.tri], 1))
    s.x_first = np.concatenate([s.x_first, np.array([c[0] for c in cases])])
    s.x_last = np.concatenate([s.x_last, np.array([c[1] for c in cases])])
    s.eta = np.concatenate([s.eta, np.tile([1.0, 1.5, 1.0], (len(cases), 1))])
    s.types = np.concatenate([s.types, np.full((len(cases), 2), binding.SPOLY_T, np.int32)])
    s.k = np.concatenate([s.k, np.full(len(cases), 2, np.int32)])
    s.chains = np.ascontiguousarray(np.concatenate([s.chains, np.array(rows, np.int32)]))
    with torch.cuda.stream(stream):
        d = [torch.from_numpy(np.ascontiguousarray(a)).cuda()
             for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, s.chains)]
    stream.synchronize()
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:6])
    table = binding.spoly_default_sqrt_table()
    cut = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT_CONE, margin=1e-3, explicit=d[6])
    mlp = ctx.spoly_mlp_create(seed=9)
    gated = ctx.spoly_gate(mlp, mesh, q, cut, -3e38)
    kept = ctx.spoly_chains_copy(gated)
    assert kept.shape[0] == ctx.spoly_chains_count(cut)
    one = torch.from_numpy(np.ascontiguousarray(kept[kept[:, 2] < 0])).cuda()
    ch1 = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=one)
    ctx.spoly_autotune(mesh, q, ch1, binding.MIXED)
    ctx.spoly_chains_free(ch1)
    sol = ctx.spoly_solve(mesh, q, gated, precision=binding.MIXED, flags=binding.SOLVE_PERSISTENT,
                          sqrt_table=table)
    paths = ctx.spoly_paths(sol)
    stats = ctx.spoly_stats(sol)
    ctx.spoly_solution_free(sol)
    # the same list captured once into a CUDA graph (1- and 2-bounce parts,
    # the 2-bounce pass without host read-backs) and replayed: the paths of
    # the staged solve, on both calls
    gsol = None
    for _ in range(2):
        gsol = ctx.spoly_solve(mesh, q, gated, precision=binding.MIXED,
                               flags=binding.SOLVE_PERSISTENT | binding.SOLVE_GRAPH, sqrt_table=table, reuse=gsol)
        gp = ctx.spoly_paths(gsol)
        assert _keys(gp) == _keys(paths)
    gstats = ctx.spoly_stats(gsol)
    assert gstats["k2_systems"] == stats["k2_systems"] and gstats["admissible"] == stats["admissible"]
    ctx.spoly_solution_free(gsol)
    for h in (gated, cut):
        ctx.spoly_chains_free(h)
    ctx.spoly_mlp_free(mlp)
    # 1 bounce: every chain of the unculled list
    ex1 = np.ascontiguousarray(s.chains[s.chains[:, 2] < 0])
    ref1, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, ex1)
    g1 = paths[paths["tri"][:, 1] < 0]
    assert ref1.size > 10
    assert_parity(g1, ref1, ex1.shape[0])
    # 2 bounces: a sample
    rng = np.random.default_rng(12)
    k2kept = kept[kept[:, 2] >= 0]
    ex2 = s.chains[s.chains[:, 2] >= 0]
    g2 = paths[paths["tri"][:, 1] >= 0]
    with_path = {(int(a), int(b), int(c)) for a, b, c in zip(g2["query"], g2["tri"][:, 0], g2["tri"][:, 1])}
    rows = set(with_path)
    rows |= {tuple(r) for r in k2kept[rng.choice(k2kept.shape[0], min(200, k2kept.shape[0]), replace=False)].tolist()}
    rows |= {tuple(r) for r in ex2[rng.choice(ex2.shape[0], 100, replace=False)].tolist()}
    sample = np.array(sorted(rows), np.int32)
    ref2, _ = oracle_pool.tt_solve(s.tri, s.x_first, s.x_last, s.eta, sample, table[1])
    mine = g2[[(int(a), int(b), int(c)) in rows for a, b, c in zip(g2["query"], g2["tri"][:, 0], g2["tri"][:, 1])]]
    matched, un, worst = _compare(mine, ref2)
    bad = [u for u in un if not (u[3] & (binding.FLAG_ILL_COND | binding.FLAG_EDGE))]
    assert not bad, (bad, stats)
    assert len(un) <= max(1, 1e-4 * sample.shape[0]), (un, stats)
    assert matched >= len(cases) - 1 and worst <= 1e-5
    assert stats["k2_systems"] > 0 and stats["unsolved"] == 0
