"""GPU tests of the scheduling layer: the persistent work-queue isolation
kernel, graph-captured replays of the 1-bounce solve and the launch-shape
autotuner, on uneven candidate lists and a mixed 1- and 2-bounce batch."""
import numpy as np
import pytest

from paper_2405_13409_gb300 import binding, scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sctx():
    """A context on a non-default stream (graph capture needs one)."""
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    stream = torch.cuda.Stream()
    c = binding.Context(0, stream.cuda_stream)
    yield c, stream
    c.close()


def _keys(p):
    return sorted(zip(p["query"].tolist(), p["tri"][:, 0].tolist(), np.round(p["uv"][:, 0], 10).tolist(),
                      np.round(p["uv"][:, 1], 10).tolist()))


def _uneven_refraction(ctx, stream):
    """Refraction workload on a reduced receiver grid, chains from the cone
    cull: per-receiver candidate counts vary by orders of magnitude."""
    s = scenes.refract_scene(seed=0, n_cells=32, n_recv=48)
    with torch.cuda.stream(stream):
        d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
    stream.synchronize()
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_CONE, margin=1e-3)
    return s, d, mesh, q, ch


@pytest.mark.parametrize("precision", [binding.MIXED, binding.PLAIN_FP64])
def test_persistent_isolation_matches_grid_stride(sctx, precision):
    ctx, stream = sctx
    s, d, mesh, q, ch = _uneven_refraction(ctx, stream)
    ref_sol = ctx.spoly_solve(mesh, q, ch, precision=precision)
    ref = ctx.spoly_paths(ref_sol)
    ref_stats = ctx.spoly_stats(ref_sol)
    sol = ctx.spoly_solve(mesh, q, ch, precision=precision, flags=binding.SOLVE_PERSISTENT)
    got = ctx.spoly_paths(sol)
    stats = ctx.spoly_stats(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_solution_free(ref_sol)
    ctx.spoly_chains_free(ch)
    assert ref.size > 50
    assert _keys(got) == _keys(ref)
    for k in ("candidates", "v_roots", "queued", "admissible"):
        assert stats[k] == ref_stats[k], k


def test_graph_replays_match_and_recapture(sctx):
    ctx, stream = sctx
    s, d, mesh, q, ch = _uneven_refraction(ctx, stream)
    base = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED)
    want = _keys(ctx.spoly_paths(base))
    ctx.spoly_solution_free(base)
    sol = None
    for _ in range(3):
        sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED, flags=binding.SOLVE_GRAPH | binding.SOLVE_PERSISTENT,
                              reuse=sol)
        assert _keys(ctx.spoly_paths(sol)) == want
    # the replayed solve against the FP64 oracle's exhaustive solve of 96
    # sampled receivers (every triangle)
    import oracle
    from .parity import assert_parity
    rng = np.random.default_rng(8)
    qs = np.sort(rng.choice(s.n_queries, 96, replace=False)).astype(np.int32)
    every = np.stack([np.repeat(qs, s.n_tris), np.tile(np.arange(s.n_tris, dtype=np.int32), qs.size),
                      -np.ones(qs.size * s.n_tris, np.int32)], -1).astype(np.int32)
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, every)
    got = ctx.spoly_paths(sol)
    assert ref.size > 10
    assert_parity(got[np.isin(got["query"], qs)], ref, every.shape[0])
    # a different chain list (a triangle range) is captured again
    ch2 = ctx.spoly_build_chains(mesh, q, binding.CHAINS_CONE, margin=1e-3, tri_range=(0, s.n_tris // 2))
    ref2 = ctx.spoly_solve(mesh, q, ch2, precision=binding.MIXED)
    want2 = _keys(ctx.spoly_paths(ref2))
    ctx.spoly_solution_free(ref2)
    sol = ctx.spoly_solve(mesh, q, ch2, precision=binding.MIXED, flags=binding.SOLVE_GRAPH, reuse=sol)
    assert _keys(ctx.spoly_paths(sol)) == want2
    ctx.spoly_solution_free(sol)
    # a path buffer too small for the replay falls back to the staged solve
    sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED, flags=binding.SOLVE_GRAPH, path_capacity=8)
    assert _keys(ctx.spoly_paths(sol)) == want
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    ctx.spoly_chains_free(ch2)


def test_graph_needs_a_stream():
    import __graft_entry__ as g
    g.build()
    c = binding.Context(0, None)
    s = scenes.reflect_scene(n_cells=4, n_recv=4)
    mesh, q = c.mesh(s.tri), c.queries(s.x_first, s.x_last, s.eta, s.types, s.k)
    ch = c.spoly_build_chains(mesh, q, binding.CHAINS_ALL)
    with pytest.raises(binding.SpolyError):
        c.spoly_solve(mesh, q, ch, flags=binding.SOLVE_GRAPH)
    c.spoly_chains_free(ch)
    c.close()


def test_autotune_table_and_choice(sctx):
    ctx, stream = sctx
    s, d, mesh, q, ch = _uneven_refraction(ctx, stream)
    best, table = ctx.spoly_autotune(mesh, q, ch, binding.MIXED)
    assert len(table) == 32
    assert all(t[3] > 0 for t in table)
    assert best[3] == min(t[3] for t in table)
    assert best[:3] in [t[:3] for t in table]
    # the tuned shape is used by later persistent solves and gives the same paths
    ref = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED)
    sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED, flags=binding.SOLVE_PERSISTENT)
    assert _keys(ctx.spoly_paths(sol)) == _keys(ctx.spoly_paths(ref))
    ctx.spoly_solution_free(sol)
    ctx.spoly_solution_free(ref)
    ctx.spoly_chains_free(ch)


def test_mixed_bounce_batch_matches_separate_solves(sctx):
    """A batch of queries with k in {1, 2} and candidate counts spread over
    two orders of magnitude, solved in one call (persistent isolation for
    the 1-bounce part), equals the separate solves of each part."""
    ctx, stream = sctx
    from tests.test_tt_oracle import planted_slab_cases
    rng = np.random.default_rng(5)
    slab = scenes.slab_scene(seed=0, n_cells=16, n_recv=4)
    half = slab.n_tris // 2
    cases = planted_slab_cases(21, 8)
    nq = 24
    k = np.where(np.arange(nq) < 8, 2, 1).astype(np.int32)
    xf = np.tile(slab.x_first[0], (nq, 1))
    xl = np.concatenate([np.array([c[1] for c in cases]), rng.uniform([-1, -1, -0.2], [1, 1, -0.1], (nq - 8, 3))])
    eta = np.tile([1.0, 1.5, 1.0], (nq, 1))
    types = np.full((nq, 2), binding.SPOLY_T, np.int32)
    rows = []
    for i in range(nq):
        n = int(round(10 ** rng.uniform(1, 3)))
        if k[i] == 2:
            c = cases[i]
            rows.append([i, c[2], c[3]])
            t1 = rng.integers(0, half, n)
            rows += [[i, int(a), int(a) + half] for a in t1]
        else:
            rows += [[i, int(t), -1] for t in rng.choice(half, min(n, half), replace=False)]
    chains = np.array(rows, np.int32)
    with torch.cuda.stream(stream):
        d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (slab.tri, xf, xl, eta, types, k)]
    stream.synchronize()
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=chains)
    sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED, flags=binding.SOLVE_PERSISTENT)
    both = ctx.spoly_paths(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    parts = []
    for sel in (chains[:, 2] < 0, chains[:, 2] >= 0):
        ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=np.ascontiguousarray(chains[sel]))
        sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED)
        parts.append(ctx.spoly_paths(sol))
        ctx.spoly_solution_free(sol)
        ctx.spoly_chains_free(ch)
    sep = np.concatenate(parts)
    assert both.size == sep.size and both.size >= 8
    assert sorted(zip(both["query"].tolist(), both["tri"][:, 0].tolist(), both["tri"][:, 1].tolist(),
                      np.round(both["uv"].reshape(-1, 4), 9).tolist())) == \
        sorted(zip(sep["query"].tolist(), sep["tri"][:, 0].tolist(), sep["tri"][:, 1].tolist(),
                   np.round(sep["uv"].reshape(-1, 4), 9).tolist()))
    assert np.all(chains[both["chain"], 0] == both["query"])
