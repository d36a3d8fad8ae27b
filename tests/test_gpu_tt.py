"""GPU tests of 2-bounce refraction (TT) chains against the FP64 TT oracle:
planted paths through the curved slab, a sample of candidate pairs, flat
slabs with Fermat's closed form, and chain lists that mix 1- and 2-bounce
chains."""
import json
import os

import numpy as np
import pytest

from oracle import tt
from paper_2405_13409_gb300 import binding, scenes

from .test_tt_oracle import _fermat, planted_slab_cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = binding.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


def _table():
    g = json.load(open(os.path.join(HERE, "golden", "sqrt_pieces.json")))
    return np.array(g["breaks"]), np.array(g["coeffs"])


def _solve(ctx, tri, x0s, x3s, chains, precision=binding.MIXED, kk=2):
    n = x0s.shape[0]
    eta = np.tile([1.0, 1.5, 1.0], (n, 1))
    types = np.full((n, 2), binding.SPOLY_T, np.int32)
    k = np.full(n, kk, np.int32)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (tri, x0s, x3s, eta, types, k)]
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=np.ascontiguousarray(chains, np.int32))
    sol = ctx.spoly_solve(mesh, q, ch, precision=precision, sqrt_table=_table())
    paths = ctx.spoly_paths(sol)
    stats = ctx.spoly_stats(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    return paths, stats, eta


def _compare(paths, ref, tol=1e-5):
    """Pairs GPU and oracle TT paths by (query, tri0, tri1) and (u1,v1,u2,v2)."""
    from collections import defaultdict
    G = defaultdict(list)
    for p in paths:
        G[(int(p["query"]), int(p["tri"][0]), int(p["tri"][1]))].append((p["uv"].ravel(), int(p["flags"])))
    R = defaultdict(list)
    for p in ref:
        R[(int(p["query"]), int(p["tri0"]), int(p["tri1"]))].append((p["uv"].ravel(), int(p["flags"])))
    matched, unmatched, worst = 0, [], 0.0
    for key in set(G) | set(R):
        a, b = list(G.get(key, [])), list(R.get(key, []))
        used = set()
        for x, fx in a:
            best = None
            for j, (y, fy) in enumerate(b):
                if j in used:
                    continue
                d = float(np.max(np.abs(x - y)))
                if d <= tol and (best is None or d < best[0]):
                    best = (d, j)
            if best is None:
                unmatched.append(("gpu", key, x.tolist(), fx))
            else:
                used.add(best[1])
                matched += 1
                worst = max(worst, best[0])
        for j, (y, fy) in enumerate(b):
            if j not in used:
                unmatched.append(("ref", key, y.tolist(), fy))
    return matched, unmatched, worst


ALLOWED = binding.FLAG_ILL_COND | binding.FLAG_EDGE


@pytest.mark.parametrize("precision", [binding.MIXED, binding.PLAIN_FP64])
def test_planted_slab_paths_match_oracle(ctx, precision):
    cases = planted_slab_cases(11, 24)
    s = scenes.slab_scene(seed=0, n_cells=16, n_recv=4)
    x0s = np.array([c[0] for c in cases])
    x3s = np.array([c[1] for c in cases])
    chains = np.array([[i, c[2], c[3]] for i, c in enumerate(cases)], np.int32)
    paths, stats, eta = _solve(ctx, s.tri, x0s, x3s, chains, precision)
    breaks, coeffs = _table()
    ref, _ = tt.solve(s.tri, x0s, x3s, eta, chains, coeffs)
    matched, un, worst = _compare(paths, ref)
    bad = [u for u in un if not (u[3] & ALLOWED)]
    assert not bad, (bad, stats)
    assert matched >= len(cases) - 1, (un, stats)
    assert worst < 1e-9
    # every planted path is returned
    for i, c in enumerate(cases):
        got = paths[paths["query"] == i]
        assert any(np.max(np.abs(p["uv"].ravel() - c[4])) < 1e-9 for p in got), (i, c[4], got["uv"])
    assert np.all(paths["flags"] & binding.FLAG_NEWTON)
    assert np.all(paths["residual"] < 1e-9)
    assert stats["unsolved"] == 0


def test_candidate_sample_matches_oracle(ctx):
    """Receivers below the slab and (top, bottom) pairs near the planted
    paths' triangles: most have no path; the path sets agree."""
    cases = planted_slab_cases(12, 6)
    s = scenes.slab_scene(seed=0, n_cells=16, n_recv=4)
    half = s.n_tris // 2
    x0s = np.array([c[0] for c in cases])
    x3s = np.array([c[1] for c in cases])
    rng = np.random.default_rng(3)
    rows = []
    for i, c in enumerate(cases):
        t1, t2 = c[2], c[3]
        for d1 in (-2, -1, 0, 1, 2):
            for d2 in (-34, -2, 0, 2, 32):
                a, b = t1 + d1, t2 + d2
                if 0 <= a < half and half <= b < s.n_tris:
                    rows.append([i, a, b])
        for _ in range(10):
            rows.append([i, int(rng.integers(0, half)), int(rng.integers(half, s.n_tris))])
    chains = np.array(rows, np.int32)
    paths, stats, eta = _solve(ctx, s.tri, x0s, x3s, chains)
    breaks, coeffs = _table()
    ref, _ = tt.solve(s.tri, x0s, x3s, eta, chains, coeffs)
    matched, un, worst = _compare(paths, ref)
    bad = [u for u in un if not (u[3] & ALLOWED)]
    assert not bad, (bad, stats)
    assert matched >= len(cases)
    assert len(un) <= max(1, 1e-2 * chains.shape[0])
    assert stats["candidates"] == chains.shape[0]


@pytest.mark.parametrize("table_kind", ["oracle", "library default"])
def test_large_sample_reaches_fp64_resampling_and_split_pieces(ctx, table_kind):
    """About 4,000 (top, bottom) pairs around 48 planted paths in mixed
    precision, half of them seen from a grazing light so that the sqrt
    argument over the top triangle spans two pieces (SQRT_SPLIT): against
    the TT oracle with the same sqrt table (the oracle's fitted pieces, or
    the library's default pieces fed to the oracle).  Unflagged paths agree
    one to one, flagged disagreements stay within 1e-4 of the candidates,
    the FP64 re-sampling of noisy systems runs, and split paths are found."""
    from tests import oracle_pool
    s = scenes.slab_scene(seed=0, n_cells=16, n_recv=4)
    half = s.n_tris // 2
    cases = planted_slab_cases(12, 24) + planted_slab_cases(21, 24, x0=[-2.2, 0.0, 1.0], x_range=(-0.45, -0.1))
    x0s = np.array([c[0] for c in cases])
    x3s = np.array([c[1] for c in cases])
    rng = np.random.default_rng(3)
    rows = []
    for i, c in enumerate(cases):
        t1, t2 = c[2], c[3]
        for d1 in (-2, -1, 0, 1, 2):
            for d2 in (-34, -2, 0, 2, 32):
                a, b = t1 + d1, t2 + d2
                if 0 <= a < half and half <= b < s.n_tris:
                    rows.append([i, a, b])
        for _ in range(58):
            rows.append([i, int(rng.integers(0, half)), int(rng.integers(half, s.n_tris))])
    chains = np.array(rows, np.int32)
    table = _table() if table_kind == "oracle" else binding.spoly_default_sqrt_table()
    n = x0s.shape[0]
    eta = np.tile([1.0, 1.5, 1.0], (n, 1))
    types = np.full((n, 2), binding.SPOLY_T, np.int32)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, x0s, x3s, eta, types, np.full(n, 2, np.int32))]
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=chains)
    sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED, sqrt_table=table)
    paths, stats = ctx.spoly_paths(sol), ctx.spoly_stats(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    ref, _ = oracle_pool.tt_solve(s.tri, x0s, x3s, eta, chains, table[1])
    matched, un, worst = _compare(paths, ref)
    bad = [u for u in un if not (u[3] & ALLOWED)]
    assert not bad, (bad, stats)
    assert len(un) <= max(1, 1e-4 * chains.shape[0]), (un, stats)
    assert worst < 1e-9
    assert stats["k2_fp64_samples"] > 0, stats
    split = paths[(paths["flags"] & binding.FLAG_SQRT_SPLIT) != 0]
    assert split.size >= 8, (split.size, stats)
    assert np.sum((ref["flags"] & binding.FLAG_SQRT_SPLIT) != 0) == split.size
    for i, c in enumerate(cases):
        got = paths[paths["query"] == i]
        assert any(np.max(np.abs(p["uv"].ravel() - c[4])) < 1e-9 for p in got), (i, c[4], got["uv"])


def test_flat_slab_fermat(ctx):
    rng = np.random.default_rng(4)
    P1 = np.array([[-1.0, -1.0, 0.0], [1.5, -1.0, 0.0], [-1.0, 1.5, 0.0]])
    P2 = P1 + [0.0, 0.0, -0.3]
    n = np.array([0.0, 0.0, 1.0])
    tri = np.zeros((18, 2))
    tri[0:9, 0] = P1.ravel()
    tri[9:18, 0] = np.tile(n, 3)
    tri[0:9, 1] = P2.ravel()
    tri[9:18, 1] = np.tile(n, 3)
    x0s = np.array([0.2, 0.1, 2.0]) + rng.normal(size=(6, 3)) * 0.2
    x3s = np.array([0.0, 0.0, -1.0]) + rng.normal(size=(6, 3)) * 0.3
    chains = np.array([[i, 0, 1] for i in range(6)], np.int32)
    paths, stats, eta = _solve(ctx, tri, x0s, x3s, chains)
    n_in = 0
    for i in range(6):
        want = _fermat(x0s[i], x3s[i], (1.0, 1.5, 1.0), P1, P2)
        got = paths[paths["query"] == i]
        inside = min(want[0], want[1], 1 - want[0] - want[1], want[2], want[3], 1 - want[2] - want[3]) > 1e-6
        if inside:
            n_in += 1
            assert got.size == 1
            np.testing.assert_allclose(got[0]["uv"].ravel(), want, atol=1e-7)
        else:
            assert got.size == 0
    assert n_in >= 3


def test_mixed_one_and_two_bounce_lists(ctx):
    """One list with 1-bounce (tri1 = -1) and 2-bounce chains returns the
    union of the two solves, with each path's chain index."""
    cases = planted_slab_cases(13, 6)
    s = scenes.slab_scene(seed=0, n_cells=16, n_recv=4)
    n = len(cases)
    x0s = np.array([c[0] for c in cases])
    x3s = np.array([c[1] for c in cases])
    # queries 0..n-1: 2-bounce; n..2n-1: 1-bounce refraction from x0 into the slab top to a point below it
    eta1 = np.tile([1.0, 1.5, 1.0], (n, 1))
    rows2 = [[i, c[2], c[3]] for i, c in enumerate(cases)]
    rows1 = [[n + i, c[2], -1] for i, c in enumerate(cases)]
    chains = np.array([r for pair in zip(rows2, rows1) for r in pair], np.int32)
    xf = np.concatenate([x0s, x0s])
    xl = np.concatenate([x3s, x3s * [1, 1, 0] + [0, 0, -0.15]])
    eta = np.concatenate([eta1, eta1])
    types = np.full((2 * n, 2), binding.SPOLY_T, np.int32)
    k = np.concatenate([np.full(n, 2, np.int32), np.full(n, 1, np.int32)])
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, xf, xl, eta, types, k)]
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=chains)
    sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED, sqrt_table=_table())
    paths = ctx.spoly_paths(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    two = paths[paths["tri"][:, 1] >= 0]
    one = paths[paths["tri"][:, 1] < 0]
    assert two.size >= n - 1
    assert np.all(chains[two["chain"], 2] >= 0) and np.all(chains[one["chain"], 2] == -1)
    assert np.all(chains[two["chain"], 0] == two["query"]) and np.all(chains[one["chain"], 0] == one["query"])
    # the 1-bounce part equals a solve of the 1-bounce chains alone
    only1 = np.array(rows1, np.int32)
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=only1)
    sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED)
    ref1 = ctx.spoly_paths(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    assert sorted(map(tuple, np.round(one["uv"][:, :2], 9).tolist())) == \
        sorted(map(tuple, np.round(ref1["uv"][:, :2], 9).tolist()))


def _slab_queries(s, x3s):
    n = x3s.shape[0]
    xf = np.tile(s.x_first[0], (n, 1))
    return (xf, np.ascontiguousarray(x3s), np.tile([1.0, 1.5, 1.0], (n, 1)),
            np.full((n, 2), binding.SPOLY_T, np.int32), np.full(n, 2, np.int32))


def test_tt_cone_keeps_planted_and_exhaustive_paths(ctx):
    """The 2-bounce cone cull over the slab keeps every planted pair and every
    pair with a path in an exhaustive solve of four receivers (all 262,144
    (top, bottom) pairs each)."""
    cases = planted_slab_cases(14, 4)
    s = scenes.slab_scene(seed=0, n_cells=16, n_recv=4)
    half = s.n_tris // 2
    x3s = np.array([c[1] for c in cases])
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, *_slab_queries(s, x3s))]
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_CONE, margin=1e-3, tri_range=(0, half),
                                second_range=(half, s.n_tris))
    kept = ctx.spoly_chains_copy(ch)
    ctx.spoly_chains_free(ch)
    keys = set(map(tuple, kept.tolist()))
    for i, c in enumerate(cases):
        assert (i, c[2], c[3]) in keys
    # exhaustive: every (top, bottom) pair for each receiver
    t1 = np.repeat(np.arange(half), half)
    t2 = np.tile(np.arange(half, s.n_tris), half)
    allc = np.concatenate([np.stack([np.full(t1.size, i), t1, t2], -1) for i in range(len(cases))]).astype(np.int32)
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=allc)
    sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED, sqrt_table=_table())
    paths = ctx.spoly_paths(sol)
    stats = ctx.spoly_stats(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    print("tt cone: kept", kept.shape[0], "of", allc.shape[0], "exhaustive paths", paths.size, stats)
    assert paths.size >= len(cases)
    for p in paths:
        assert (int(p["query"]), int(p["tri"][0]), int(p["tri"][1])) in keys, p
    assert kept.shape[0] < 0.05 * allc.shape[0]
