"""GPU tests of 2-bounce reflection (RR) chains against the FP64 RR oracle:
planted paths through the corridor of two heightfield mirrors in both
precisions, a sample of candidate pairs around them, and one list mixing RR
chains with 1-bounce reflection chains."""
import numpy as np
import pytest

import oracle
from oracle import rr
from paper_2405_13409_gb300 import binding, scenes

from .test_gpu_tt import _compare
from .test_rr_oracle import planted_corridor_cases

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ALLOWED = binding.FLAG_ILL_COND | binding.FLAG_EDGE


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = binding.Context(0, torch.cuda.current_stream().cuda_stream)
    yield c
    c.close()


@pytest.fixture(scope="module")
def corridor():
    return scenes.corridor_scene(seed=0, n_cells=16, n_recv=2)


def _solve(ctx, tri, x0s, x3s, chains, k, types, precision=binding.MIXED):
    n = x0s.shape[0]
    eta = np.ones((n, 3))
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (tri, x0s, x3s, eta, types, k)]
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=np.ascontiguousarray(chains, np.int32))
    sol = ctx.spoly_solve(mesh, q, ch, precision=precision)
    paths = ctx.spoly_paths(sol)
    stats = ctx.spoly_stats(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    return paths, stats


def _rr(n):
    return np.full(n, 2, np.int32), np.full((n, 2), binding.SPOLY_R, np.int32)


@pytest.mark.parametrize("precision", [binding.MIXED, binding.PLAIN_FP64])
def test_planted_corridor_paths_match_oracle(ctx, corridor, precision):
    cases = planted_corridor_cases(31, 24)
    x0s = np.array([c[0] for c in cases])
    x3s = np.array([c[1] for c in cases])
    chains = np.array([[i, c[2], c[3]] for i, c in enumerate(cases)], np.int32)
    paths, stats = _solve(ctx, corridor.tri, x0s, x3s, chains, *_rr(len(cases)), precision=precision)
    ref = rr.solve(corridor.tri, x0s, x3s, chains)
    matched, un, worst = _compare(paths, ref)
    bad = [u for u in un if not (u[3] & ALLOWED)]
    assert not bad, (bad, stats)
    assert matched >= len(cases) - 1, (un, stats)
    assert worst < 1e-9
    for i, c in enumerate(cases):
        got = paths[paths["query"] == i]
        assert any(np.max(np.abs(p["uv"].ravel() - c[4])) < 1e-9 for p in got), (i, c[4], got["uv"])
    assert np.all(paths["flags"] & binding.FLAG_NEWTON)
    assert np.all(paths["residual"] < 1e-9)
    assert stats["unsolved"] == 0


def test_corridor_candidate_sample_matches_oracle(ctx, corridor):
    """(floor, ceiling) pairs around planted paths' triangles and random
    pairs: most have no path; the path sets agree with the oracle's."""
    cases = planted_corridor_cases(32, 4)
    half = corridor.n_tris // 2
    x0s = np.array([c[0] for c in cases])
    x3s = np.array([c[1] for c in cases])
    rng = np.random.default_rng(4)
    rows = []
    for i, c in enumerate(cases):
        for d1 in (-1, 0, 1, 32):
            for d2 in (-32, -1, 0, 2):
                a, b = c[2] + d1, c[3] + d2
                if 0 <= a < half and half <= b < corridor.n_tris:
                    rows.append([i, a, b])
        for _ in range(6):
            rows.append([i, int(rng.integers(0, half)), int(rng.integers(half, corridor.n_tris))])
    chains = np.array(rows, np.int32)
    paths, stats = _solve(ctx, corridor.tri, x0s, x3s, chains, *_rr(len(cases)))
    ref = rr.solve(corridor.tri, x0s, x3s, chains)
    matched, un, worst = _compare(paths, ref)
    bad = [u for u in un if not (u[3] & ALLOWED)]
    assert not bad, (bad, stats)
    assert matched >= len(cases)
    assert len(un) <= max(1, 1e-2 * chains.shape[0])
    assert worst < 1e-9
    assert stats["candidates"] == chains.shape[0]


def test_corridor_large_sample_reaches_fp64_resampling(ctx, corridor):
    """About 1,300 (floor, ceiling) pairs around 16 planted paths and random
    pairs in mixed precision, against the RR oracle (in parallel): unflagged
    paths agree one to one, flagged disagreements stay within 1e-4 of the
    candidates, and the FP64 re-sampling of noisy systems runs."""
    from tests import oracle_pool
    cases = planted_corridor_cases(32, 16)
    half = corridor.n_tris // 2
    x0s = np.array([c[0] for c in cases])
    x3s = np.array([c[1] for c in cases])
    rng = np.random.default_rng(5)
    rows = []
    for i, c in enumerate(cases):
        for d1 in (-2, -1, 0, 1, 2):
            for d2 in (-34, -2, 0, 2, 32):
                a, b = c[2] + d1, c[3] + d2
                if 0 <= a < half and half <= b < corridor.n_tris:
                    rows.append([i, a, b])
        for _ in range(60):
            rows.append([i, int(rng.integers(0, half)), int(rng.integers(half, corridor.n_tris))])
    chains = np.array(rows, np.int32)
    paths, stats = _solve(ctx, corridor.tri, x0s, x3s, chains, *_rr(len(cases)))
    ref = oracle_pool.rr_solve(corridor.tri, x0s, x3s, chains)
    matched, un, worst = _compare(paths, ref)
    bad = [u for u in un if not (u[3] & ALLOWED)]
    assert not bad, (bad, stats)
    assert len(un) <= max(1, 1e-4 * chains.shape[0]), (un, stats)
    assert worst < 1e-9
    assert stats["k2_fp64_samples"] > 0, stats
    for i, c in enumerate(cases):
        got = paths[paths["query"] == i]
        assert any(np.max(np.abs(p["uv"].ravel() - c[4])) < 1e-9 for p in got), (i, c[4], got["uv"])


def test_rr_and_one_bounce_chains_in_one_list(ctx, corridor):
    """One explicit list with RR chains and 1-bounce reflection chains on
    the floor: each part equals its own oracle (RR oracle, C oracle)."""
    oracle.build()
    cases = planted_corridor_cases(33, 6)
    n2 = len(cases)
    half = corridor.n_tris // 2
    x0s = np.array([c[0] for c in cases] + [[-0.6, 0.1, 0.5]] * 4)
    x3s = np.array([c[1] for c in cases] + [[0.3, -0.2, 0.6], [0.1, 0.4, 0.7], [-0.2, -0.5, 0.4], [0.5, 0.5, 0.5]])
    k = np.array([2] * n2 + [1] * 4, np.int32)
    types = np.full((n2 + 4, 2), binding.SPOLY_R, np.int32)
    rows = [[i, c[2], c[3]] for i, c in enumerate(cases)]
    for q in range(n2, n2 + 4):
        rows += [[q, t, -1] for t in range(half)]
    chains = np.array(rows, np.int32)
    paths, stats = _solve(ctx, corridor.tri, x0s, x3s, chains, k, types)
    two = paths[paths["tri"][:, 1] >= 0]
    one = paths[paths["tri"][:, 1] < 0]
    ref2 = rr.solve(corridor.tri, x0s, x3s, chains[:n2])
    m2, un2, w2 = _compare(two, ref2)
    assert not [u for u in un2 if not (u[3] & ALLOWED)], un2
    assert m2 >= n2 and w2 < 1e-9
    ref1, _ = oracle.solve(corridor.tri, x0s, x3s, np.ones((n2 + 4, 3)), types, k, chains[n2:])
    got = sorted((int(p["query"]), int(p["tri"][0])) for p in one)
    want = sorted((int(p["query"]), int(p["tri0"])) for p in ref1)
    assert got == want and len(want) >= 4


def test_rr_cone_keeps_planted_and_exhaustive_paths(ctx, corridor):
    """The 2-bounce cone cull over the corridor (reflected-direction boxes)
    keeps every planted pair and every pair with a path in an exhaustive
    solve of four receivers (all 262,144 (floor, ceiling) pairs each); the
    per-chain test of explicit lists keeps them too."""
    cases = planted_corridor_cases(34, 4, jitter=False)
    half = corridor.n_tris // 2
    n = len(cases)
    x3s = np.array([c[1] for c in cases])
    k, types = _rr(n)
    host = (corridor.tri, np.tile(corridor.x_first[0], (n, 1)), x3s, np.ones((n, 3)), types, k)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in host]
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_CONE, margin=1e-3, tri_range=(0, half),
                                second_range=(half, corridor.n_tris))
    kept = ctx.spoly_chains_copy(ch)
    ctx.spoly_chains_free(ch)
    keys = set(map(tuple, kept.tolist()))
    for i, c in enumerate(cases):
        assert (i, c[2], c[3]) in keys
    t1 = np.repeat(np.arange(half), half)
    t2 = np.tile(np.arange(half, corridor.n_tris), half)
    allc = np.concatenate([np.stack([np.full(t1.size, i), t1, t2], -1) for i in range(n)]).astype(np.int32)
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT_CONE, margin=1e-3,
                                explicit=torch.from_numpy(allc).cuda())
    kept_exp = set(map(tuple, ctx.spoly_chains_copy(ch).tolist()))
    ctx.spoly_chains_free(ch)
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_EXPLICIT, explicit=torch.from_numpy(allc).cuda())
    sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED)
    paths = ctx.spoly_paths(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    assert paths.size >= n
    for p in paths:
        key = (int(p["query"]), int(p["tri"][0]), int(p["tri"][1]))
        assert key in keys and key in kept_exp, p
    assert kept.shape[0] < 0.05 * allc.shape[0]
    assert keys <= kept_exp


@pytest.mark.parametrize("precision", [binding.MIXED, binding.PLAIN_FP64])
def test_two_flat_mirrors_double_image(ctx, precision):
    """Two flat parallel mirrors with face normals: the one path is the
    double mirror image of x3 (closed form), as in the oracle's pin."""
    rng = np.random.default_rng(13)
    F = np.array([[-2.0, -2.0, 0.0], [4.0, -2.0, 0.0], [-2.0, 4.0, 0.0]])
    h = 1.2
    tri = np.zeros((18, 2))
    tri[0:9, 0], tri[9:18, 0] = F.ravel(), np.tile([0.0, 0.0, 1.0], 3)
    tri[0:9, 1], tri[9:18, 1] = (F + [0.0, 0.0, h]).ravel(), np.tile([0.0, 0.0, -1.0], 3)
    n = 6
    x0s = np.c_[rng.uniform(-0.3, 0.3, (n, 2)), rng.uniform(0.2, 0.8, n) * h]
    x3s = np.c_[rng.uniform(0.2, 0.8, (n, 2)), rng.uniform(0.2, 0.8, n) * h]
    chains = np.array([[i, 0, 1] for i in range(n)], np.int32)
    paths, stats = _solve(ctx, tri, x0s, x3s, chains, *_rr(n), precision=precision)
    assert paths.size == n, (paths.size, stats)
    E = np.stack([F[1] - F[0], F[2] - F[0]], 1)
    for i in range(n):
        x0, x3 = x0s[i], x3s[i]
        img = np.r_[x3[:2], -(2.0 * h - x3[2])]
        x1 = x0 + x0[2] / (x0[2] - img[2]) * (img - x0)
        x2 = np.r_[(x0 + (x0[2] + h) / (x0[2] - img[2]) * (img - x0))[:2], h]
        w = np.r_[np.linalg.lstsq(E, x1 - F[0], rcond=None)[0], np.linalg.lstsq(E, x2 - F[0] - [0, 0, h], rcond=None)[0]]
        got = paths[paths["query"] == i]
        assert got.size == 1 and np.max(np.abs(got[0]["uv"].ravel() - w)) < 1e-9, (i, got["uv"], w)


@pytest.mark.parametrize("precision", [binding.MIXED, binding.PLAIN_FP64])
def test_two_bounce_degenerate_inputs(ctx, precision):
    """Degenerate 2-bounce inputs run to completion with no path through
    them: a zero-area triangle, a sliver (collinear vertices), a triangle
    with zero normals, and a light in the first mirror's plane.  The regular
    chain of the same list keeps its closed-form path (double mirror image)."""
    F = np.array([[-2.0, -2.0, 0.0], [4.0, -2.0, 0.0], [-2.0, 4.0, 0.0]])
    h = 1.2
    P = [F, F + [0.0, 0.0, h], np.full((3, 3), [0.3, 0.3, 0.0]), np.array([[0.0, 0, 0], [1, 1, 0], [2, 2, 0]]), F]
    N = [np.tile([0.0, 0, 1], (3, 1)), np.tile([0.0, 0, -1], (3, 1)), np.tile([0.0, 0, 1], (3, 1)),
         np.tile([0.0, 0, 1], (3, 1)), np.zeros((3, 3))]
    tri = np.zeros((18, 5))
    for t in range(5):
        tri[0:9, t], tri[9:18, t] = P[t].ravel(), N[t].ravel()
    x0s = np.array([[0.1, 0.0, 0.6], [0.2, 0.1, 0.0]])
    x3s = np.array([[0.5, 0.3, 0.6], [0.5, 0.3, 0.6]])
    chains = np.array([[0, 0, 1], [0, 2, 1], [0, 0, 2], [0, 3, 1], [0, 1, 3], [0, 4, 1], [0, 0, 4], [1, 0, 1]],
                      np.int32)
    paths, stats = _solve(ctx, tri, x0s, x3s, chains, *_rr(2), precision=precision)
    assert paths.size == 1, (paths, stats)
    p = paths[0]
    assert (int(p["query"]), int(p["tri"][0]), int(p["tri"][1])) == (0, 0, 1)
    x0, x3 = x0s[0], x3s[0]
    img = np.r_[x3[:2], -(2.0 * h - x3[2])]
    x1 = x0 + x0[2] / (x0[2] - img[2]) * (img - x0)
    assert np.allclose(p["x"].ravel()[:3], x1, atol=1e-9) and np.all(np.isfinite(p["uv"]))
    assert p["residual"] < 1e-9


def test_two_bounce_types_and_empty_lists(ctx, corridor):
    """Mixed bounce types (R T) are rejected on host queries and give no
    paths on device queries, where the RR chains of the same list are still
    solved; an empty explicit list is rejected."""
    cases = planted_corridor_cases(35, 2)
    x0s = np.array([c[0] for c in cases] + [cases[0][0]])
    x3s = np.array([c[1] for c in cases] + [cases[0][1]])
    k = np.full(3, 2, np.int32)
    types = np.full((3, 2), binding.SPOLY_R, np.int32)
    types[2] = (binding.SPOLY_R, binding.SPOLY_T)
    chains = np.array([[0, cases[0][2], cases[0][3]], [1, cases[1][2], cases[1][3]], [2, cases[0][2], cases[0][3]]],
                      np.int32)
    eta = np.tile([1.0, 1.5, 1.0], (3, 1))
    mesh = ctx.mesh(torch.from_numpy(np.ascontiguousarray(corridor.tri)).cuda())
    qh = ctx.queries(x0s, x3s, eta, types, k)  # host arrays
    ch = ctx.spoly_build_chains(mesh, qh, binding.CHAINS_EXPLICIT, explicit=chains)
    with pytest.raises(binding.SpolyError) as err:
        ctx.spoly_solve(mesh, qh, ch, precision=binding.MIXED)
    assert err.value.status == binding.SPOLY_EUNSUPPORTED
    ctx.spoly_chains_free(ch)
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x0s, x3s, eta, types, k)]
    qd = ctx.queries(*d)
    ch = ctx.spoly_build_chains(mesh, qd, binding.CHAINS_EXPLICIT, explicit=chains)
    sol = ctx.spoly_solve(mesh, qd, ch, precision=binding.MIXED)
    paths = ctx.spoly_paths(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    assert set(paths["query"].tolist()) == {0, 1}
    for i in (0, 1):
        got = paths[paths["query"] == i]
        assert any(np.max(np.abs(g["uv"].ravel() - cases[i][4])) < 1e-9 for g in got)
    with pytest.raises(binding.SpolyError) as err:
        ctx.spoly_build_chains(mesh, qd, binding.CHAINS_EXPLICIT, explicit=np.zeros((0, 3), np.int32))
    assert err.value.status == binding.SPOLY_EINVAL
