"""GPU tests of the visibility test and the contributions (the path phase's
last steps, Sec. 4.3) against the FP64 oracle (oracle/render.py), on a
reduced glint scene with a blocker triangle hovering between part of the
surface and the light: occluded paths match the oracle's brute-force
segment tests, contributions match per path, and the glint image (Sec. 5.1)
matches per pixel."""
import numpy as np
import pytest

import oracle
from oracle import render
from paper_2405_13409_gb300 import binding, scenes

from .parity import footprint_numpy, project_pixels

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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
def scene():
    """The reduced glint scene plus one flat blocker triangle at z = 0.3 that
    shadows part of the surface from the light; its footprint (numpy) and the
    oracle's pixel-filtered solve of it."""
    s = scenes.glint_scene(seed=3, n_cells=256, res=64, n_terms=16)
    blk = np.zeros((18, 1))
    blk[0:9, 0] = np.array([[0.05, -0.35, 0.3], [0.75, -0.35, 0.3], [0.05, 0.45, 0.3]]).ravel()
    blk[9:18, 0] = np.tile([0.0, 0.0, -1.0], 3)  # facing down: no reflection paths on it
    s.tri = np.ascontiguousarray(np.concatenate([s.tri, blk], 1))
    cam = s.meta["camera"].as_array()
    fp = np.array(sorted(footprint_numpy(s, cam)), np.int32)
    chains = np.stack([fp[:, 0], fp[:, 1], -np.ones(fp.shape[0], np.int32)], -1).astype(np.int32)
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, chains)
    ref = ref[project_pixels(cam, ref["x"][:, :3]) == ref["query"]]
    vis, f = render.path_terms(s.tri, s.x_first, s.x_last, s.eta, s.types, ref)
    return s, cam, ref, vis, f


def _gpu(ctx, s, cam):
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_FOOTPRINT_UNIQUE, camera=cam)
    sol = ctx.spoly_solve(mesh, q, ch, precision=binding.MIXED, camera=cam, flags=binding.SOLVE_PIXEL_ASSIGN)
    n_vis = ctx.spoly_visibility(mesh, q, sol)
    n = ctx.spoly_stats(sol)["admissible"]
    per = torch.zeros(max(n, 1), dtype=torch.float64, device="cuda")
    img = torch.zeros(s.n_queries, dtype=torch.float64, device="cuda")
    ctx.spoly_contributions(mesh, q, sol, 1.0, per_path=per, image=img)
    paths = ctx.spoly_paths(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    return paths, n_vis, per.cpu().numpy()[:paths.size], img.cpu().numpy()


def test_visibility_and_contributions_match_oracle(ctx, scene):
    s, cam, ref, vis, f = scene
    paths, n_vis, per, img = _gpu(ctx, s, cam)
    assert ref.size > 20 and 0 < int((~vis).sum()) < ref.size, "the blocker must shadow some paths"
    occluded = (paths["flags"] & binding.FLAG_OCCLUDED) != 0
    assert n_vis == int((~occluded).sum())
    # pair GPU and oracle paths by (pixel, triangle) and (u, v)
    pos = {}
    for i, p in enumerate(ref):
        pos.setdefault((int(p["query"]), int(p["tri0"])), []).append(i)
    matched = 0
    for j, p in enumerate(paths):
        cand = pos.get((int(p["query"]), int(p["tri"][0])), [])
        best = [i for i in cand if np.max(np.abs(ref[i]["uv"][:2] - p["uv"][:2])) <= 1e-5]
        if not best:
            assert p["flags"] & (binding.FLAG_ILL_COND | binding.FLAG_EDGE), p
            continue
        i = best[0]
        matched += 1
        assert bool(vis[i]) == (not occluded[j]), (i, vis[i], p["flags"])
        if vis[i]:
            assert abs(per[j] - f[i]) <= 1e-6 * abs(f[i]), (per[j], f[i])
        else:
            assert per[j] == 0.0
    assert matched >= ref.size - 1
    # the image: per-pixel sums of the visible paths' contributions
    want = render.glint_image(ref, f, vis, int(cam[14]), int(cam[15])).ravel()
    assert np.all(np.abs(img - want) <= 1e-6 * np.maximum(np.abs(want), 1e-300) + 1e-300)
    assert np.count_nonzero(want) > 10
