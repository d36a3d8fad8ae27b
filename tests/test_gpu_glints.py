"""GPU tests of the glint workload pieces: the pixel-footprint chain builder
and the pixel filter of the path phase, on a reduced glint scene (256x256
cells, 64x64 pixels) so the oracle can solve exhaustively."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_13409_gb300 import binding, scenes

from .parity import assert_parity
from .parity import footprint_numpy as _footprint_numpy
from .parity import project_pixels as _project

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
def small():
    s = scenes.glint_scene(seed=3, n_cells=256, res=64, n_terms=16)
    cam = s.meta["camera"].as_array()
    s.meta["footprint"] = _footprint_numpy(s, cam)  # computed once for the module
    return s, cam


def _dev(s):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]


def test_footprint_chains_match_brute_force(ctx, small):
    s, cam = small
    d = _dev(s)
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_FOOTPRINT, camera=cam)
    got = ctx.spoly_chains_copy(ch)
    ctx.spoly_chains_free(ch)
    want = s.meta["footprint"]
    gset = set(map(tuple, got[:, :2].tolist()))
    assert len(gset) == got.shape[0], "duplicate candidates"
    # FP32 footprint boxes vs FP64 numpy: allow boundary ties only
    assert len(want - gset) <= 1e-3 * len(want) and len(gset - want) <= 1e-3 * len(want), (len(want), len(gset))
    assert np.all(np.diff(got[:, 0]) >= 0), "candidates are ordered by pixel"


@pytest.mark.parametrize("precision", [binding.PLAIN_FP64, binding.MIXED])
def test_pixel_filtered_solve_matches_oracle(ctx, small, precision):
    s, cam = small
    d = _dev(s)
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_FOOTPRINT, camera=cam)
    n_chains = ctx.spoly_chains_count(ch)
    sol = ctx.spoly_solve(mesh, q, ch, precision=precision, camera=cam)
    paths = ctx.spoly_paths(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    # the oracle solves the brute-force footprint (numpy), not the library's list
    fp = np.array(sorted(s.meta["footprint"]), np.int32)
    chains = np.stack([fp[:, 0], fp[:, 1], -np.ones(fp.shape[0], np.int32)], -1).astype(np.int32)
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, chains)
    keep = _project(cam, ref["x"][:, :3]) == ref["query"]
    ref = ref[keep]
    assert ref.size > 10
    assert_parity(paths, ref, max(n_chains, chains.shape[0]))
    assert np.all(_project(cam, paths["x"][:, :3]) == paths["query"])


def test_footprint_is_conservative(ctx, small):
    """Every admissible path of a sampled pixel (exhaustive oracle over all
    triangles) that projects into the pixel comes from a footprint candidate."""
    s, cam = small
    d = _dev(s)
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_FOOTPRINT, camera=cam)
    chains = ctx.spoly_chains_copy(ch)
    ctx.spoly_chains_free(ch)
    kept = set(map(tuple, chains[:, :2].tolist()))
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k,
                          np.stack([np.zeros(s.n_tris), np.arange(s.n_tris), -np.ones(s.n_tris)], -1).astype(np.int32))
    pix = _project(cam, ref["x"][:, :3])
    hits = [(int(p), int(t)) for p, t in zip(pix, ref["tri0"]) if p >= 0]
    assert len(hits) > 5
    assert all(h in kept for h in hits)


def test_distinct_triangle_footprint_matches_brute_force(ctx, small):
    """FOOTPRINT_UNIQUE keeps the distinct triangles of the brute-force
    footprint, once each, and counts its (pixel, triangle) pairs."""
    s, cam = small
    d = _dev(s)
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_FOOTPRINT_UNIQUE, camera=cam)
    got = ctx.spoly_chains_copy(ch)
    pairs = ctx.spoly_chains_footprint_pairs(ch)
    ctx.spoly_chains_free(ch)
    want = s.meta["footprint"]
    tris = {t for _, t in want}
    assert np.all(got[:, 0] == 0) and np.all(got[:, 2] == -1)
    assert len(set(got[:, 1].tolist())) == got.shape[0], "duplicate triangles"
    gt = set(got[:, 1].tolist())
    assert len(tris - gt) <= 1e-3 * len(tris) and len(gt - tris) <= 1e-3 * len(tris), (len(tris), len(gt))
    assert abs(pairs - len(want)) <= 1e-3 * len(want), (pairs, len(want))
    # chunks of 256 consecutive triangles stay in order
    chunk = got[:, 1] // 256
    for c in np.unique(chunk):
        assert np.all(np.diff(got[chunk == c, 1]) > 0)


@pytest.mark.parametrize("precision", [binding.PLAIN_FP64, binding.MIXED])
def test_pixel_assigned_distinct_solve_matches_oracle(ctx, small, precision):
    """Solving each distinct triangle once and handing every path to the pixel
    its vertex projects into gives the oracle's pixel-filtered solve of the
    brute-force (pixel, triangle) footprint."""
    s, cam = small
    d = _dev(s)
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_FOOTPRINT_UNIQUE, camera=cam)
    pairs = ctx.spoly_chains_footprint_pairs(ch)
    sol = ctx.spoly_solve(mesh, q, ch, precision=precision, camera=cam, flags=binding.SOLVE_PIXEL_ASSIGN)
    paths = ctx.spoly_paths(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    fp = np.array(sorted(s.meta["footprint"]), np.int32)
    chains = np.stack([fp[:, 0], fp[:, 1], -np.ones(fp.shape[0], np.int32)], -1).astype(np.int32)
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, chains)
    ref = ref[_project(cam, ref["x"][:, :3]) == ref["query"]]
    assert ref.size > 10
    assert_parity(paths, ref, max(pairs, chains.shape[0]))
    assert np.all(_project(cam, paths["x"][:, :3]) == paths["query"])


def test_distinct_footprint_rejects_queries_that_differ(ctx, small):
    s, cam = small
    xl = s.x_last.copy()
    xl[7] += 1e-3
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, s.x_first, xl, s.eta, s.types, s.k)]
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    with pytest.raises(binding.SpolyError) as e:
        ctx.spoly_build_chains(mesh, q, binding.CHAINS_FOOTPRINT_UNIQUE, camera=cam)
    assert e.value.status == binding.SPOLY_EINVAL
