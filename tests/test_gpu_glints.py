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
