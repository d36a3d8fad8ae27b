"""GPU tests of the glint workload pieces: the pixel-footprint chain builder
and the pixel filter of the path phase, on a reduced glint scene (256x256
cells, 64x64 pixels) so the oracle can solve exhaustively."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_13409_gb300 import binding, scenes

from .parity import assert_parity

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
    return s, s.meta["camera"].as_array()


def _dev(s):
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]


def _project(cam, x):
    o, f, r, u = cam[0:3], cam[3:6], cam[6:9], cam[9:12]
    th, asp, w, h = cam[12], cam[13], int(cam[14]), int(cam[15])
    d = x - o
    fz = d @ f
    sx = (d @ r) / (fz * th * asp)
    sy = (d @ u) / (fz * th)
    fx = (sx + 1) * 0.5 * w
    fy = (1 - sy) * 0.5 * h
    ok = (fz > 0) & (fx >= 0) & (fx < w) & (fy >= 0) & (fy < h)
    pix = np.floor(fy).astype(np.int64) * w + np.floor(fx).astype(np.int64)
    return np.where(ok, pix, -1)


def _footprint_numpy(s, cam):
    """Brute force: triangles whose xy bbox meets each pixel's footprint box."""
    T = s.tri
    xs, ys, zs = T[[0, 3, 6]], T[[1, 4, 7]], T[[2, 5, 8]]
    txl, txh, tyl, tyh = xs.min(0), xs.max(0), ys.min(0), ys.max(0)
    zlo, zhi = float(np.float32(zs.min())), float(np.float32(zs.max()))
    o, f, r, u = cam[0:3], cam[3:6], cam[6:9], cam[9:12]
    th, asp, w, h = cam[12], cam[13], int(cam[14]), int(cam[15])
    out = set()
    for q in range(w * h):
        ix, iy = q % w, q // w
        pts = []
        for k in range(4):
            sx = -1 + 2 * (ix + (k & 1)) / w
            sy = 1 - 2 * (iy + (k >> 1)) / h
            d = f + sx * th * asp * r + sy * th * u
            if d[2] >= 0:
                pts = None
                break
            for z in (zlo, zhi):
                t = (z - o[2]) / d[2]
                pts.append(o + t * d)
        if pts is None:
            continue
        pts = np.array(pts)
        m = 1e-5 * (1 + max(abs(pts[:, 0].min()), abs(pts[:, 1].max())))
        xl, xh = pts[:, 0].min() - m, pts[:, 0].max() + m
        yl, yh = pts[:, 1].min() - m, pts[:, 1].max() + m
        hit = np.where(~((txh < xl) | (txl > xh) | (tyh < yl) | (tyl > yh)))[0]
        out.update((q, int(t)) for t in hit)
    return out


def test_footprint_chains_match_brute_force(ctx, small):
    s, cam = small
    d = _dev(s)
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_FOOTPRINT, camera=cam)
    got = ctx.spoly_chains_copy(ch)
    ctx.spoly_chains_free(ch)
    want = _footprint_numpy(s, cam)
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
    chains = ctx.spoly_chains_copy(ch)
    sol = ctx.spoly_solve(mesh, q, ch, precision=precision, camera=cam)
    paths = ctx.spoly_paths(sol)
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, chains)
    keep = _project(cam, ref["x"][:, :3]) == ref["query"]
    ref = ref[keep]
    assert ref.size > 10
    assert_parity(paths, ref, chains.shape[0])
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
