"""The no-allocation entry point (spoly_solve_noalloc) against the regular
spoly_solve, through the C ABI, on two calls in a row.

It serves callers that cannot allocate device memory; its scratch is a
static device array shared by every call, so this file runs last (it is
named to be collected last) and also passes when run alone."""
import numpy as np
import pytest

from paper_2405_13409_gb300 import binding, scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _keys(paths):
    return sorted(zip(paths["query"].tolist(), paths["tri"][:, 0].tolist(), paths["uv"][:, 0].tolist(),
                      paths["uv"][:, 1].tolist()))


@pytest.mark.parametrize("precision", [binding.PLAIN_FP64, binding.MIXED])
def test_noalloc_matches_spoly_solve_twice(precision):
    import __graft_entry__ as g
    g.build_library()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    stream = torch.cuda.current_stream().cuda_stream
    s = scenes.reflect_scene(seed=4, n_cells=4, n_recv=8)  # 32 triangles x 64 receivers = 2048 chains
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
    ctx = binding.Context(0, stream)
    mesh, q = ctx.mesh(d[0]), ctx.queries(*d[1:])
    ch = ctx.spoly_build_chains(mesh, q, binding.CHAINS_ALL)
    sol = ctx.spoly_solve(mesh, q, ch, precision=precision)
    ref = ctx.spoly_paths(sol)
    chains = torch.from_numpy(ctx.spoly_chains_copy(ch)).cuda()
    ctx.spoly_solution_free(sol)
    ctx.spoly_chains_free(ch)
    ctx.close()
    assert ref.size > 10 and chains.shape[0] <= 4096
    cap = 4 * ref.size + 64
    for call in range(2):
        buf = torch.zeros(cap * binding.PATH_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        st, n, msg = binding.spoly_solve_noalloc(0, stream, *d, chains, precision, buf, cap)
        assert st == binding.SPOLY_OK, msg
        got = np.frombuffer(buf.cpu().numpy().tobytes(), dtype=binding.PATH_DTYPE)[:n]
        assert n == ref.size, (call, n, ref.size)
        for a, b in zip(_keys(got), _keys(ref)):
            assert a[:2] == b[:2] and abs(a[2] - b[2]) <= 1e-5 and abs(a[3] - b[3]) <= 1e-5, (call, a, b)


def _setup():
    import __graft_entry__ as g
    g.build()
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.cuda.current_stream().cuda_stream


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _call(stream, d, chains, precision, cap):
    buf = torch.zeros(max(cap, 1) * binding.PATH_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    st, n, msg = binding.spoly_solve_noalloc(0, stream, *d, _dev(chains), precision, buf, cap)
    got = np.frombuffer(buf.cpu().numpy().tobytes(), dtype=binding.PATH_DTYPE)[:min(n, cap)]
    return st, n, msg, got


@pytest.mark.parametrize("precision", [binding.PLAIN_FP64, binding.MIXED])
def test_noalloc_matches_oracle_refraction_and_flat(precision):
    """Refraction chains of curved triangles plus flat-shaded triangles
    (which the mixed solve sends to its FP64 side queue) against the FP64
    oracle, twice in a row."""
    import oracle
    from tests.parity import assert_parity
    stream = _setup()
    s = scenes.refract_scene(seed=2, n_cells=8, n_recv=8)  # 128 triangles x 64 receivers
    tri = s.tri.copy()
    tri[12:18, :16] = np.tile(tri[9:12, :16], (2, 1))  # the first 16 triangles flat-shaded
    chains = scenes.all_pairs(s.n_queries, s.n_tris)[:4096]
    ref, _ = oracle.solve(tri, s.x_first, s.x_last, s.eta, s.types, s.k, chains)
    assert ref.size > 5
    d = [_dev(a) for a in (tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
    for _ in range(2):
        st, n, msg, got = _call(stream, d, chains, precision, 4 * ref.size + 64)
        assert st == binding.SPOLY_OK, msg
        assert_parity(got, ref, chains.shape[0])


def test_noalloc_capacity_and_invalid_chains():
    """ECAPACITY reports the full count and writes a prefix of the path set;
    an out-of-range index, a 2-bounce chain and a k = 2 query are rejected
    with SPOLY_EINVAL and the chain's index before any solve runs; a valid
    call afterwards still matches."""
    stream = _setup()
    s = scenes.reflect_scene(seed=4, n_cells=4, n_recv=8)
    d = [_dev(a) for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
    chains = scenes.all_pairs(s.n_queries, s.n_tris)
    st, n, msg, full = _call(stream, d, chains, binding.MIXED, 4096)
    assert st == binding.SPOLY_OK and n > 4, msg
    st, n2, msg, part = _call(stream, d, chains, binding.MIXED, 3)
    assert st == binding.SPOLY_ECAPACITY and n2 == n, (st, n2, msg)
    keys = set(_keys(full))
    assert len(part) == 3 and all(k in keys for k in _keys(part))
    for bad_row, what in (([0, s.n_tris, -1], "triangle"), ([s.n_queries, 0, -1], "query"),
                          ([0, 0, 1], "second triangle")):
        bad = chains.copy()
        bad[100] = bad_row
        st, _, msg, _ = _call(stream, d, bad, binding.MIXED, 16)
        assert st == binding.SPOLY_EINVAL and "chain 100" in msg and what in msg, msg
    k2 = s.k.copy()
    k2[5] = 2
    d2 = d[:5] + [_dev(k2)]
    st, _, msg, _ = _call(stream, d2, chains, binding.MIXED, 16)
    first = int(np.nonzero(chains[:, 0] == 5)[0][0])
    assert st == binding.SPOLY_EINVAL and f"chain {first}" in msg and "k != 1" in msg, msg
    st, n3, msg, again = _call(stream, d, chains, binding.MIXED, 4096)
    assert st == binding.SPOLY_OK and n3 == n and sorted(_keys(again)) == sorted(_keys(full)), msg


def test_noalloc_rejects_oversized_batches():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    stream = torch.cuda.current_stream().cuda_stream
    s = scenes.reflect_scene(seed=4, n_cells=4, n_recv=12)  # 32 x 144 = 4608 chains > 4096
    d = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (s.tri, s.x_first, s.x_last, s.eta, s.types, s.k)]
    chains = torch.from_numpy(scenes.all_pairs(s.n_queries, s.n_tris)).cuda()
    buf = torch.zeros(104, dtype=torch.uint8, device="cuda")
    st, n, msg = binding.spoly_solve_noalloc(0, stream, *d, chains, binding.MIXED, buf, 1)
    assert st == binding.SPOLY_EINVAL and "4096" in msg
