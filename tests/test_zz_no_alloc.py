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
