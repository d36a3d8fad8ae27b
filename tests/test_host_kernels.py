"""The CUDA path's per-candidate device functions, compiled for the host
(tests/host_k1.cpp), checked against the FP64 oracle on small cases.  This
exercises the kernels' arithmetic without a GPU; the GPU tests are the parity
tests proper."""
import numpy as np
import pytest

import oracle
from paper_2405_13409_gb300 import scenes

from . import host_kernels
from .parity import assert_parity
from .test_oracle_pins import _planted_cases

PATH_LIKE = np.dtype([("query", "<i4"), ("tri", "<i4", (2,)), ("uv", "<f8", (4,)), ("flags", "<u4")])


def _host_solve(tri, x0, x2, eta, types, chains, precision):
    rows = []
    for c, (q, t, _) in enumerate(chains):
        p, st = host_kernels.candidate(tri[:, t], x0[q], x2[q], int(types[q, 0]), eta[q, 0], eta[q, 1], precision)
        for u, v, f in p:
            rows.append((q, (t, -1), (u, v, 0.0, 0.0), int(f)))
    return np.array(rows, dtype=PATH_LIKE)


@pytest.mark.parametrize("precision", [0, 1])
def test_host_kernels_reflection_small(precision):
    s = scenes.reflect_scene(seed=3, n_cells=6, n_recv=10)
    ref, _ = oracle.solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.k, s.chains)
    got = _host_solve(s.tri, s.x_first, s.x_last, s.eta, s.types, s.chains, precision)
    assert ref.size > 20
    assert_parity(got, ref, s.chains.shape[0])


@pytest.mark.parametrize("type_", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_host_kernels_planted(type_, precision):
    tri, x0, x2 = _planted_cases(90 + type_, 400, type_)
    n = tri.shape[1]
    eta = np.tile([1.0, 1.5 if type_ else 1.0, 1.0], (n, 1))
    types = np.full((n, 2), type_, np.int32)
    chains = np.stack([np.arange(n), np.arange(n), -np.ones(n)], -1).astype(np.int32)
    ref, _ = oracle.solve(tri, x0, x2, eta, types, np.ones(n, np.int32), chains)
    got = _host_solve(tri, x0, x2, eta, types, chains, precision)
    assert ref.size > 300
    assert_parity(got, ref, n, min_recall=1.0, max_flagged_frac=1e-4)


@pytest.mark.parametrize("type_", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_host_kernels_planted_gpu_test_cases(type_, precision):
    """The strongly curved planted cases of the GPU parity test, through the
    kernels' host build: both precisions at the benchmark spec's bound."""
    tri, x0, x2 = _planted_cases(70 + type_, 2000, type_)
    n = tri.shape[1]
    eta = np.tile([1.0, 1.5 if type_ else 1.0, 1.0], (n, 1))
    types = np.full((n, 2), type_, np.int32)
    chains = np.stack([np.arange(n), np.arange(n), -np.ones(n)], -1).astype(np.int32)
    ref, _ = oracle.solve(tri, x0, x2, eta, types, np.ones(n, np.int32), chains)
    got = _host_solve(tri, x0, x2, eta, types, chains, precision)
    assert ref.size > 1500
    assert_parity(got, ref, n, min_recall=1.0, max_flagged_frac=1e-4)
