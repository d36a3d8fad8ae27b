"""Parallel runs of the numpy 2-bounce oracles (test infrastructure).

The oracles solve one chain at a time in plain numpy; larger parity samples
split the chain list over worker processes.  The pool uses the ``spawn``
start method, so it is safe to create after CUDA has been initialised in the
parent (a forked child of a CUDA process can hang).  Paths come back with
their chain indices remapped to the caller's list.
"""
import multiprocessing as mp
import os

import numpy as np

_POOL = None
_BLAS_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")


def _workers():
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(32, n))


def pool():
    """The worker pool.  Each worker runs numpy single-threaded (the
    environment variables are inherited by the spawned children before they
    import numpy), so that the workers do not oversubscribe the cores with
    BLAS threads."""
    global _POOL
    if _POOL is None:
        saved = {k: os.environ.get(k) for k in _BLAS_VARS}
        for k in _BLAS_VARS:
            os.environ[k] = "1"
        try:
            _POOL = mp.get_context("spawn").Pool(_workers())
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    return _POOL


def _tt_part(args):
    tri, xf, xl, eta, chains, coeffs, n_intervals, v_solver = args
    from oracle import tt
    return tt.solve(tri, xf, xl, eta, chains, coeffs, n_intervals, v_solver=v_solver)


def _rr_part(args):
    tri, xf, xl, chains, n_intervals, v_solver = args
    from oracle import rr
    return rr.solve(tri, xf, xl, chains, n_intervals, v_solver=v_solver), None


def _run(fn, parts_args, offsets):
    outs = pool().map(fn, parts_args, chunksize=1)
    recs, unref = [], []
    for (paths, un), off in zip(outs, offsets):
        if paths.size:
            paths = paths.copy()
            paths["chain"] += off
            recs.append(paths)
            if un is not None:
                unref.append(un)
    from oracle import PATH_DTYPE
    paths = np.concatenate(recs) if recs else np.zeros(0, PATH_DTYPE)
    return paths, (np.concatenate(unref) if unref else np.zeros((0, 4)))


def _split(chains, n_parts):
    n = len(chains)
    bounds = np.linspace(0, n, n_parts + 1).astype(int)
    return [(chains[a:b], a) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]


def tt_solve(tri, xf, xl, eta, chains, coeffs, n_intervals=4096, v_solver="bisect"):
    """oracle.tt.solve over the chains, in parallel.  Returns (paths, unrefined uv)."""
    parts = _split(np.asarray(chains, np.int32), 4 * _workers())
    return _run(_tt_part, [(tri, xf, xl, eta, c, coeffs, n_intervals, v_solver) for c, _ in parts],
                [o for _, o in parts])


def rr_solve(tri, xf, xl, chains, n_intervals=4096, v_solver="bisect"):
    """oracle.rr.solve over the chains, in parallel."""
    parts = _split(np.asarray(chains, np.int32), 4 * _workers())
    return _run(_rr_part, [(tri, xf, xl, c, n_intervals, v_solver) for c, _ in parts], [o for _, o in parts])[0]


def _bf_part(args):
    tri, xf, xl, eta, chains, grid = args
    from tests.test_tt_oracle import _brute_force
    T = np.asarray(tri, float)
    out = []
    for q, t1, t2 in chains:
        P1, N1 = T[0:9, t1].reshape(3, 3), T[9:18, t1].reshape(3, 3)
        P2, N2 = T[0:9, t2].reshape(3, 3), T[9:18, t2].reshape(3, 3)
        for w in _brute_force(xf[q], xl[q], eta[q], P1, N1, P2, N2, grid=grid):
            out.append((int(q), int(t1), int(t2), np.asarray(w, float)))
    return out


def tt_brute_force(tri, xf, xl, eta, chains, grid=6):
    """The exact TT path set of each chain by the polynomial-free 4D Newton
    brute force of the TT oracle pins, in parallel.  Returns
    [(query, tri0, tri1, (u1, v1, u2, v2))]."""
    parts = _split(np.asarray(chains, np.int32), 4 * _workers())
    res = pool().map(_bf_part, [(tri, xf, xl, eta, c, grid) for c, _ in parts], chunksize=1)
    return [r for part in res for r in part]
