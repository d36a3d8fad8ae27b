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


def _workers():
    return max(1, min(32, os.cpu_count() or 1))


def pool():
    global _POOL
    if _POOL is None:
        _POOL = mp.get_context("spawn").Pool(_workers())
    return _POOL


def _tt_part(args):
    tri, xf, xl, eta, chains, coeffs, n_intervals = args
    from oracle import tt
    return tt.solve(tri, xf, xl, eta, chains, coeffs, n_intervals)


def _rr_part(args):
    tri, xf, xl, chains, n_intervals = args
    from oracle import rr
    return rr.solve(tri, xf, xl, chains, n_intervals), None


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


def tt_solve(tri, xf, xl, eta, chains, coeffs, n_intervals=4096):
    """oracle.tt.solve over the chains, in parallel.  Returns (paths, unrefined uv)."""
    parts = _split(np.asarray(chains, np.int32), 4 * _workers())
    return _run(_tt_part, [(tri, xf, xl, eta, c, coeffs, n_intervals) for c, _ in parts], [o for _, o in parts])


def rr_solve(tri, xf, xl, chains, n_intervals=4096):
    """oracle.rr.solve over the chains, in parallel."""
    parts = _split(np.asarray(chains, np.int32), 4 * _workers())
    return _run(_rr_part, [(tri, xf, xl, c, n_intervals) for c, _ in parts], [o for _, o in parts])[0]
