"""FP64 CPU oracle for the specular-polynomial solve (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline
and reference legs may import this package.  The product path (the CUDA
library and its binding) never imports, links or runs it, and the oracle
shares no code with it: the C++ source here is compiled on its own with g++.

``build()`` compiles ``spoly_oracle.cpp`` into ``_liboracle.so`` beside it.
``solve()`` runs the full 1-bounce pipeline (Sec. 3.5 R/T, Eq. eq_bezout,
Sec. 4.2, Sec. 4.3) over an explicit chain list on all host cores.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spoly_oracle.cpp")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

F_ILL_COND = 1
F_EDGE = 2
F_BACKFACE = 4
F_NEWTON_REFINED = 8
F_SQRT_SPLIT = 16
F_TANGENT = 32

PATH_DTYPE = np.dtype([
    ("chain", "<i8"), ("query", "<i4"), ("tri0", "<i4"), ("tri1", "<i4"), ("pad", "<i4"),
    ("uv", "<f8", (4,)), ("x", "<f8", (6,)), ("residual", "<f8"), ("flags", "<u4"), ("pad2", "<u4"),
])


class _Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in
                ("candidates", "degenerate", "v_roots", "u_roots", "admissible", "flagged")]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, C++17, pthreads)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + ".tmp"
            subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread", "-o", tmp, _SRC],
                           check=True)
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.oracle_solve.argtypes = [P, ctypes.c_int64, P, P, P, P, P, P, ctypes.c_int64, P, ctypes.c_int64,
                                     P, P, ctypes.c_int]
        lib.oracle_solve.restype = ctypes.c_int
        lib.oracle_system_k1.argtypes = [P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P, P]
        lib.oracle_system_k1.restype = ctypes.c_int
        lib.oracle_resultant.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int]
        lib.oracle_resultant.restype = ctypes.c_int
        lib.oracle_isolate.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double, P, P, ctypes.c_int]
        lib.oracle_isolate.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def solve(tri, x_first, x_last, eta, types, k, chains, n_threads: int = 0, capacity: int | None = None):
    """Solve every chain; returns (paths structured array, counters dict)."""
    lib = _load()
    tri = _c(tri, np.float64)
    x_first = _c(x_first, np.float64)
    x_last = _c(x_last, np.float64)
    eta = _c(eta, np.float64)
    types = _c(types, np.int32)
    k = _c(k, np.int32)
    chains = _c(chains, np.int32).reshape(-1, 3)
    if capacity is None:
        capacity = max(1024, 4 * chains.shape[0])
    while True:
        out = np.zeros(capacity, dtype=PATH_DTYPE)
        n_out = ctypes.c_int64(0)
        cnt = _Counters()
        rc = lib.oracle_solve(_ptr(tri), tri.shape[1], _ptr(x_first), _ptr(x_last), _ptr(eta), _ptr(types),
                              _ptr(k), _ptr(chains), chains.shape[0], _ptr(out), capacity,
                              ctypes.byref(n_out), ctypes.byref(cnt), int(n_threads))
        if rc == -1:
            capacity = int(n_out.value)
            continue
        if rc != 0:
            raise RuntimeError(f"oracle_solve failed with code {rc}")
        counters = {n: int(getattr(cnt, n)) for n, _ in _Counters._fields_}
        return out[: n_out.value].copy(), counters


def system_k1(tri18, x0, x2, type_, eta0=1.0, eta1=1.0):
    """Bivariate system of one candidate: (a grid [7,7], b grid [7,7], info dict)."""
    lib = _load()
    tri18 = _c(np.asarray(tri18).reshape(18), np.float64)
    a = np.zeros(49)
    b = np.zeros(49)
    info = np.zeros(6, dtype=np.int32)
    lib.oracle_system_k1(_ptr(tri18), _ptr(_c(x0, np.float64)), _ptr(_c(x2, np.float64)), int(type_),
                         float(eta0), float(eta1), _ptr(a), _ptr(b), _ptr(info))
    keys = ("total_deg_a", "total_deg_b", "deg_u_a", "deg_u_b", "edge", "b_axis")
    return a.reshape(7, 7), b.reshape(7, 7), dict(zip(keys, (int(x) for x in info)))


def resultant(a_grid, b_grid):
    """r(v) = det Bezout_u(a, b) for square coefficient grids; coefficients low to high."""
    lib = _load()
    a_grid = _c(a_grid, np.float64)
    b_grid = _c(b_grid, np.float64)
    dmax = a_grid.shape[0] - 1
    assert a_grid.shape == b_grid.shape == (dmax + 1, dmax + 1)
    cap = 4 * (dmax + 1) ** 2 + 8
    r = np.zeros(cap)
    n = lib.oracle_resultant(_ptr(a_grid), _ptr(b_grid), dmax, _ptr(r), cap)
    if n < 0:
        raise RuntimeError("resultant buffer too small")
    return r[:n].copy()


def isolate(p, lo, hi):
    """Real roots of sum p_i x^i on [lo, hi]; returns (roots, flags)."""
    lib = _load()
    p = _c(p, np.float64)
    cap = max(8, 2 * p.size)
    roots = np.zeros(cap)
    flags = np.zeros(cap, dtype=np.uint32)
    n = lib.oracle_isolate(_ptr(p), p.size, float(lo), float(hi), _ptr(roots), _ptr(flags), cap)
    if n < 0:
        raise RuntimeError("isolate buffer too small")
    return roots[:n].copy(), flags[:n].copy()
