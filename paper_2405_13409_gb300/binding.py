"""Thin ctypes binding of libspoly (include/spoly.h).

Argument marshalling only: every step of the solve runs in the CUDA
library.  Functions keep the C names.  Device arrays are torch CUDA tensors
(PyTorch supplies device memory and streams); host arrays are numpy arrays.
There is no fallback: if the compiled library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libspoly.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "spoly.h")

SPOLY_OK = 0
SPOLY_EINVAL = -1
SPOLY_ENOMEM = -2
SPOLY_ECUDA = -3
SPOLY_ECAPACITY = -4
SPOLY_ETIMEOUT = -5
SPOLY_EUNSUPPORTED = -6

SPOLY_R = 0
SPOLY_T = 1

FLAG_ILL_COND = 1
FLAG_EDGE = 2
FLAG_BACKFACE = 4
FLAG_NEWTON = 8
FLAG_SQRT_SPLIT = 16
FLAG_TANGENT = 32
FLAG_OCCLUDED = 64

CHAINS_ALL = 0
CHAINS_CONE = 1
CHAINS_EXPLICIT = 2
CHAINS_FOOTPRINT = 3
CHAINS_EXPLICIT_CONE = 4
CHAINS_FOOTPRINT_UNIQUE = 5

PLAIN_FP64 = 0
MIXED = 1
SOLVE_ASYNC = 1
SOLVE_TIMING = 2
SOLVE_PERSISTENT = 4
SOLVE_GRAPH = 8
SOLVE_PIXEL_ASSIGN = 16
PEAK_FP32_FMA = 0
PEAK_FP64_FMA = 1
MLP_FEATURES = 24
MLP_PARAMS = 10497

c_void_p = ctypes.c_void_p
c_int32 = ctypes.c_int32
c_int64 = ctypes.c_int64


class spoly_mesh(ctypes.Structure):
    _fields_ = [("tri", c_void_p), ("n_tris", c_int64), ("on_device", c_int32), ("reserved", c_int32)]


class spoly_queries(ctypes.Structure):
    _fields_ = [("x_first", c_void_p), ("x_last", c_void_p), ("eta", c_void_p), ("types", c_void_p),
                ("k", c_void_p), ("n_queries", c_int64), ("on_device", c_int32), ("reserved", c_int32)]


class spoly_chain_opts(ctypes.Structure):
    _fields_ = [("mode", c_int32), ("second_begin", c_int32), ("tri_begin", c_int32), ("tri_end", c_int32),
                ("margin", ctypes.c_double), ("explicit_chains", c_void_p), ("n_explicit", c_int64),
                ("explicit_on_device", c_int32), ("second_end", c_int32), ("camera", c_void_p),
                ("cell", ctypes.c_double)]


class spoly_solve_opts(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("flags", c_int32), ("path_capacity", c_int64), ("camera", c_void_p),
                ("sqrt_table", c_void_p), ("n_intervals", c_int32), ("reserved3", c_int32)]


class spoly_path(ctypes.Structure):
    _fields_ = [("query", c_int32), ("tri", c_int32 * 2), ("chain", c_int32),
                ("uv", ctypes.c_double * 4), ("x", ctypes.c_double * 6),
                ("residual", ctypes.c_float), ("flags", ctypes.c_uint32)]


class spoly_counters(ctypes.Structure):
    _fields_ = [(n, c_int64) for n in ("candidates", "degenerate", "v_roots", "queued", "prefiltered",
                                       "polish_lost", "u_roots", "admissible", "flagged", "fallback",
                                       "unsolved", "k2_systems", "k2_evals", "k2_eval_n3", "k2_fp64_samples",
                                       "k2_evals32", "k2_eval32_n3")]


class spoly_tune_entry(ctypes.Structure):
    _fields_ = [("block", c_int32), ("blocks_per_sm", c_int32), ("chunk", c_int32), ("ms", ctypes.c_float)]


class spoly_mlp_train_opts(ctypes.Structure):
    _fields_ = [("steps", c_int64), ("batch", c_int32), ("lr", ctypes.c_float), ("lr_final", ctypes.c_float),
                ("pos_weight", ctypes.c_float), ("pos_fraction", ctypes.c_float), ("reserved", c_int32),
                ("seed", ctypes.c_uint64)]


PATH_DTYPE = np.dtype([("query", "<i4"), ("tri", "<i4", (2,)), ("chain", "<i4"), ("uv", "<f8", (4,)),
                       ("x", "<f8", (6,)), ("residual", "<f4"), ("flags", "<u4")])
assert PATH_DTYPE.itemsize == ctypes.sizeof(spoly_path) == 104

_lib = None


def header_functions() -> list[str]:
    """Names of the entry points declared in include/spoly.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:spoly_status|const char\*|void)\s+(spoly_\w+)\s*\(", text, re.M)))


def load():
    """Loads libspoly.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() (or "
                           "python paper_2405_13409_gb300/build.py) first; there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    P = c_void_p
    sig = {
        "spoly_version": ([], ctypes.c_char_p),
        "spoly_ctx_create": ([ctypes.c_int, P, ctypes.POINTER(P)], c_int32),
        "spoly_ctx_destroy": ([P], c_int32),
        "spoly_last_error": ([P], ctypes.c_char_p),
        "spoly_build_chains": ([P, ctypes.POINTER(spoly_mesh), ctypes.POINTER(spoly_queries),
                                ctypes.POINTER(spoly_chain_opts), ctypes.POINTER(P)], c_int32),
        "spoly_default_sqrt_table": ([P, c_int32], c_int32),
        "spoly_visibility": ([P, ctypes.POINTER(spoly_mesh), ctypes.POINTER(spoly_queries), P, ctypes.POINTER(c_int64)],
                             c_int32),
        "spoly_contributions": ([P, ctypes.POINTER(spoly_mesh), ctypes.POINTER(spoly_queries), P, ctypes.c_double, P, P,
                                 c_int64], c_int32),
        "spoly_upload": ([P, ctypes.POINTER(spoly_mesh), ctypes.POINTER(spoly_queries), ctypes.POINTER(spoly_mesh),
                          ctypes.POINTER(spoly_queries)], c_int32),
        "spoly_chains_count": ([P, ctypes.POINTER(c_int64)], c_int32),
        "spoly_chains_footprint_pairs": ([P, ctypes.POINTER(c_int64)], c_int32),
        "spoly_chains_copy": ([P, P, P, c_int64, ctypes.POINTER(c_int64), c_int32], c_int32),
        "spoly_chains_free": ([P], c_int32),
        "spoly_solve": ([P, ctypes.POINTER(spoly_mesh), ctypes.POINTER(spoly_queries), P,
                         ctypes.POINTER(spoly_solve_opts), ctypes.POINTER(P)], c_int32),
        "spoly_paths": ([P, P, P, c_int64, ctypes.POINTER(c_int64), c_int32], c_int32),
        "spoly_stats": ([P, P, ctypes.POINTER(spoly_counters)], c_int32),
        "spoly_solution_free": ([P], c_int32),
        "spoly_phase_ms": ([P, P, ctypes.POINTER(ctypes.c_float), c_int32], c_int32),
        "spoly_measure_peak": ([P, c_int32, ctypes.POINTER(ctypes.c_double)], c_int32),
        "spoly_solve_noalloc": ([ctypes.c_int, P, P, c_int64, P, P, P, P, P, c_int64, P, c_int64, c_int32, P,
                                 c_int64, ctypes.POINTER(c_int64), ctypes.c_char_p, c_int32], c_int32),
        "spoly_mlp_create": ([P, ctypes.c_uint64, ctypes.POINTER(P)], c_int32),
        "spoly_mlp_free": ([P], c_int32),
        "spoly_mlp_set_wait_limit": ([P, c_int64], c_int32),
        "spoly_mlp_get_params": ([P, P, P], c_int32),
        "spoly_mlp_set_params": ([P, P, P], c_int32),
        "spoly_mlp_save": ([P, P, ctypes.c_char_p], c_int32),
        "spoly_mlp_load": ([P, ctypes.c_char_p, ctypes.POINTER(P)], c_int32),
        "spoly_mlp_features": ([P, ctypes.POINTER(spoly_mesh), ctypes.POINTER(spoly_queries), P, P], c_int32),
        "spoly_chain_labels": ([P, P, c_int64, P], c_int32),
        "spoly_mlp_forward": ([P, P, P, c_int64, P], c_int32),
        "spoly_mlp_grad": ([P, P, P, P, c_int64, ctypes.c_float, P, ctypes.POINTER(ctypes.c_float)], c_int32),
        "spoly_mlp_train": ([P, P, P, P, c_int64, ctypes.POINTER(spoly_mlp_train_opts),
                             ctypes.POINTER(ctypes.c_float)], c_int32),
        "spoly_mlp_calibrate": ([P, P, P, P, c_int64, ctypes.c_double, ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_double)], c_int32),
        "spoly_gate": ([P, P, ctypes.POINTER(spoly_mesh), ctypes.POINTER(spoly_queries), P, ctypes.c_float,
                        ctypes.POINTER(P)], c_int32),
        "spoly_autotune": ([P, ctypes.POINTER(spoly_mesh), ctypes.POINTER(spoly_queries), P, c_int32,
                            ctypes.POINTER(spoly_tune_entry), c_int32, ctypes.POINTER(c_int32),
                            ctypes.POINTER(spoly_tune_entry)], c_int32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


class SpolyError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"spoly status {status}: {msg}")
        self.status = status


def _ptr(x) -> int:
    """Raw address of a numpy array or a torch tensor."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


def _on_device(x) -> int:
    return 0 if isinstance(x, np.ndarray) else int(x.is_cuda)


class Context:
    """Owns a spoly_ctx bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        h = c_void_p()
        st = self.lib.spoly_ctx_create(int(device), c_void_p(stream or 0), ctypes.byref(h))
        if st != SPOLY_OK:
            raise SpolyError(st, "spoly_ctx_create failed")
        self.h = h
        self._keep = []

    def check(self, st: int, what: str):
        if st != SPOLY_OK:
            raise SpolyError(st, f"{what}: {self.lib.spoly_last_error(self.h).decode()}")

    def close(self):
        if self.h:
            self.lib.spoly_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def mesh(tri) -> spoly_mesh:
        """A view of a [18, n_tris] FP64 array; the view holds a reference
        to the array, so the memory stays valid while the view lives."""
        m = spoly_mesh(_ptr(tri), int(tri.shape[1]), _on_device(tri), 0)
        m._owner = (tri,)
        return m

    @staticmethod
    def queries(x_first, x_last, eta, types, k) -> spoly_queries:
        """A view of the query arrays; like mesh(), it keeps them alive."""
        q = spoly_queries(_ptr(x_first), _ptr(x_last), _ptr(eta), _ptr(types), _ptr(k),
                          int(x_first.shape[0]), _on_device(x_first), 0)
        q._owner = (x_first, x_last, eta, types, k)
        return q

    def spoly_visibility(self, mesh: spoly_mesh, q: spoly_queries, sol) -> int:
        """Marks occluded paths of the solution set in place; returns the
        number of visible paths."""
        n = c_int64()
        self.check(self.lib.spoly_visibility(self.h, ctypes.byref(mesh), ctypes.byref(q), sol, ctypes.byref(n)),
                   "spoly_visibility")
        return int(n.value)

    def spoly_contributions(self, mesh: spoly_mesh, q: spoly_queries, sol, intensity: float = 1.0, per_path=None,
                            image=None):
        """per_path / image: device FP64 tensors (or None)."""
        self.check(self.lib.spoly_contributions(self.h, ctypes.byref(mesh), ctypes.byref(q), sol, float(intensity),
                                                c_void_p(_ptr(per_path)) if per_path is not None else None,
                                                c_void_p(_ptr(image)) if image is not None else None,
                                                int(image.numel()) if image is not None else 0),
                   "spoly_contributions")

    def spoly_upload(self, mesh: spoly_mesh, q: spoly_queries):
        """Host inputs staged into the context's device buffers; returns
        device views (spoly_mesh, spoly_queries) for the calls that follow."""
        mo, qo = spoly_mesh(), spoly_queries()
        self.check(self.lib.spoly_upload(self.h, ctypes.byref(mesh), ctypes.byref(q), ctypes.byref(mo),
                                         ctypes.byref(qo)), "spoly_upload")
        return mo, qo

    def spoly_build_chains(self, mesh: spoly_mesh, q: spoly_queries, mode: int, margin: float = 1e-3,
                           explicit=None, tri_range=(0, 0), reuse=None, camera=None, cell: float = 0.0,
                           second_range=(0, 0)):
        cam = None if camera is None else np.ascontiguousarray(camera, dtype=np.float64)
        opts = spoly_chain_opts(mode, int(second_range[0]), int(tri_range[0]), int(tri_range[1]), float(margin),
                                _ptr(explicit) if explicit is not None else 0,
                                int(explicit.shape[0]) if explicit is not None else 0,
                                _on_device(explicit) if explicit is not None else 0, int(second_range[1]),
                                cam.ctypes.data if cam is not None else None, float(cell))
        h = c_void_p(reuse.value if reuse is not None else None)
        self.check(self.lib.spoly_build_chains(self.h, ctypes.byref(mesh), ctypes.byref(q), ctypes.byref(opts),
                                               ctypes.byref(h)), "spoly_build_chains")
        return h

    def spoly_chains_count(self, chains) -> int:
        n = c_int64()
        self.check(self.lib.spoly_chains_count(chains, ctypes.byref(n)), "spoly_chains_count")
        return int(n.value)

    def spoly_chains_footprint_pairs(self, chains) -> int:
        n = c_int64()
        self.check(self.lib.spoly_chains_footprint_pairs(chains, ctypes.byref(n)), "spoly_chains_footprint_pairs")
        return int(n.value)

    def spoly_chains_copy(self, chains) -> np.ndarray:
        n = self.spoly_chains_count(chains)
        out = np.zeros((n, 3), dtype=np.int32)
        tot = c_int64()
        self.check(self.lib.spoly_chains_copy(self.h, chains, c_void_p(out.ctypes.data), n, ctypes.byref(tot), 0),
                   "spoly_chains_copy")
        return out

    def spoly_chains_free(self, chains):
        self.lib.spoly_chains_free(chains)

    def spoly_solve(self, mesh: spoly_mesh, q: spoly_queries, chains, precision: int = MIXED, flags: int = 0,
                    path_capacity: int = 0, reuse=None, camera=None, sqrt_table=None, n_intervals: int = 0):
        """sqrt_table: optional (breaks[7], coeffs[6][3]) of the 2-bounce
        refraction mapping; None uses the library's default."""
        cam = None if camera is None else np.ascontiguousarray(camera, dtype=np.float64)
        tab = None
        if sqrt_table is not None:
            breaks, coeffs = sqrt_table
            tab = np.ascontiguousarray(np.concatenate([np.asarray(breaks, np.float64).ravel(),
                                                       np.asarray(coeffs, np.float64).ravel()]))
            assert tab.size == 25
        opts = spoly_solve_opts(int(precision), int(flags), int(path_capacity),
                                cam.ctypes.data if cam is not None else None,
                                tab.ctypes.data if tab is not None else None, int(n_intervals), 0)
        h = c_void_p(reuse.value if reuse is not None else None)
        self.check(self.lib.spoly_solve(self.h, ctypes.byref(mesh), ctypes.byref(q), chains, ctypes.byref(opts),
                                        ctypes.byref(h)), "spoly_solve")
        return h

    def spoly_paths(self, sol) -> np.ndarray:
        """All paths of a solution set as a PATH_DTYPE array (host)."""
        tot = c_int64()
        st = self.lib.spoly_paths(self.h, sol, None, 0, ctypes.byref(tot), 0)
        if st not in (SPOLY_OK, SPOLY_ECAPACITY) or (st == SPOLY_ECAPACITY and tot.value == 0):
            self.check(st, "spoly_paths")
        out = np.zeros(int(tot.value), dtype=PATH_DTYPE)
        if tot.value:
            self.check(self.lib.spoly_paths(self.h, sol, c_void_p(out.ctypes.data), int(tot.value),
                                            ctypes.byref(tot), 0), "spoly_paths")
        return out

    def spoly_paths_into(self, sol, dst, capacity: int) -> int:
        """Copies up to `capacity` paths into a host or device buffer; returns the count."""
        tot = c_int64()
        st = self.lib.spoly_paths(self.h, sol, c_void_p(_ptr(dst)), int(capacity), ctypes.byref(tot),
                                  _on_device(dst))
        if st != SPOLY_ECAPACITY:
            self.check(st, "spoly_paths")
        return int(tot.value)

    def spoly_stats(self, sol) -> dict:
        c = spoly_counters()
        self.check(self.lib.spoly_stats(self.h, sol, ctypes.byref(c)), "spoly_stats")
        return {n: int(getattr(c, n)) for n, _ in spoly_counters._fields_ if n != "reserved"}

    def spoly_solution_free(self, sol):
        self.lib.spoly_solution_free(sol)

    def spoly_phase_ms(self, sol) -> tuple:
        """(1-bounce isolation, 1-bounce polish + paths, 2-bounce pipeline,
        2-bounce sign passes) in ms."""
        ms = (ctypes.c_float * 4)()
        self.check(self.lib.spoly_phase_ms(self.h, sol, ms, 4), "spoly_phase_ms")
        return float(ms[0]), float(ms[1]), float(ms[2]), float(ms[3])

    def spoly_measure_peak(self, kind: int) -> float:
        t = ctypes.c_double()
        self.check(self.lib.spoly_measure_peak(self.h, int(kind), ctypes.byref(t)), "spoly_measure_peak")
        return float(t.value)

    def spoly_autotune(self, mesh: spoly_mesh, q: spoly_queries, chains, precision: int = MIXED):
        """Times the persistent isolation kernel's launch shapes on `chains`
        and keeps the fastest in the context.  Returns (best, table)."""
        tab = (spoly_tune_entry * 64)()
        n = c_int32()
        best = spoly_tune_entry()
        self.check(self.lib.spoly_autotune(self.h, ctypes.byref(mesh), ctypes.byref(q), chains, int(precision), tab, 64,
                                           ctypes.byref(n), ctypes.byref(best)), "spoly_autotune")
        rows = [(t.block, t.blocks_per_sm, t.chunk, float(t.ms)) for t in tab[:n.value]]
        return (best.block, best.blocks_per_sm, best.chunk, float(best.ms)), rows

    # ------------------------------------------------------------ gate
    def spoly_mlp_create(self, seed: int = 0):
        h = c_void_p()
        self.check(self.lib.spoly_mlp_create(self.h, int(seed), ctypes.byref(h)), "spoly_mlp_create")
        return h

    def spoly_mlp_free(self, mlp):
        self.lib.spoly_mlp_free(mlp)

    def spoly_mlp_set_wait_limit(self, mlp, cycles: int):
        st = self.lib.spoly_mlp_set_wait_limit(mlp, int(cycles))
        if st != SPOLY_OK:
            raise SpolyError(st, "spoly_mlp_set_wait_limit: bad arguments")

    def spoly_mlp_get_params(self, mlp) -> np.ndarray:
        out = np.zeros(MLP_PARAMS, dtype=np.float32)
        self.check(self.lib.spoly_mlp_get_params(self.h, mlp, c_void_p(out.ctypes.data)), "spoly_mlp_get_params")
        return out

    def spoly_mlp_set_params(self, mlp, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        assert t.shape == (MLP_PARAMS,)
        self.check(self.lib.spoly_mlp_set_params(self.h, mlp, c_void_p(t.ctypes.data)), "spoly_mlp_set_params")

    def spoly_mlp_save(self, mlp, path: str):
        self.check(self.lib.spoly_mlp_save(self.h, mlp, os.fsencode(path)), "spoly_mlp_save")

    def spoly_mlp_load(self, path: str):
        h = c_void_p()
        self.check(self.lib.spoly_mlp_load(self.h, os.fsencode(path), ctypes.byref(h)), "spoly_mlp_load")
        return h

    def spoly_mlp_features(self, mesh: spoly_mesh, q: spoly_queries, chains, dst):
        """Features of a chain list into a device FP32 tensor [n][24]."""
        self.check(self.lib.spoly_mlp_features(self.h, ctypes.byref(mesh), ctypes.byref(q), chains,
                                               c_void_p(_ptr(dst))), "spoly_mlp_features")

    def spoly_chain_labels(self, sol, n_chains: int, dst):
        self.check(self.lib.spoly_chain_labels(self.h, sol, int(n_chains), c_void_p(_ptr(dst))),
                   "spoly_chain_labels")

    def spoly_mlp_forward(self, mlp, feat, logits):
        self.check(self.lib.spoly_mlp_forward(self.h, mlp, c_void_p(_ptr(feat)), int(feat.shape[0]),
                                              c_void_p(_ptr(logits))), "spoly_mlp_forward")

    def spoly_mlp_grad(self, mlp, feat, labels, pos_weight: float):
        g = np.zeros(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        self.check(self.lib.spoly_mlp_grad(self.h, mlp, c_void_p(_ptr(feat)), c_void_p(_ptr(labels)),
                                           int(feat.shape[0]), float(pos_weight), c_void_p(g.ctypes.data),
                                           ctypes.byref(loss)), "spoly_mlp_grad")
        return float(loss.value), g

    def spoly_mlp_train(self, mlp, feat, labels, steps: int, batch: int = 4096, lr: float = 2e-3,
                        lr_final: float = 2e-4, pos_weight: float = 1.0, pos_fraction: float = 0.25, seed: int = 0):
        o = spoly_mlp_train_opts(int(steps), int(batch), float(lr), float(lr_final), float(pos_weight),
                                 float(pos_fraction), 0, int(seed))
        loss = ctypes.c_float()
        self.check(self.lib.spoly_mlp_train(self.h, mlp, c_void_p(_ptr(feat)), c_void_p(_ptr(labels)),
                                            int(feat.shape[0]), ctypes.byref(o), ctypes.byref(loss)),
                   "spoly_mlp_train")
        return float(loss.value)

    def spoly_mlp_calibrate(self, mlp, feat, labels, target_recall: float):
        tau = ctypes.c_float()
        frac = ctypes.c_double()
        self.check(self.lib.spoly_mlp_calibrate(self.h, mlp, c_void_p(_ptr(feat)), c_void_p(_ptr(labels)),
                                                int(feat.shape[0]), float(target_recall), ctypes.byref(tau),
                                                ctypes.byref(frac)), "spoly_mlp_calibrate")
        return float(tau.value), float(frac.value)

    def spoly_gate(self, mlp, mesh: spoly_mesh, q: spoly_queries, chains, tau_logit: float, reuse=None):
        h = c_void_p(reuse.value if reuse is not None else None)
        self.check(self.lib.spoly_gate(self.h, mlp, ctypes.byref(mesh), ctypes.byref(q), chains, float(tau_logit),
                                       ctypes.byref(h)), "spoly_gate")
        return h


def spoly_default_sqrt_table():
    """The library's default sqrt pieces as (breaks[7], coeffs[6][3])."""
    lib = load()
    t = np.zeros(25)
    st = lib.spoly_default_sqrt_table(c_void_p(t.ctypes.data), 25)
    if st != SPOLY_OK:
        raise SpolyError(st, "spoly_default_sqrt_table")
    return t[:7].copy(), t[7:].reshape(6, 3).copy()


def spoly_solve_noalloc(device: int, stream, tri, x_first, x_last, eta, types, k, chains, precision: int, paths,
                        path_capacity: int):
    """Calls the no-allocation solve on device tensors.  Returns (status,
    n_paths, message); the paths land in the caller's device buffer."""
    lib = load()
    n = c_int64(0)
    msg = ctypes.create_string_buffer(256)
    st = lib.spoly_solve_noalloc(int(device), c_void_p(stream or 0), _ptr(tri), int(tri.shape[1]), _ptr(x_first),
                                 _ptr(x_last), _ptr(eta), _ptr(types), _ptr(k), int(x_first.shape[0]),
                                 _ptr(chains), int(chains.shape[0]), int(precision), _ptr(paths),
                                 int(path_capacity), ctypes.byref(n), msg, 256)
    return int(st), int(n.value), msg.value.decode()
