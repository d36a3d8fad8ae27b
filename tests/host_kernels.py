"""ctypes loader of tests/host_k1.cpp: the CUDA path's per-candidate device
functions compiled for the host with g++ (test infrastructure only)."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "host_k1.cpp")
CSRC = os.path.join(ROOT, "paper_2405_13409_gb300", "csrc")
_lib = None


def load(csrc: str = CSRC):
    global _lib
    if _lib is None or csrc != CSRC:
        d = tempfile.mkdtemp(prefix="spoly_host_")
        so = os.path.join(d, "host_k1.so")
        subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-I", csrc,
                        "-I", os.path.join(ROOT, "include"), SRC, "-o", so], check=True)
        lib = ctypes.CDLL(so)
        P = ctypes.c_void_p
        lib.host_k1_candidate.argtypes = [P, P, P, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                          P, ctypes.c_int, P]
        lib.host_k1_candidate.restype = ctypes.c_int
        if csrc != CSRC:
            return lib
        _lib = lib
    return _lib


def candidate(tri18, x0, x2, type_, eta0=1.0, eta1=1.0, precision=1, lib=None):
    """Returns (paths [n, 3] of (u, v, flags), status [8])."""
    lib = lib or load()
    t = np.ascontiguousarray(np.asarray(tri18, dtype=np.float64).reshape(18))
    a = np.ascontiguousarray(x0, dtype=np.float64)
    b = np.ascontiguousarray(x2, dtype=np.float64)
    out = np.zeros((64, 3))
    st = np.zeros(8, dtype=np.int32)
    n = lib.host_k1_candidate(t.ctypes.data, a.ctypes.data, b.ctypes.data, int(type_), float(eta0), float(eta1),
                              int(precision), out.ctypes.data, 64, st.ctypes.data)
    return out[:n].copy(), st
