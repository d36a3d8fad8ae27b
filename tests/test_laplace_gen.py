"""The generated straight-line Laplace expansions (kernel code) compiled on
the host with g++ and checked against numpy determinants of the symmetric
polynomial matrices they expand (Sec. 4.2), plus a check that the committed
header is what the generator writes."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2405_13409_gb300", "csrc")
CONFIGS = [("R2", 2, 5), ("R3", 3, 5), ("R4", 4, 5), ("T2", 2, 7), ("T3", 3, 7), ("T4", 4, 7), ("T5", 5, 7),
           ("T6", 6, 7)]


def _packing(N, ED):
    offs, o = {}, 0
    for i in range(N):
        for j in range(i, N):
            offs[(i, j)] = o
            if ED - i - j >= 0:
                o += ED - i - j + 1
    return offs, o


@pytest.fixture(scope="module")
def glib():
    text = open(os.path.join(CSRC, "laplace_gen.cuh")).read()
    text = text.replace('#include "common.cuh"', "#include <cmath>\nusing std::fma;").replace("SPOLY_D", "inline")
    wrappers = []
    for name, N, ED in CONFIGS:
        _, sym = _packing(N, ED)
        rd = N * (ED - N + 1)
        wrappers.append(f'extern "C" void lap_{name}(const double* e, double* r) {{ double E[{sym}]; double R[{rd + 1}];'
                        f' for (int i = 0; i < {sym}; ++i) E[i] = e[i]; spoly::laplace_{name}<double>(E, R);'
                        f' for (int i = 0; i <= {rd}; ++i) r[i] = R[i]; }}')
        wrappers.append(f'extern "C" void labs_{name}(const double* e, double* r) {{ double E[{sym}]; double R[{rd + 1}];'
                        f' for (int i = 0; i < {sym}; ++i) E[i] = e[i]; spoly::laplace_abs_{name}<double>(E, R);'
                        f' for (int i = 0; i <= {rd}; ++i) r[i] = R[i]; }}')
    d = tempfile.mkdtemp()
    src = os.path.join(d, "lap.cpp")
    so = os.path.join(d, "lap.so")
    open(src, "w").write(text.replace("#pragma once", "") + "\n" + "\n".join(wrappers) + "\n")
    subprocess.run(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", src, "-o", so], check=True)
    return ctypes.CDLL(so)


@pytest.mark.parametrize("name,N,ED", CONFIGS)
def test_generated_laplace_equals_determinant(glib, name, N, ED):
    rng = np.random.default_rng(N * 10 + ED)
    offs, sym = _packing(N, ED)
    rd = N * (ED - N + 1)
    fn = getattr(glib, f"lap_{name}")
    for _ in range(20):
        e = rng.normal(size=sym)
        r = np.zeros(rd + 1)
        fn(e.ctypes.data_as(ctypes.c_void_p), r.ctypes.data_as(ctypes.c_void_p))
        for z in rng.uniform(-1.5, 1.5, 5):
            M = np.zeros((N, N))
            for i in range(N):
                for j in range(N):
                    a, b = min(i, j), max(i, j)
                    d = ED - a - b
                    if d >= 0:
                        M[i, j] = np.polyval(e[offs[(a, b)]:offs[(a, b)] + d + 1][::-1], z)
            want = np.linalg.det(M)
            got = np.polyval(r[::-1], z)
            scale = np.prod(np.abs(M).sum(axis=1))
            assert abs(got - want) <= 1e-10 * scale, (name, z, got, want)


def test_committed_header_matches_generator():
    import importlib.util
    spec = importlib.util.spec_from_file_location("gen_laplace", os.path.join(CSRC, "gen_laplace.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    want = "// Generated by gen_laplace.py: straight-line memoised Laplace expansions of"
    text = open(os.path.join(CSRC, "laplace_gen.cuh")).read()
    assert text.startswith(want)
    for name, N, ED in mod.CONFIGS:
        assert mod.generate(name, N, ED) in text
        assert mod.generate(name, N, ED, absolute=True) in text


@pytest.mark.parametrize("name,N,ED", CONFIGS)
def test_absolute_expansion_is_the_permanent(glib, name, N, ED):
    """The expansion over |E| with every sign made positive is, by
    definition, the permanent of the matrix of |E| polynomials: the sum over
    all permutations of the products of entries, computed here by brute
    force with numpy polynomial products."""
    import itertools
    rng = np.random.default_rng(N * 31 + ED)
    offs, sym = _packing(N, ED)
    rd = N * (ED - N + 1)
    fn = getattr(glib, f"labs_{name}")
    for _ in range(5):
        e = np.abs(rng.normal(size=sym))
        r = np.zeros(rd + 1)
        fn(e.ctypes.data_as(ctypes.c_void_p), r.ctypes.data_as(ctypes.c_void_p))

        def entry(i, j):
            a, b = min(i, j), max(i, j)
            d = ED - a - b
            return e[offs[(a, b)]:offs[(a, b)] + d + 1] if d >= 0 else None

        perm = np.zeros(rd + 1)
        for sigma in itertools.permutations(range(N)):
            prod = np.ones(1)
            for i in range(N):
                p = entry(i, sigma[i])
                if p is None:
                    prod = None
                    break
                prod = np.polynomial.polynomial.polymul(prod, p)
            if prod is not None:
                perm[:prod.size] += prod
        assert np.allclose(r, perm, rtol=1e-12, atol=0), (name, r, perm)
