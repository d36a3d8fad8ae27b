"""C-ABI checks that need no GPU: the library loads, exports every entry
point include/spoly.h declares, and its struct layouts match the binding."""
import ctypes
import os
import subprocess
import tempfile

import pytest

from paper_2405_13409_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build_library()
    return binding.load()


def test_header_declares_the_boundary():
    names = binding.header_functions()
    for n in ("spoly_ctx_create", "spoly_build_chains", "spoly_solve", "spoly_paths", "spoly_stats"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in binding.header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "spoly.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(spoly_mesh), sizeof(spoly_queries), sizeof(spoly_chain_opts),
         sizeof(spoly_solve_opts), sizeof(spoly_path), sizeof(spoly_counters));
  printf("%zu %zu %zu\n", offsetof(spoly_path, uv), offsetof(spoly_path, residual), offsetof(spoly_path, flags));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(x) for x in out]
    expect = [ctypes.sizeof(binding.spoly_mesh), ctypes.sizeof(binding.spoly_queries),
              ctypes.sizeof(binding.spoly_chain_opts), ctypes.sizeof(binding.spoly_solve_opts),
              ctypes.sizeof(binding.spoly_path), ctypes.sizeof(binding.spoly_counters),
              binding.spoly_path.uv.offset, binding.spoly_path.residual.offset, binding.spoly_path.flags.offset]
    assert sizes == expect


def test_version_string(lib):
    assert b"sm_103a" in lib.spoly_version()


def test_null_arguments_are_rejected_without_a_device(lib):
    assert lib.spoly_ctx_create(0, None, None) == binding.SPOLY_EINVAL
    assert lib.spoly_ctx_destroy(None) == binding.SPOLY_EINVAL
    assert lib.spoly_chains_free(None) == binding.SPOLY_EINVAL
    assert lib.spoly_solution_free(None) == binding.SPOLY_EINVAL


def test_ctx_create_reports_missing_device(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.spoly_ctx_create(0, None, ctypes.byref(h)) == binding.SPOLY_ECUDA
    assert not h.value


def test_views_keep_their_arrays_alive():
    """A mesh or query view built from temporaries must not dangle: the view
    holds the arrays its pointers name."""
    import gc
    import weakref

    import numpy as np

    def make():
        tri = np.zeros((18, 4))
        xs = [np.zeros((2, 3)), np.zeros((2, 3)), np.ones((2, 3)), np.zeros((2, 2), np.int32), np.ones(2, np.int32)]
        refs = [weakref.ref(a) for a in [tri] + xs]
        return binding.Context.mesh(tri), binding.Context.queries(*xs), refs

    m, q, refs = make()
    gc.collect()
    assert all(r() is not None for r in refs)
    assert m.tri == refs[0]().ctypes.data and q.x_first == refs[1]().ctypes.data
    del m, q
    gc.collect()
    assert all(r() is None for r in refs)
