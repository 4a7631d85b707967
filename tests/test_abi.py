"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/stokes.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stokes.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*[A-Za-z_][A-Za-z0-9_ \*]*?\b(stokes_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_1010_2832_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("stokes_create", "stokes_build_weights", "stokes_apply", "stokes_solve_step",
                     "stokes_destroy", "stokes_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1010_2832_gb300 import stokes
    assert set(declared_functions()) <= set(stokes.EXPORTED)


def test_argument_errors_without_gpu(lib):
    # stokes_create validates its arguments on the host before touching CUDA
    from paper_1010_2832_gb300 import stokes
    L = stokes.load_library()
    g = stokes.Grid()
    g.dim, g.nx, g.ny, g.nz, g.h, g.dt = 4, 8, 8, 0, 0.1, 0.1
    h = ctypes.c_void_p()
    assert L.stokes_create(ctypes.byref(h), ctypes.byref(g), None) == -1
    assert b"dim" in L.stokes_last_error(None)
    g.dim, g.h = 2, -1.0
    assert L.stokes_create(ctypes.byref(h), ctypes.byref(g), None) == -1
    assert L.stokes_destroy(None) == 0
