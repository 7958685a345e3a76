"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and exports
every function that include/fmmpc.h declares; argument errors come back as codes."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fmmpc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fmmpc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1308_3339_gb300 import build
    build.build()
    from paper_1308_3339_gb300 import _lib
    return _lib.load()


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_every_declared_symbol():
    from paper_1308_3339_gb300 import _lib
    assert set(declared_functions()) == set(_lib.SIGNATURES)


def test_version_string(lib):
    assert lib.fmmpc_version().decode().startswith("fmmpc")


def test_create_rejects_bad_arguments_without_touching_a_gpu(lib):
    from paper_1308_3339_gb300 import _lib
    h = C.c_void_p()
    # non-square grid and p outside the supported set are rejected before any CUDA call
    g = _lib.Grid(64, 32, 0.0, 0.0, 1.0, 1.0)
    prm = _lib.Params(10, 64, 0.4, 1, 1, 0)
    assert lib.fmmpc_create(C.byref(h), C.byref(g), C.byref(prm), None) == -1
    assert b"nx must equal ny" in lib.fmmpc_last_error(None)
    g = _lib.Grid(64, 64, 0.0, 0.0, 1.0, 1.0)
    prm = _lib.Params(7, 64, 0.4, 1, 1, 0)
    assert lib.fmmpc_create(C.byref(h), C.byref(g), C.byref(prm), None) == -1
    prm = _lib.Params(10, 64, 1.5, 1, 1, 0)
    assert lib.fmmpc_create(C.byref(h), C.byref(g), C.byref(prm), None) == -1
    g = _lib.Grid(96, 96, 0.0, 0.0, 1.0, 1.0)  # leaf side 6 is not supported
    prm = _lib.Params(10, 64, 0.4, 1, 1, 0)
    assert lib.fmmpc_create(C.byref(h), C.byref(g), C.byref(prm), None) == -1
    assert lib.fmmpc_apply(None, None, None, 1) == -1
    lib.fmmpc_destroy(None)
