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


def documented_orders():
    src = open(os.path.join(ROOT, "include", "fmmpc.h")).read()
    m = re.search(r"p must be one of ([0-9, ]+)", src)
    assert m, "fmmpc.h must state the accepted expansion orders"
    return sorted(int(v) for v in m.group(1).replace(" ", "").strip(",").split(","))


def test_documented_expansion_orders_are_the_accepted_ones(lib):
    # every order fmmpc.h documents passes argument validation, every other one is rejected
    # with FMMPC_ERR_INVALID before any CUDA call (without a GPU an accepted order then fails
    # later with an allocation or CUDA error, never with _INVALID)
    from paper_1308_3339_gb300 import _lib
    orders = documented_orders()
    assert orders == [4, 6, 8, 10, 12, 16]
    g = _lib.Grid(64, 64, 0.0, 0.0, 1.0, 1.0)
    for p in range(0, 25):
        h = C.c_void_p()
        prm = _lib.Params(p, 64, 0.4, 1, 1, 0)
        rc = lib.fmmpc_create(C.byref(h), C.byref(g), C.byref(prm), None)
        if p in orders:
            assert rc != -1 or b"p must be one of" not in lib.fmmpc_last_error(None), p
            if rc == 0:
                lib.fmmpc_destroy(h)
        else:
            assert rc == -1 and b"p must be one of" in lib.fmmpc_last_error(None), p
