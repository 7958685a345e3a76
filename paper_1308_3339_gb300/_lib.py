"""ctypes view of the C ABI in include/fmmpc.h (argument marshalling only).

There is no CPU fallback: if the compiled library is missing the import of any
compute entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import lib_path

OK = 0
ERRORS = {-1: "INVALID", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED", -5: "NAN", -6: "TIMEOUT",
          -7: "UNSUPPORTED"}
PREC = {"fp64": 0, "fp32": 1, "mixed_bf16": 2, "mixed_tf32": 3}
METHOD = {"cg": 0, "gmres": 1, "fgmres": 2}
PART = {"full": 0, "vr": 1, "near": 2, "vcol": 3, "q": 4}
OPERATOR = {"fd5": 0, "fd5_var": 1, "q1": 2}
QUERY = {"L": 0, "leaf_side": 1, "n_m2l": 2, "n_p2p": 3, "n_m2l_vb": 4, "n_p2p_vb": 5, "NG": 6,
         "n_cell": 7, "N": 8, "stencil": 9, "launches": 10, "device_bytes": 11, "device_errors": 12,
         "tc_p2p": 13, "tc_m2l": 14}
STAGES = ["weights", "upward", "colloc", "bem", "bnd_upward", "m2l", "m2l_bnd", "l2l", "bnd_near", "p2p", "l2p"]
EXPORT = {"keys": 0, "perm": 1, "cell_start": 2, "m2l": 3, "p2p": 4, "m2l_vb": 5, "p2p_vb": 6}


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("x0", C.c_double), ("y0", C.c_double),
                ("x1", C.c_double), ("y1", C.c_double)]


class Params(C.Structure):
    _fields_ = [("p", C.c_int32), ("leaf_max", C.c_int32), ("theta", C.c_double),
                ("precision", C.c_int32), ("n_rhs", C.c_int32), ("autotune", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("method", C.c_int32), ("restart", C.c_int32), ("maxit", C.c_int32),
                ("rtol", C.c_double), ("use_graphs", C.c_int32)]


class TuneEntry(C.Structure):
    _fields_ = [("leaf_max", C.c_int32), ("p", C.c_int32), ("rel_err", C.c_double),
                ("solve_ms", C.c_double), ("iters", C.c_int32), ("ok", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("rel_res", C.c_double), ("t_setup_ms", C.c_double),
                ("t_solve_ms", C.c_double), ("status", C.c_int32)]


_LIB = None

# name -> (restype, argtypes); every function declared in include/fmmpc.h
SIGNATURES = {
    "fmmpc_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Grid), C.POINTER(Params), C.c_void_p]),
    "fmmpc_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "fmmpc_apply_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "fmmpc_apply_part": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32]),
    "fmmpc_spmv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "fmmpc_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                              C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    "fmmpc_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                   C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
    "fmmpc_query": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]),
    "fmmpc_export": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64]),
    "fmmpc_set_graphs": (C.c_int, [C.c_void_p, C.c_int32]),
    "fmmpc_set_operator": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "fmmpc_apply_bc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "fmmpc_set_bem_form": (C.c_int, [C.c_void_p, C.c_int32]),
    "fmmpc_apply_transpose": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "fmmpc_set_p2p_engine": (C.c_int, [C.c_void_p, C.c_int32]),
    "fmmpc_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "fmmpc_get_timing": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.c_int32, C.POINTER(C.c_int32)]),
    "fmmpc_near_field_noalloc": (C.c_int, [C.c_int32, C.c_double, C.c_int32, C.c_double, C.c_void_p,
                                           C.c_void_p, C.c_void_p]),
    "fmmpc_destroy": (None, [C.c_void_p]),
    "fmmpc_autotune": (C.c_int, [C.POINTER(Grid), C.POINTER(Params), C.POINTER(SolveOpts), C.c_void_p,
                                 C.c_double, C.c_void_p, C.POINTER(Params), C.c_void_p, C.c_int32,
                                 C.POINTER(C.c_int32)]),
    "fmmpc_create_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_void_p, C.POINTER(Params), C.c_void_p]),
    "fmmpc_solve_batched": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveOpts),
                                      C.c_void_p]),
    "fmmpc_batch_query": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_int64)]),
    "fmmpc_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "fmmpc_destroy_batched": (None, [C.c_void_p]),
    "fmmpc_last_error": (C.c_char_p, [C.c_void_p]),
    "fmmpc_version": (C.c_char_p, []),
}


def load(path: str | None = None):
    """Load libfmmpc; raise if it has not been built (no fallback path exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libfmmpc not found at {path}; build it with "
                           "paper_1308_3339_gb300.build.build() -- there is no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class FmmpcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fmmpc error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


def check(rc: int, handle=None):
    if rc != OK:
        msg = load().fmmpc_last_error(handle)
        raise FmmpcError(rc, msg.decode() if msg else "")
