"""GB300-native FMM-BEM preconditioner for finite-difference Poisson systems.

Method: Ibeid, Yokota, Pestana and Keyes, "Fast Multipole Preconditioners for Sparse
Matrices Arising from Elliptic Equations" (arXiv:1308.3339).  All arithmetic runs in the
CUDA library ``libfmmpc`` (C ABI in ``include/fmmpc.h``); this module marshals torch CUDA
tensors (device memory, current stream) into its calls.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import FmmpcError, check

__all__ = ["FmmPreconditioner", "FmmBatch", "FmmpcError", "autotune", "version"]


def version() -> str:
    return _lib.load().fmmpc_version().decode()


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class FmmPreconditioner:
    """One grid: tree, interaction lists, BEM inverse and workspace (fmmpc_create).

    Vectors are torch float64 CUDA tensors shaped [n_rhs, n, n] or [n, n] in natural
    order (x fastest).  The handle is bound to the torch stream current at construction.
    """

    def __init__(self, n: int, p: int = 10, leaf_max: int = 64, theta: float = 0.4,
                 precision: str = "fp32", n_rhs: int = 1, x0: float = 0.0, y0: float = 0.0,
                 side: float = 1.0, stream=None):
        import torch
        self.lib = _lib.load()
        self.n, self.p, self.n_rhs_max = n, p, n_rhs
        self.x0, self.y0, self.side = x0, y0, side
        self.h = side / (n + 1)
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        g = _lib.Grid(n, n, x0, y0, x0 + side, y0 + side)
        prm = _lib.Params(p, leaf_max, theta, _lib.PREC[precision], n_rhs, 0)
        h = C.c_void_p()
        rc = self.lib.fmmpc_create(C.byref(h), C.byref(g), C.byref(prm), C.c_void_p(self.stream.cuda_stream))
        check(rc, None)
        self._h = h

    # ------------------------------------------------------------------ helpers
    def _vec(self, t, nrhs=None):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError("expected a contiguous float64 CUDA tensor")
        k = t.numel() // (self.n * self.n)
        if k * self.n * self.n != t.numel():
            raise ValueError("tensor size is not a multiple of n*n")
        return k

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fmmpc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, what: str) -> int:
        v = C.c_int64()
        check(self.lib.fmmpc_query(self._h, _lib.QUERY[what], C.byref(v)), self._h)
        return v.value

    def export(self, what: str) -> np.ndarray:
        sizes = {"keys": ("N", 1), "perm": ("N", 1), "cell_start": ("n_cell", 1), "m2l": ("n_m2l", 3),
                 "p2p": ("n_p2p", 2), "m2l_vb": ("n_m2l_vb", 3), "p2p_vb": ("n_p2p_vb", 2)}
        cnt, w = sizes[what]
        n = self.query(cnt)
        a = np.empty((n, w) if w > 1 else (n,), np.uint32 if what == "keys" else np.int32)
        check(self.lib.fmmpc_export(self._h, _lib.EXPORT[what], a.ctypes.data_as(C.c_void_p), a.nbytes), self._h)
        return a

    def set_p2p_engine(self, engine: str = "tc"):
        """Near-field engine: "tc" (tensor cores where the grid allows it) or "simt"."""
        check(self.lib.fmmpc_set_p2p_engine(self._h, {"tc": 0, "simt": 1}[engine]), self._h)

    def set_operator(self, op: str = "fd5", a=None):
        """Operator of the solves (fmmpc_set_operator): "fd5", "fd5_var" with the diffusion
        coefficient a (float64 CUDA tensor of (n+2)^2 full-grid node values), or "q1"."""
        ap = C.c_void_p(0) if a is None else _ptr(a)
        check(self.lib.fmmpc_set_operator(self._h, _lib.OPERATOR[op], ap), self._h)

    def set_bem_form(self, form: str = "single_layer"):
        """Boundary correction: "single_layer" (Eq. e:ubound, the default) or "double_layer"
        (second kind, (-1/2 I + K) mu = -(V r)|_Gamma)."""
        check(self.lib.fmmpc_set_bem_form(self._h, {"single_layer": 0, "double_layer": 1}[form]), self._h)

    def apply_transpose(self, zb, out=None):
        """rb = P^{-T} zb (fmmpc_apply_transpose): the FMM-transpose pass."""
        import torch
        k = self._vec(zb)
        out = torch.empty_like(zb) if out is None else out
        check(self.lib.fmmpc_apply_transpose(self._h, _ptr(zb), _ptr(out), k), self._h)
        return out

    def apply_bc(self, f, g, out=None):
        """u from Eqs. e:ubound / e:uinter with Dirichlet data g at the 4n element midpoints."""
        import torch
        k = self._vec(f)
        out = torch.empty_like(f) if out is None else out
        check(self.lib.fmmpc_apply_bc(self._h, _ptr(f), _ptr(g), _ptr(out), k), self._h)
        return out

    def set_graphs(self, on: bool = True):
        check(self.lib.fmmpc_set_graphs(self._h, 1 if on else 0), self._h)

    def set_timing(self, on=True):
        """True / 1: every stage; 2: only the M2L and P2P kernels; False / 0: off."""
        mode = 0 if on is False else (1 if on is True else int(on))
        check(self.lib.fmmpc_set_timing(self._h, mode), self._h)

    def stage_times(self) -> dict:
        """Stage durations (ms) of the last apply, from CUDA events on the handle stream."""
        buf = (C.c_float * 16)()
        cnt = C.c_int32()
        check(self.lib.fmmpc_get_timing(self._h, buf, 16, C.byref(cnt)), self._h)
        return {name: float(buf[i]) for i, name in enumerate(_lib.STAGES[: cnt.value])}

    # ------------------------------------------------------------------ compute
    def apply(self, r, out=None):
        """z = P^{-1} r (fmmpc_apply)."""
        import torch
        k = self._vec(r)
        out = torch.empty_like(r) if out is None else out
        check(self.lib.fmmpc_apply(self._h, _ptr(r), _ptr(out), k), self._h)
        return out

    def apply_part(self, part: str, r):
        import torch
        k = self._vec(r)
        if part in ("vcol", "q"):
            out = torch.empty((k, 4 * self.n), dtype=torch.float64, device=r.device)
        else:
            out = torch.empty_like(r)
        check(self.lib.fmmpc_apply_part(self._h, _lib.PART[part], _ptr(r), _ptr(out), k), self._h)
        return out

    def apply_host(self, r: np.ndarray) -> np.ndarray:
        r = np.ascontiguousarray(r, np.float64)
        z = np.empty_like(r)
        k = r.size // (self.n * self.n)
        check(self.lib.fmmpc_apply_host(self._h, r.ctypes.data_as(C.c_void_p), z.ctypes.data_as(C.c_void_p), k), self._h)
        return z

    def spmv(self, x, out=None):
        import torch
        k = self._vec(x)
        out = torch.empty_like(x) if out is None else out
        check(self.lib.fmmpc_spmv(self._h, _ptr(x), _ptr(out), k), self._h)
        return out

    def solve(self, f, g=None, u0=None, method="fgmres", restart=30, maxit=200, rtol=1e-8,
              use_graphs=2, raise_on_fail=True):
        """Krylov solve of A u = f (+ boundary values g); returns (u, info dict).
        use_graphs: 2 the whole solve as one CUDA graph (device-side convergence), 1 a host
        loop replaying the preconditioner's graph, 0 a host loop of single launches."""
        import torch
        k = self._vec(f)
        u = torch.zeros_like(f) if u0 is None else u0.clone()
        opts = _lib.SolveOpts(_lib.METHOD[method], restart, maxit, rtol, use_graphs)
        info = _lib.SolveInfo()
        gp = C.c_void_p(0) if g is None else _ptr(g)
        rc = self.lib.fmmpc_solve(self._h, _ptr(f), gp, _ptr(u), k, C.byref(opts), C.byref(info))
        out = dict(iters=info.iters, rel_res=info.rel_res, t_setup_ms=info.t_setup_ms,
                   t_solve_ms=info.t_solve_ms, status=info.status)
        if rc != 0 and (raise_on_fail or rc not in (-4,)):
            check(rc, self._h)
        return u, out

    def solve_host(self, f: np.ndarray, g=None, method="fgmres", restart=30, maxit=200, rtol=1e-8):
        f = np.ascontiguousarray(f, np.float64)
        u = np.zeros_like(f)
        k = f.size // (self.n * self.n)
        opts = _lib.SolveOpts(_lib.METHOD[method], restart, maxit, rtol, 0)
        info = _lib.SolveInfo()
        gp = None if g is None else np.ascontiguousarray(g, np.float64).ctypes.data_as(C.c_void_p)
        rc = self.lib.fmmpc_solve_host(self._h, f.ctypes.data_as(C.c_void_p), gp,
                                       u.ctypes.data_as(C.c_void_p), k, C.byref(opts), C.byref(info))
        check(rc, self._h)
        return u, dict(iters=info.iters, rel_res=info.rel_res, t_solve_ms=info.t_solve_ms)


def autotune(f, n: int, tol: float = 1e-5, precision: str = "fp32", theta: float = 0.4,
             side: float = 1.0, x0: float = 0.0, y0: float = 0.0, method: str = "fgmres",
             restart: int = 30, maxit: int = 100, rtol: float = 1e-8, stream=None):
    """fmmpc_autotune: best (leaf_max, p) for right-hand side f and the candidate report."""
    import torch
    lib = _lib.load()
    stream = stream if stream is not None else torch.cuda.current_stream()
    g = _lib.Grid(n, n, x0, y0, x0 + side, y0 + side)
    base = _lib.Params(10, 64, theta, _lib.PREC[precision], 1, 0)
    opts = _lib.SolveOpts(_lib.METHOD[method], restart, maxit, rtol, 1)
    best = _lib.Params()
    rep = (_lib.TuneEntry * 16)()
    cnt = C.c_int32()
    rc = lib.fmmpc_autotune(C.byref(g), C.byref(base), C.byref(opts), _ptr(f), tol,
                            C.c_void_p(stream.cuda_stream), C.byref(best), rep, 16, C.byref(cnt))
    check(rc, None)
    report = [dict(leaf_max=e.leaf_max, p=e.p, rel_err=e.rel_err, solve_ms=e.solve_ms, iters=e.iters,
                   ok=bool(e.ok)) for e in rep[: cnt.value]]
    return dict(leaf_max=best.leaf_max, p=best.p), report


class FmmBatch:
    """Independent problems of uneven size solved together (fmmpc_create_batched)."""

    def __init__(self, sides, p: int = 10, leaf_max: int = 64, theta: float = 0.4,
                 precision: str = "fp32", autotune: bool = False, stream=None):
        import torch
        self.lib = _lib.load()
        self.sides = [int(s) for s in sides]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        grids = (_lib.Grid * len(self.sides))(*[_lib.Grid(s, s, 0.0, 0.0, 1.0, 1.0) for s in self.sides])
        prm = _lib.Params(p, leaf_max, theta, _lib.PREC[precision], 1, 1 if autotune else 0)
        h = C.c_void_p()
        check(self.lib.fmmpc_create_batched(C.byref(h), len(self.sides), grids, C.byref(prm),
                                            C.c_void_p(self.stream.cuda_stream)), None)
        self._h = h

    def config(self, i: int):
        v = C.c_int64()
        self.lib.fmmpc_batch_query(self._h, i, 1, C.byref(v))
        leaf = v.value
        self.lib.fmmpc_batch_query(self._h, i, 100, C.byref(v))
        return dict(leaf_side=leaf, p=v.value)

    def solve(self, fs, us=None, restart: int = 30, maxit: int = 200, rtol: float = 1e-8, use_graphs: int = 1):
        import torch
        k = len(self.sides)
        us = [torch.zeros_like(f) for f in fs] if us is None else us
        fp = (C.c_void_p * k)(*[f.data_ptr() for f in fs])
        up = (C.c_void_p * k)(*[u.data_ptr() for u in us])
        opts = _lib.SolveOpts(_lib.METHOD["fgmres"], restart, maxit, rtol, use_graphs)
        infos = (_lib.SolveInfo * k)()
        rc = self.lib.fmmpc_solve_batched(self._h, fp, None, up, C.byref(opts), infos)
        out = [dict(iters=i.iters, rel_res=i.rel_res, status=i.status, t_solve_ms=i.t_solve_ms) for i in infos]
        if rc != 0:
            raise FmmpcError(rc, (self.lib.fmmpc_batch_last_error(self._h) or b"").decode())
        return us, out

    def close(self):
        if getattr(self, "_h", None):
            self.lib.fmmpc_destroy_batched(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
