"""FP64 CPU oracle for the FMM-BEM preconditioned Poisson solve (arXiv:1308.3339).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py`` may import this package.  It wraps the plain C
restatement in ``fmm_oracle.c`` (built with gcc, no CUDA) and shares no code with the
GPU library.  Each wrapper names the paper passage the C routine follows.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_LIBDIR = os.path.join(_HERE, "_build")
_LIB = None

# integer views of the oracle's problem sizes (orc_query)
Q_L, Q_LEAF_SIDE, Q_NM2L, Q_NP2P, Q_NM2L_VB, Q_NP2P_VB, Q_NG, Q_NCELL, Q_LU_OK = range(9)
E_KEYS, E_PERM, E_CELL_START, E_M2L, E_P2P, E_M2L_VB, E_P2P_VB = range(7)


def lib_path() -> str:
    return os.path.join(_LIBDIR, f"liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, no FMA contraction)."""
    out = lib_path()
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(_LIBDIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    if _LIB is not None:
        return _LIB
    L = C.CDLL(build())
    d, i, i64, vp = C.c_double, C.c_int, C.c_int64, C.c_void_p
    L.orc_version.restype = i
    L.orc_threads.restype = i
    L.orc_spmv5.argtypes = [i, d, vp, vp]
    L.orc_fold_rhs.argtypes = [i, d, vp, vp, vp]
    L.orc_spmv5_var.argtypes = [i, d, vp, vp, vp]
    L.orc_fold_rhs_var.argtypes = [i, d, vp, vp, vp, vp]
    L.orc_spmv_q1.argtypes = [i, vp, vp]
    L.orc_q1_load.argtypes = [i, d, vp, vp]
    L.orc_q1_mass_solve.argtypes = [i, d, vp, vp]
    L.orc_set_operator.argtypes = [vp, i, vp]
    L.orc_set_operator.restype = i
    L.orc_self_constant.restype = d
    L.orc_direct_V.argtypes = [i, d, d, d, vp, vp]
    L.orc_direct_V_at.argtypes = [i, d, d, d, vp, i, vp, vp, vp]
    L.orc_direct_V_nodes.argtypes = [i, d, d, d, vp, i, vp, vp]
    L.orc_p2m.argtypes = [i, i, vp, vp, vp, d, d, vp]
    L.orc_m2m.argtypes = [i, vp, d, d, vp]
    L.orc_m2l.argtypes = [i, vp, d, d, vp]
    L.orc_l2l.argtypes = [i, vp, d, d, vp]
    L.orc_l2p.argtypes = [i, vp, d, d]
    L.orc_l2p.restype = d
    L.orc_m2p.argtypes = [i, vp, d, d]
    L.orc_m2p.restype = d
    L.orc_seg_int_log.argtypes = [d] * 6
    L.orc_seg_int_log.restype = d
    L.orc_seg_int_dlog.argtypes = [d] * 6
    L.orc_seg_int_dlog.restype = d
    L.orc_elements.argtypes = [i, d, d, d] + [vp] * 6
    L.orc_bem_matrices.argtypes = [i, d, d, d, vp, vp]
    L.orc_bem_rows.argtypes = [i, d, d, d, i, vp, vp, vp]
    L.orc_layers_at.argtypes = [i, d, d, d, vp, vp, i, vp, vp, vp, vp]
    L.orc_lu.argtypes = [i, vp, vp]
    L.orc_lu.restype = i
    L.orc_lu_solve.argtypes = [i, vp, vp, vp]
    L.orc_morton_keys.argtypes = [i, vp]
    L.orc_sort_perm.argtypes = [i, vp, vp]
    L.orc_leaf_level.argtypes = [i, i]
    L.orc_leaf_level.restype = i
    L.orc_create.argtypes = [i, d, d, d, i, i, i, i]
    L.orc_create.restype = vp
    L.orc_destroy.argtypes = [vp]
    L.orc_query.argtypes = [vp, i]
    L.orc_query.restype = i64
    L.orc_export.argtypes = [vp, i, vp]
    L.orc_apply.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp]
    L.orc_apply.restype = i
    L.orc_apply_bc.argtypes = [vp, i, vp, vp, vp, vp]
    L.orc_apply_bc.restype = i
    L.orc_apply_dl.argtypes = [vp, i, vp, vp, vp]
    L.orc_apply_transpose.argtypes = [vp, i, vp, vp]
    L.orc_apply_transpose.restype = i
    L.orc_lu_solve_transpose.argtypes = [i, vp, vp, vp]
    L.orc_apply_dl.restype = i
    L.orc_solve.argtypes = [vp, i, i, i, d, i, vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_double), vp]
    L.orc_solve.restype = i
    _LIB = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def threads() -> int:
    return _lib().orc_threads()


# ---------------------------------------------------------------- discrete system
def spmv5(n: int, h: float, x: np.ndarray) -> np.ndarray:
    """A x for the 5-point stencil (Eq. e:axb, FD reading)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    y = np.empty_like(x)
    _lib().orc_spmv5(n, h, _p(x), _p(y))
    return y


def fold_rhs(n: int, h: float, f: np.ndarray, g: np.ndarray | None) -> np.ndarray:
    """b = f + boundary values of the stencil neighbours / h^2 (Eq. e:pbound)."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    b = np.empty_like(f)
    _lib().orc_fold_rhs(n, h, _p(f), _p(gg), _p(b))
    return b


def spmv5_var(n: int, h: float, a: np.ndarray, x: np.ndarray) -> np.ndarray:
    """A x for -div(a grad u), five-point flux form (Sec. 4.4, Sec. 6.4); a at the
    (n+2)^2 nodes of the full grid."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    assert a.size == (n + 2) ** 2
    y = np.empty_like(x)
    _lib().orc_spmv5_var(n, h, _p(a), _p(x), _p(y))
    return y


def fold_rhs_var(n, h, a, f, g):
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    gg = None if g is None else np.ascontiguousarray(g, dtype=np.float64).reshape(-1)
    b = np.empty_like(f)
    _lib().orc_fold_rhs_var(n, h, _p(a), _p(f), _p(gg), _p(b))
    return b


def spmv_q1(n: int, x: np.ndarray) -> np.ndarray:
    """A x for the Q1 stiffness of -lap on the uniform grid (Sec. 6.1), zero Dirichlet."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    y = np.empty_like(x)
    _lib().orc_spmv_q1(n, _p(x), _p(y))
    return y


def q1_load(n, h, f):
    """Lumped Q1 load vector b = h^2 f."""
    f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
    b = np.empty_like(f)
    _lib().orc_q1_load(n, h, _p(f), _p(b))
    return b


def q1_mass_solve(n, h, r):
    """c with M c = r, M the consistent Q1 mass matrix of the interior nodes."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    c = np.empty_like(r)
    _lib().orc_q1_mass_solve(n, h, _p(r), _p(c))
    return c


def self_constant() -> float:
    """Mean of ln|x| over the unit square centred at the origin (self term of G)."""
    return _lib().orc_self_constant()


def direct_V(n, x0, y0, side, r):
    """(V r)_i by the O(N^2) sum of Eq. e:volume_integral."""
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    out = np.empty_like(r)
    _lib().orc_direct_V(n, x0, y0, side, _p(r), _p(out))
    return out


def direct_V_at(n, x0, y0, side, r, tx, ty):
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    tx = np.ascontiguousarray(tx, dtype=np.float64)
    ty = np.ascontiguousarray(ty, dtype=np.float64)
    out = np.empty(tx.size)
    _lib().orc_direct_V_at(n, x0, y0, side, _p(r), tx.size, _p(tx), _p(ty), _p(out))
    return out


def direct_V_nodes(n, x0, y0, side, r, idx):
    r = np.ascontiguousarray(r, dtype=np.float64).reshape(-1)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.empty(idx.size)
    _lib().orc_direct_V_nodes(n, x0, y0, side, _p(r), idx.size, _p(idx), _p(out))
    return out


# ---------------------------------------------------------------- expansions (Sec. 5.3)
def p2m(p, px, py, f, c: complex):
    px = np.ascontiguousarray(px, np.float64); py = np.ascontiguousarray(py, np.float64)
    f = np.ascontiguousarray(f, np.float64)
    M = np.zeros(p, np.complex128)
    _lib().orc_p2m(p, px.size, _p(px), _p(py), _p(f), c.real, c.imag, _p(M))
    return M


def m2m(M_child, zMmu: complex):
    M_child = np.ascontiguousarray(M_child, np.complex128)
    out = np.zeros_like(M_child)
    _lib().orc_m2m(M_child.size, _p(M_child), zMmu.real, zMmu.imag, _p(out))
    return out


def m2l(M, zLM: complex):
    M = np.ascontiguousarray(M, np.complex128)
    out = np.zeros_like(M)
    _lib().orc_m2l(M.size, _p(M), zLM.real, zLM.imag, _p(out))
    return out


def l2l(Lp, zlL: complex):
    Lp = np.ascontiguousarray(Lp, np.complex128)
    out = np.zeros_like(Lp)
    _lib().orc_l2l(Lp.size, _p(Lp), zlL.real, zlL.imag, _p(out))
    return out


def l2p(Lc, zil: complex) -> float:
    Lc = np.ascontiguousarray(Lc, np.complex128)
    return _lib().orc_l2p(Lc.size, _p(Lc), zil.real, zil.imag)


def m2p(M, ziM: complex) -> float:
    M = np.ascontiguousarray(M, np.complex128)
    return _lib().orc_m2p(M.size, _p(M), ziM.real, ziM.imag)


# ---------------------------------------------------------------- boundary (Sec. 4)
def seg_int_log(x, a, b) -> float:
    """int over segment [a,b] of ln|x-y| ds_y, closed form."""
    return _lib().orc_seg_int_log(x[0], x[1], a[0], a[1], b[0], b[1])


def seg_int_dlog(x, a, b) -> float:
    """int over segment [a,b] of d/dn_y ln|x-y| ds_y, outward normal."""
    return _lib().orc_seg_int_dlog(x[0], x[1], a[0], a[1], b[0], b[1])


def elements(n, x0, y0, side):
    NG = 4 * n
    arrs = [np.empty(NG) for _ in range(6)]
    _lib().orc_elements(n, x0, y0, side, *[_p(a) for a in arrs])
    return arrs  # ax, ay, bx, by, cx, cy


def bem_matrices(n, x0, y0, side):
    NG = 4 * n
    S = np.empty((NG, NG)); K = np.empty((NG, NG))
    _lib().orc_bem_matrices(n, x0, y0, side, _p(S), _p(K))
    return S, K


def bem_rows(n, x0, y0, side, rows):
    """Rows of the single- and double-layer matrices (Sec. 4.3) at collocation indices rows."""
    rows = np.ascontiguousarray(rows, np.int32)
    NG = 4 * n
    S = np.empty((rows.size, NG)); K = np.empty((rows.size, NG))
    _lib().orc_bem_rows(n, x0, y0, side, rows.size, _p(rows), _p(S), _p(K))
    return S, K


def layers_at(n, x0, y0, side, tx, ty, q=None, mu=None):
    """Single-layer (density q) and double-layer (density mu) potentials of constant
    elements at targets (tx, ty) off the boundary: the boundary terms of Eq. e:uinter."""
    tx = np.ascontiguousarray(tx, np.float64); ty = np.ascontiguousarray(ty, np.float64)
    qq = None if q is None else np.ascontiguousarray(q, np.float64)
    mm = None if mu is None else np.ascontiguousarray(mu, np.float64)
    sl, dl = np.zeros(tx.size), np.zeros(tx.size)
    _lib().orc_layers_at(n, x0, y0, side, _p(qq), _p(mm), tx.size, _p(tx), _p(ty), _p(sl), _p(dl))
    return sl, dl


# ---------------------------------------------------------------- tree (Sec. 5.1)
def lu_solve_transpose(LU, piv, b):
    """x with A^T x = b from orc_lu's factors of A."""
    N = LU.shape[0]
    x = np.array(b, np.float64)
    _lib().orc_lu_solve_transpose(N, _p(np.ascontiguousarray(LU)), _p(np.ascontiguousarray(piv, np.int32)), _p(x))
    return x


def lu(A):
    """orc_lu's in-place factors of A (copied) and pivots."""
    LU = np.array(A, np.float64)
    piv = np.empty(LU.shape[0], np.int32)
    if _lib().orc_lu(LU.shape[0], _p(LU), _p(piv)):
        raise RuntimeError("oracle: singular matrix")
    return LU, piv


def morton_keys(n):
    k = np.empty(n * n, np.uint32)
    _lib().orc_morton_keys(n, _p(k))
    return k


def sort_perm(keys):
    keys = np.ascontiguousarray(keys, np.uint32)
    perm = np.empty(keys.size, np.int32)
    _lib().orc_sort_perm(keys.size, _p(keys), _p(perm))
    return perm


def leaf_level(n, leaf_max):
    return _lib().orc_leaf_level(n, leaf_max)


class Problem:
    """Tree, interaction lists, boundary elements and BEM LU factors for one grid
    (the analogue of the paper's PCSetUp, Sec. 7.1)."""

    def __init__(self, n, p=10, leaf_max=64, theta=(2, 5), x0=0.0, y0=0.0, side=1.0):
        self.n, self.p, self.theta = n, p, theta
        self.x0, self.y0, self.side = x0, y0, side
        self.h = side / (n + 1)
        self._h = _lib().orc_create(n, x0, y0, side, leaf_max, p, theta[0], theta[1])
        if not self._h:
            raise ValueError(f"oracle: unsupported grid n={n} leaf_max={leaf_max} p={p}")
        q = lambda w: _lib().orc_query(self._h, w)
        self.L, self.leaf_side = q(Q_L), q(Q_LEAF_SIDE)
        self.n_m2l, self.n_p2p = q(Q_NM2L), q(Q_NP2P)
        self.n_m2l_vb, self.n_p2p_vb = q(Q_NM2L_VB), q(Q_NP2P_VB)
        self.NG, self.n_cell, self.lu_ok = q(Q_NG), q(Q_NCELL), bool(q(Q_LU_OK))

    def __del__(self):
        if getattr(self, "_h", None):
            _lib().orc_destroy(self._h)
            self._h = None

    def set_operator(self, op, a=None):
        """Operator of later solves: "fd5" (Eq. e:axb), "fd5_var" with coefficient a at the
        (n+2)^2 full-grid nodes (Sec. 6.4), or "q1" (Sec. 6.1; the preconditioner then acts
        on M^{-1} r, M the consistent Q1 mass matrix)."""
        code = {"fd5": 0, "fd5_var": 1, "q1": 2}[op]
        aa = None if a is None else np.ascontiguousarray(a, np.float64).reshape(-1)
        if _lib().orc_set_operator(self._h, code, _p(aa)):
            raise ValueError("oracle: bad operator")
        self._a = aa

    def export(self, what):
        N = self.n * self.n
        shape = {E_KEYS: (N,), E_PERM: (N,), E_CELL_START: (self.n_cell,),
                 E_M2L: (self.n_m2l, 3), E_P2P: (self.n_p2p, 2),
                 E_M2L_VB: (self.n_m2l_vb, 3), E_P2P_VB: (self.n_p2p_vb, 2)}[what]
        a = np.empty(shape, np.uint32 if what == E_KEYS else np.int32)
        _lib().orc_export(self._h, what, _p(a))
        return a

    def apply(self, r, mode="fmm", stages=False):
        """z = P^{-1} r (Sec. 3.2).  mode 'direct' or 'fmm'.  With stages=True also
        returns V r at nodes, V r at collocation points, q, and (fmm) near/far parts."""
        N = self.n * self.n
        r = np.ascontiguousarray(r, np.float64).reshape(-1)
        z = np.empty(N)
        vr, vc, q = np.empty(N), np.empty(self.NG), np.empty(self.NG)
        near, far = np.empty(N), np.empty(N)
        st = _lib().orc_apply(self._h, 0 if mode == "direct" else 1, _p(r), _p(z), _p(vr), _p(vc),
                              _p(q), _p(near), _p(far))
        if st:
            raise RuntimeError("oracle: singular BEM matrix")
        if not stages:
            return z
        out = dict(z=z, vr=vr, vr_col=vc, q=q)
        if mode != "direct":
            out.update(near=near, far=far)
        return out

    def apply_bc(self, f, g, mode="fmm", with_q=False):
        """The boundary-integral solution of -lap u = f, u = g (Sec. 4.1, Eqs. e:ubound and
        e:uinter) at the nodes; g at the 4n element midpoints, side order."""
        N = self.n * self.n
        f = np.ascontiguousarray(f, np.float64).reshape(-1)
        g = np.ascontiguousarray(g, np.float64).reshape(-1)
        assert g.size == self.NG
        u, q = np.empty(N), np.empty(self.NG)
        if _lib().orc_apply_bc(self._h, 0 if mode == "direct" else 1, _p(f), _p(g), _p(u), _p(q)):
            raise RuntimeError("oracle: singular BEM matrix")
        return (u, q) if with_q else u

    def apply_transpose(self, zb, mode="fmm"):
        """rb = P^{-T} zb, the transpose of apply (gradient with respect to the source weights)."""
        zb = np.ascontiguousarray(zb, np.float64).reshape(-1)
        rb = np.empty_like(zb)
        if _lib().orc_apply_transpose(self._h, 0 if mode == "direct" else 1, _p(zb), _p(rb)):
            raise RuntimeError("oracle: singular BEM matrix")
        return rb

    def apply_dl(self, r, mode="fmm", with_mu=False):
        """The preconditioner with the second-kind double-layer correction:
        (-1/2 I + K) mu = -(V r)|_Gamma, z = V r + int_Gamma mu dG/dn."""
        N = self.n * self.n
        r = np.ascontiguousarray(r, np.float64).reshape(-1)
        z, mu = np.empty(N), np.empty(self.NG)
        if _lib().orc_apply_dl(self._h, 0 if mode == "direct" else 1, _p(r), _p(z), _p(mu)):
            raise RuntimeError("oracle: singular double-layer system")
        return (z, mu) if with_mu else z

    def solve(self, b, method="fgmres", restart=30, maxit=200, rtol=1e-8, prec="fmm", x0=None,
              history=False):
        """Krylov solve of A x = b (Sec. 3.1). Returns (x, iters, true relres, converged[, hist])."""
        N = self.n * self.n
        b = np.ascontiguousarray(b, np.float64).reshape(-1)
        x = np.zeros(N) if x0 is None else np.array(x0, np.float64).reshape(-1)
        it, rr = C.c_int(0), C.c_double(0.0)
        hist = np.full(maxit + 1, np.nan)
        m = {"cg": 0, "gmres": 1, "fgmres": 2}[method]
        pr = {"none": 0, "direct": 1, "fmm": 2, "fmm_dl": 3}[prec]
        conv = _lib().orc_solve(self._h, m, restart, maxit, rtol, pr, _p(b), _p(x), C.byref(it),
                                C.byref(rr), _p(hist))
        if conv < 0:
            raise RuntimeError("oracle: singular BEM matrix")
        res = (x, it.value, rr.value, bool(conv))
        return res + (hist[: it.value + 1],) if history else res
