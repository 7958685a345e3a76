"""Pins for the oracle's discrete system and Krylov solvers (Sec. 2.1, Sec. 3.1).

Independent checks: the Kronecker-sum form of the 5-point matrix (scipy.sparse), the
closed-form eigenpair sin(pi x) sin(pi y), exactness of FD on quadratics (the Table t:p3
solution u = x^2 + y^2), and scipy's sparse direct solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
import synth_inputs as S
from conftest import rel_l2


def kron_laplacian(n, h):
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1])
    I = sp.identity(n)
    return ((sp.kron(I, T) + sp.kron(T, I)) / h ** 2).tocsr()


def test_spmv_matches_kronecker_sum():
    n = 12
    h = 1.0 / 13
    x = np.random.default_rng(1).standard_normal(n * n)
    assert rel_l2(O.spmv5(n, h, x), kron_laplacian(n, h) @ x) < 1e-14


@pytest.mark.parametrize("n", [8, 33, 64])
def test_spmv_eigenvector_closed_form(n):
    X, Y, h = S.grid_coords(n)
    u = np.sin(np.pi * X) * np.sin(np.pi * Y)
    lam = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    assert rel_l2(O.spmv5(n, h, u), lam * u) < 1e-12


def test_fold_rhs_quadratic_is_exact():
    # u = x^2 + y^2, f = -4 on [-1,1]^2 (Sec. 6.1, Table t:p3): 5-point FD is exact.
    n = 16
    X, Y, h = S.grid_coords(n, -1.0, -1.0, 2.0)
    u = X ** 2 + Y ** 2
    g = S.boundary_values(n, lambda x, y: x ** 2 + y ** 2, -1.0, -1.0, 2.0)
    b = O.fold_rhs(n, h, -4.0 * np.ones(n * n), g)
    assert rel_l2(O.spmv5(n, h, u), b) < 1e-12


@pytest.mark.parametrize("method", ["cg", "gmres", "fgmres"])
def test_unpreconditioned_krylov_matches_sparse_direct(method):
    n = 24
    f = S.gaussian_mixture(n, 3)
    h = 1.0 / (n + 1)
    ref = spla.spsolve(kron_laplacian(n, h).tocsc(), f)
    P = O.Problem(n, p=4, leaf_max=64)
    x, it, rr, conv = P.solve(f, method, restart=30, maxit=2000, rtol=1e-11, prec="none")
    assert conv and rr <= 1e-11
    assert rel_l2(x, ref) < 1e-8


@pytest.mark.parametrize("method", ["cg", "gmres", "fgmres"])
def test_preconditioned_solve_hits_closed_form(method):
    # f = 2 pi^2 sin sin: the discrete solution is (2 pi^2 / lambda_h) sin sin exactly.
    n = 64
    f, u = S.manufactured_sin(n)
    h = 1.0 / (n + 1)
    lam = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    P = O.Problem(n, p=10)
    x, it, rr, conv = P.solve(f, method, restart=30, maxit=100, rtol=1e-12, prec="fmm")
    assert conv
    assert rel_l2(x, (2 * np.pi ** 2 / lam) * u) < 1e-10


def test_fd_error_is_second_order():
    errs = []
    for n in (16, 32, 64):
        f, u = S.manufactured_sin(n)
        P = O.Problem(n, p=10)
        x, *_ = P.solve(f, "fgmres", rtol=1e-12, prec="fmm")
        errs.append(rel_l2(x, u))
    h = [1 / 17, 1 / 33, 1 / 65]
    # leading term pi^2 h^2 / 12 of |2 pi^2/lambda_h - 1|
    for e, hh in zip(errs, h):
        assert abs(e / (np.pi ** 2 * hh ** 2 / 12) - 1) < 0.02
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
