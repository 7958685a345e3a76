"""Pins for the oracle's further discretisations (CPU): the variable-coefficient five-point
operator of Sec. 4.4 / Sec. 6.4 and the Q1 finite-element stiffness of Sec. 6.1, and the
FMM-preconditioned solves with them (Tables t:p1, t:p1eig, t:v1).

Independent checks: a = 1 reduces to the constant five-point operator; symmetry and
positive definiteness; exactness for linear u with linear a; second-order convergence to a
manufactured solution; the Q1 stiffness against element-by-element Gauss quadrature of the
bilinear basis and against its Kronecker form K1 (x) M1 + M1 (x) K1; mesh-independent PCG
counts and a bounded spectrum of P^{-1} A (the behaviour the paper's tables report)."""
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
import synth_inputs as S
from conftest import rel_l2

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def dense_of(apply, N):
    A = np.empty((N, N))
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1.0
        A[:, k] = apply(e)
    return A


def test_variable_coefficient_reduces_to_five_point_for_a_one():
    n = 20
    h = 1.0 / (n + 1)
    x = np.random.default_rng(0).standard_normal(n * n)
    a = np.ones((n + 2) ** 2)
    assert np.max(np.abs(O.spmv5_var(n, h, a, x) - O.spmv5(n, h, x))) < 1e-12 / h ** 2


def test_variable_coefficient_operator_is_symmetric_positive_definite():
    n = 12
    h = 1.0 / (n + 1)
    a = S.diffusion_coefficient(n, 0.25, 3, 2)
    A = dense_of(lambda v: O.spmv5_var(n, h, a, v), n * n)
    assert np.max(np.abs(A - A.T)) < 1e-12 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0


def test_variable_coefficient_exact_for_linear_u_and_a():
    # u = x, a = 1 + x + 2y: -div(a grad u) = -1; the flux form with face means is exact
    n = 16
    X, Y, h = S.grid_coords(n)
    t = np.arange(n + 2) * h
    XX, YY = np.meshgrid(t, t)
    a = (1.0 + XX + 2.0 * YY).ravel()
    g = S.boundary_values(n, lambda x, y: x + 0 * y)
    b = O.fold_rhs_var(n, h, a, -np.ones(n * n), g)
    assert np.max(np.abs(O.spmv5_var(n, h, a, X) - b)) < 1e-9
    assert np.max(np.abs(O.fold_rhs_var(n, h, np.ones((n + 2) ** 2), np.zeros(n * n), g)
                         - O.fold_rhs(n, h, np.zeros(n * n), g))) < 1e-12


def test_variable_coefficient_second_order_convergence():
    # u = sin(pi x) sin(pi y), a = 1 + mu sin(m pi x) sin(k pi y):
    # f = -(a_x u_x + a_y u_y + a lap u), computed analytically here
    mu, m, k = 0.5, 2, 1
    errs = []
    for n in (15, 31, 63):
        X, Y, h = S.grid_coords(n)
        u = np.sin(np.pi * X) * np.sin(np.pi * Y)
        ux = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
        uy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
        av = 1 + mu * np.sin(m * np.pi * X) * np.sin(k * np.pi * Y)
        ax = mu * m * np.pi * np.cos(m * np.pi * X) * np.sin(k * np.pi * Y)
        ay = mu * k * np.pi * np.sin(m * np.pi * X) * np.cos(k * np.pi * Y)
        f = -(ax * ux + ay * uy - 2 * np.pi ** 2 * av * u)
        a = S.diffusion_coefficient(n, mu, m, k)
        A = sp.csr_matrix(dense_of(lambda v: O.spmv5_var(n, h, a, v), n * n))
        uh = spla.spsolve(A, f)
        errs.append(np.max(np.abs(uh - u)))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def q1_assembled(n, h):
    """Interior Q1 stiffness of -lap by 2x2 Gauss quadrature of the bilinear basis on every
    element of the (n+1) x (n+1) element grid, zero Dirichlet rows dropped (numpy only)."""
    g = np.array([-1, 1]) / np.sqrt(3.0)
    # local basis on [-1,1]^2: phi_a = (1 + xa x)(1 + ya y)/4, nodes (xa, ya) in order
    nodes = [(-1, -1), (1, -1), (-1, 1), (1, 1)]
    Ke = np.zeros((4, 4))
    for xi in g:
        for eta in g:
            grads = [np.array([xa * (1 + ya * eta) / 4, ya * (1 + xa * xi) / 4]) * (2 / h) for xa, ya in nodes]
            for p in range(4):
                for q in range(4):
                    Ke[p, q] += grads[p] @ grads[q] * (h / 2) ** 2
    N = n * n
    A = np.zeros((N, N))
    for ey in range(n + 1):
        for ex in range(n + 1):
            gl = []
            for xa, ya in nodes:
                i, j = ex + (xa + 1) // 2 - 1, ey + (ya + 1) // 2 - 1  # interior indices
                gl.append(j * n + i if 0 <= i < n and 0 <= j < n else -1)
            for p in range(4):
                for q in range(4):
                    if gl[p] >= 0 and gl[q] >= 0:
                        A[gl[p], gl[q]] += Ke[p, q]
    return A


def test_q1_stiffness_matches_element_quadrature_and_kronecker_form():
    n = 9
    h = 2.0 / (n + 1)
    A = dense_of(lambda v: O.spmv_q1(n, v), n * n)
    assert np.max(np.abs(A - q1_assembled(n, h))) < 1e-13
    K1 = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]) / h
    M1 = sp.diags([np.ones(n - 1), 4 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) * h / 6
    Ak = (sp.kron(K1, M1) + sp.kron(M1, K1)).toarray()
    assert np.max(np.abs(A - Ak)) < 1e-13


def test_q1_mass_solve_inverts_the_kronecker_mass_matrix():
    n = 11
    h = 2.0 / (n + 1)
    M1 = sp.diags([np.ones(n - 1), 4 * np.ones(n), np.ones(n - 1)], [-1, 0, 1]) / 6
    M = (h * h * sp.kron(M1, M1)).tocsr()
    r = np.random.default_rng(4).standard_normal(n * n)
    assert rel_l2(M @ O.q1_mass_solve(n, h, r), r) < 1e-14


def test_q1_finite_elements_converge_at_second_order():
    errs = []
    for n in (15, 31, 63):
        X, Y, h = S.grid_coords(n)
        u = np.sin(np.pi * X) * np.sin(np.pi * Y)
        b = O.q1_load(n, h, 2 * np.pi ** 2 * u)
        A = sp.csr_matrix(dense_of(lambda v: O.spmv_q1(n, v), n * n))
        errs.append(np.max(np.abs(spla.spsolve(A, b) - u)))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_q1_pcg_iterations_are_mesh_independent():
    # Table t:p1: -lap u = 1 on [-1,1]^2, u = 0, PCG to a six-digit drop, FMM preconditioner:
    # the paper's counts are 5..7 and flat in h; the grids here are n = 16 .. 64 (power-of-two
    # interior sides, h = 2/(n+1)); the preconditioner acts on M^{-1} r
    gold = np.loadtxt(os.path.join(GOLD, "paper_table_p1.txt"))  # h, iterations (FMM column)
    counts = {}
    for n in (16, 32, 64, 128):
        h = 2.0 / (n + 1)
        R = O.Problem(n, p=10, x0=-1.0, y0=-1.0, side=2.0)
        R.set_operator("q1")
        _, it, rr, conv = R.solve(O.q1_load(n, h, np.ones(n * n)), "cg", maxit=20, rtol=1e-6, prec="fmm")
        assert conv and rr <= 1e-6
        counts[n] = it
        k = int(np.argmin(np.abs(np.log(gold[:, 0] / h))))  # the table row of the nearest h
        if abs(np.log2(gold[k, 0] / h)) < 0.2:
            assert abs(it - gold[k, 1]) <= 1, (n, h, it, gold[k])
    print("Q1 PCG iterations (oracle):", counts)
    assert max(counts.values()) - min(counts.values()) <= 1


def test_q1_preconditioned_spectrum_is_bounded():
    # Table t:p1eig: the eigenvalues of P^{-1} A lie in a small h-independent interval
    kap = []
    for n in (8, 16):
        h = 2.0 / (n + 1)
        R = O.Problem(n, p=12, x0=-1.0, y0=-1.0, side=2.0)
        Pinv = dense_of(lambda v: R.apply(O.q1_mass_solve(n, h, v), "fmm"), n * n)
        A = dense_of(lambda v: O.spmv_q1(n, v), n * n)
        lam = np.linalg.eigvals(Pinv @ A).real
        kap.append(lam.max() / lam.min())
        print(f"Q1 n={n}: lambda(P^-1 A) in [{lam.min():.3f}, {lam.max():.3f}], kappa {kap[-1]:.3f}")
        # the paper's Table t:p1eig: kappa 1.77-1.80 (IFISS Q1 FEM, its own BEM)
        assert 0.5 < lam.min() and lam.max() < 2.5 and kap[-1] < 2.5
    assert kap[1] < 1.1 * kap[0]


def test_variable_coefficient_pcg_with_constant_coefficient_preconditioner():
    # Sec. 6.4 / Table t:v1: -div(a grad u) = 1, a = 1 + mu sin(pi x) sin(pi y) on [-1,1]^2,
    # preconditioned by the constant-coefficient FMM-BEM P; counts grow mildly with mu and
    # stay flat in h
    counts = {}
    for mu in (2.0 ** -8, 2.0 ** -2):
        for n in (16, 32, 64):
            h = 2.0 / (n + 1)
            a = S.diffusion_coefficient(n, mu, 1, 1, -1.0, -1.0, 2.0)
            R = O.Problem(n, p=10, x0=-1.0, y0=-1.0, side=2.0)
            R.set_operator("fd5_var", a)
            _, it, rr, conv = R.solve(np.ones(n * n), "cg", maxit=30, rtol=1e-6, prec="fmm")
            assert conv
            counts[(mu, n)] = it
    print("variable-coefficient PCG iterations (oracle):", counts)
    for mu in (2.0 ** -8, 2.0 ** -2):
        c = [counts[(mu, n)] for n in (16, 32, 64)]
        assert max(c) - min(c) <= 2
    assert counts[(2.0 ** -2, 64)] >= counts[(2.0 ** -8, 64)]
