"""Pins for the oracle's boundary-element parts and the whole preconditioner
(Sec. 4.1 Eqs. e:green/e:ubound/e:uinter, Sec. 4.2-4.3, Sec. 6.1 Tables t:p1/t:p1eig).

Independent checks: Gauss-Legendre and adaptive quadrature of the element integrals,
Gauss's identity for the double layer, reproduction of harmonic functions (Table t:p2's
solution), convergence of P^{-1} f to the continuum solution, and the bounded,
mesh-independent spectrum and iteration counts that Tables t:p1eig and t:p1 report.
"""
import os

import numpy as np
import pytest
from scipy import integrate

import oracle as O
import synth_inputs as S
from conftest import rel_l2

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gl(x, a, b, fn, k=64):
    t, w = np.polynomial.legendre.leggauss(k)
    a, b = np.asarray(a, float), np.asarray(b, float)
    L = np.linalg.norm(b - a)
    pts = a[None, :] + (t[:, None] + 1) / 2 * (b - a)[None, :]
    return L / 2 * np.sum(w * fn(np.asarray(x, float)[None, :] - pts, (b - a) / L))


def test_single_layer_segment_integral_vs_quadrature():
    rng = np.random.default_rng(0)
    for _ in range(50):
        a, b = rng.uniform(-1, 1, 2), rng.uniform(-1, 1, 2)
        mid, L = (a + b) / 2, np.linalg.norm(b - a)
        x = mid + rng.uniform(1.5, 4) * L * np.array([np.cos(t := rng.uniform(0, 6.3)), np.sin(t)])
        ref = _gl(x, a, b, lambda d, e: np.log(np.hypot(d[:, 0], d[:, 1])))
        assert abs(O.seg_int_log(x, a, b) - ref) < 1e-12 * max(1, abs(ref))


def test_single_layer_self_term():
    # collocation at the midpoint: int_{-l/2}^{l/2} ln|s| ds = l (ln(l/2) - 1)
    for L in (0.01, 0.3, 2.0):
        val, _ = integrate.quad(lambda s: np.log(abs(s)), -L / 2, L / 2, points=[0.0], limit=200)
        assert abs(O.seg_int_log((0.0, 0.0), (-L / 2, 0.0), (L / 2, 0.0)) - val) < 1e-12


def test_double_layer_segment_integral_vs_quadrature():
    rng = np.random.default_rng(1)
    for _ in range(50):
        a, b = rng.uniform(-1, 1, 2), rng.uniform(-1, 1, 2)
        mid, L = (a + b) / 2, np.linalg.norm(b - a)
        x = mid + rng.uniform(1.5, 4) * L * np.array([np.cos(t := rng.uniform(0, 6.3)), np.sin(t)])

        def dlog(d, e):  # d = x - y ; normal = tangent rotated clockwise
            nvec = np.array([e[1], -e[0]])
            return -(d @ nvec) / np.sum(d * d, axis=1)
        ref = _gl(x, a, b, dlog)
        assert abs(O.seg_int_dlog(x, a, b) - ref) < 1e-12 * max(1, abs(ref))


def test_double_layer_gauss_identity():
    n = 16
    S_, K = O.bem_matrices(n, 0.0, 0.0, 1.0)
    assert np.allclose(K.sum(axis=1), -0.5, atol=1e-13)  # smooth boundary point
    ax, ay, bx, by, cx, cy = O.elements(n, 0.0, 0.0, 1.0)
    for x in [(0.5, 0.5), (0.01, 0.7), (0.9, 0.95)]:
        tot = sum(O.seg_int_dlog(x, (ax[k], ay[k]), (bx[k], by[k])) for k in range(4 * n))
        assert abs(-tot / (2 * np.pi) + 1.0) < 1e-12


def _harmonic_error(n):
    # Sec. 6.1 second problem: u = 2(1+y)/((3+x)^2+(1+y)^2) on [-1,1]^2, harmonic.
    x0, side = -1.0, 2.0
    u = lambda x, y: 2 * (1 + y) / ((3 + x) ** 2 + (1 + y) ** 2)
    S_, K = O.bem_matrices(n, x0, x0, side)
    ax, ay, bx, by, cx, cy = O.elements(n, x0, x0, side)
    g = u(cx, cy)
    q = np.linalg.solve(S_, 0.5 * g + K @ g)  # e:ubound with f = 0
    X, Y, _ = S.grid_coords(n, x0, x0, side)
    NG = 4 * n
    uh = np.empty(n * n)
    for i in range(n * n):
        xi = (X[i], Y[i])
        sl = np.array([O.seg_int_log(xi, (ax[k], ay[k]), (bx[k], by[k])) for k in range(NG)])
        dl = np.array([O.seg_int_dlog(xi, (ax[k], ay[k]), (bx[k], by[k])) for k in range(NG)])
        uh[i] = (-sl / (2 * np.pi)) @ q - (-dl / (2 * np.pi)) @ g  # e:uinter with f = 0
    return rel_l2(uh, u(X, Y))


def test_bie_reproduces_harmonic_solution():
    e1, e2 = _harmonic_error(8), _harmonic_error(16)
    assert e2 < 1e-2
    assert e1 / e2 > 1.8  # at least first order (Sec. 6.2, Fig. f:discretization)


def test_preconditioner_converges_to_continuum_solution():
    errs = []
    for n in (16, 32, 64):
        f, u = S.manufactured_sin(n)
        errs.append(rel_l2(O.Problem(n, p=10).apply(f, "fmm"), u))
    assert errs[0] / errs[1] > 1.8 and errs[1] / errs[2] > 1.8
    assert errs[2] < 1e-3


def _dense(n, mode="direct", p=12, x0=0.0, side=1.0):
    P = O.Problem(n, p=p, x0=x0, y0=x0, side=side)
    I = np.eye(n * n)
    Pm = np.stack([P.apply(e, mode) for e in I], 1)
    A = np.stack([O.spmv5(n, side / (n + 1), e) for e in I], 1)
    return Pm, A


def test_spectrum_of_preconditioned_matrix_is_bounded():
    gold = np.loadtxt(os.path.join(GOLD, "paper_table_p1eig.txt"))
    kap = []
    for n in (8, 16):
        Pm, A = _dense(n, x0=-1.0, side=2.0)
        ev = np.linalg.eigvals(Pm @ A)
        assert np.abs(ev.imag).max() < 1e-8
        lo, hi = ev.real.min(), ev.real.max()
        assert 0.3 < lo and hi < 1.1
        kap.append(hi / lo)
    # same regime as the paper's FEM values (Table t:p1eig: 1.77-1.80), h-independent
    assert abs(kap[1] - kap[0]) < 0.15
    assert max(kap) < 1.5 * gold[:, 3].max()


def test_pcg_iterations_are_mesh_independent():
    # Table t:p1 setting: -lap u = 1 on [-1,1]^2, u = 0, PCG, six-digit drop, maxit 20.
    gold = np.loadtxt(os.path.join(GOLD, "paper_table_p1.txt"))
    its = []
    for n in (16, 32, 64):
        P = O.Problem(n, p=10, x0=-1.0, y0=-1.0, side=2.0)
        x, it, rr, conv = P.solve(np.ones(n * n), "cg", maxit=20, rtol=1e-6, prec="fmm")
        assert conv
        its.append(it)
    assert max(its) - min(its) <= 1
    assert max(its) <= gold[:, 1].max() + 3


def test_fmm_and_direct_preconditioners_give_same_iterations():
    n = 32
    f = S.gaussian_mixture(n, 2)
    P = O.Problem(n, p=10)
    _, it1, rr1, c1 = P.solve(f, "fgmres", rtol=1e-8, prec="fmm")
    _, it2, rr2, c2 = P.solve(f, "fgmres", rtol=1e-8, prec="direct")
    assert c1 and c2 and abs(it1 - it2) <= 1


def _element_quadrature(n, x0, y0, side, tx, ty, dens, kind, k=48):
    """sum_k dens_k int_{Gamma_k} K(x_t, y) dGamma by Gauss-Legendre on every element, in
    numpy (no oracle code): kind 'sl' K = G = -(1/2pi) ln r, kind 'dl' K = dG/dn_y."""
    ax, ay, bx, by, _, _ = O.elements(n, x0, y0, side)
    t, w = np.polynomial.legendre.leggauss(k)
    out = np.zeros(len(tx))
    for e in range(4 * n):
        a, b = np.array([ax[e], ay[e]]), np.array([bx[e], by[e]])
        L = np.linalg.norm(b - a)
        tan = (b - a) / L
        nrm = np.array([tan[1], -tan[0]])
        pts = a[None, :] + (t[:, None] + 1) / 2 * (b - a)[None, :]
        d = np.stack([tx, ty], 1)[:, None, :] - pts[None, :, :]
        r2 = np.sum(d * d, axis=2)
        val = -0.5 * np.log(r2) / (2 * np.pi) if kind == "sl" else (d @ nrm) / r2 / (2 * np.pi)
        out += dens[e] * L / 2 * (val @ w)
    return out


def test_bem_rows_match_quadrature_and_gauss_identity():
    # rows of S and K at sampled collocation points (the sampled-row check of the boundary
    # system at grids too large for the full matrices): entries of elements at least two
    # away from the collocation point against Gauss-Legendre quadrature; every row of K
    # sums to -1/2 (Gauss's identity for a point on a smooth part of Gamma)
    n, x0, y0, side = 16, -1.0, -1.0, 2.0
    rows = np.array([0, 5, 17, 40, 63], np.int32)
    Sr, Kr = O.bem_rows(n, x0, y0, side, rows)
    _, _, _, _, cx, cy = O.elements(n, x0, y0, side)
    for i, m in enumerate(rows):
        for k in range(4 * n):
            if min(abs(k - m), 4 * n - abs(k - m)) < 2:
                continue
            e = np.zeros(4 * n)
            e[k] = 1.0
            s_ref = _element_quadrature(n, x0, y0, side, cx[m:m + 1], cy[m:m + 1], e, "sl")[0]
            assert abs(Sr[i, k] - s_ref) < 1e-10
        assert abs(Kr[i].sum() + 0.5) < 1e-12


def test_layer_potentials_at_interior_points():
    # single and double layer at interior targets against element-wise quadrature; the
    # double layer of a unit density is -1 inside (Gauss's identity)
    n, x0, y0, side = 8, 0.0, 0.0, 1.0
    rng = np.random.default_rng(3)
    tx, ty = rng.uniform(0.15, 0.85, 20), rng.uniform(0.15, 0.85, 20)
    q, mu = rng.standard_normal(4 * n), rng.standard_normal(4 * n)
    sl, dl = O.layers_at(n, x0, y0, side, tx, ty, q=q, mu=mu)
    assert np.max(np.abs(sl - _element_quadrature(n, x0, y0, side, tx, ty, q, "sl"))) < 1e-12
    assert np.max(np.abs(dl - _element_quadrature(n, x0, y0, side, tx, ty, mu, "dl"))) < 1e-12
    _, one = O.layers_at(n, x0, y0, side, tx, ty, mu=np.ones(4 * n))
    assert np.max(np.abs(one + 1.0)) < 1e-12


def test_green_representation_of_a_harmonic_function():
    # Eq. e:uinter with f = 0: u(x) = int_Gamma du/dn G - int_Gamma u dG/dn for harmonic u.
    # Constant elements at midpoint values are first-order accurate: the error falls ~2x
    # per halving of the element length.
    x0, y0, side = -1.0, -1.0, 2.0
    u = lambda x, y: 2 * (1 + y) / ((3 + x) ** 2 + (1 + y) ** 2)  # Table t:p2's solution
    def dudn(x, y, nx, ny, e=1e-6):
        return ((u(x + e * nx, y + e * ny) - u(x - e * nx, y - e * ny)) / (2 * e))
    tx, ty = np.array([0.1, -0.4, 0.5]), np.array([0.2, 0.3, -0.5])
    errs = []
    for n in (16, 32, 64):
        ax, ay, bx, by, cx, cy = O.elements(n, x0, y0, side)
        tl = np.stack([bx - ax, by - ay], 1)
        tl /= np.linalg.norm(tl, axis=1)[:, None]
        q = dudn(cx, cy, tl[:, 1], -tl[:, 0])
        sl, dl = O.layers_at(n, x0, y0, side, tx, ty, q=q, mu=u(cx, cy))
        errs.append(np.max(np.abs(sl - dl - u(tx, ty))))
    assert errs[-1] < 2e-3
    assert errs[0] / errs[1] > 1.6 and errs[1] / errs[2] > 1.6


# ---------------------------------------------------------------- boundary data and the
# second-kind double-layer variant (Sec. 4.1 Eqs. e:ubound/e:uinter with g != 0)
def _midpoint_data(n, fn, x0, y0, side):
    _, _, _, _, cx, cy = O.elements(n, x0, y0, side)
    return fn(cx, cy)


def test_apply_bc_with_zero_data_is_the_preconditioner():
    n = 16
    r = S.random_field(n, 12)
    R = O.Problem(n, p=10)
    assert rel_l2(R.apply_bc(r, np.zeros(4 * n), "direct"), R.apply(r, "direct")) < 1e-13


@pytest.mark.parametrize("case", ["harmonic", "quadratic"])
def test_apply_bc_reproduces_table_solutions_at_first_order(case):
    # Table t:p2: u = 2(1+y)/((3+x)^2+(1+y)^2), f = 0; Table t:p3: u = x^2 + y^2, f = -4; on
    # [-1,1]^2.  The boundary-integral solution with constant elements is first order in h
    # (Sec. 6.2, Fig. f:discretization): the worst node error falls by at least about 2 per
    # halving (midpoint collocation measures close to 4 here).
    if case == "harmonic":
        fn, fval = (lambda x, y: 2 * (1 + y) / ((3 + x) ** 2 + (1 + y) ** 2)), 0.0
    else:
        fn, fval = (lambda x, y: x * x + y * y), -4.0
    errs = []
    for n in (16, 32, 64):
        X, Y, _ = S.grid_coords(n, -1.0, -1.0, 2.0)
        R = O.Problem(n, p=10, x0=-1.0, y0=-1.0, side=2.0)
        u = R.apply_bc(np.full(n * n, fval), _midpoint_data(n, fn, -1.0, -1.0, 2.0), "fmm")
        errs.append(np.max(np.abs(u - fn(X, Y))))
    print(case, "apply_bc max errors", errs)
    assert errs[0] / errs[1] > 1.5 and errs[1] / errs[2] > 1.5
    assert errs[2] < 0.02 * np.max(np.abs(fn(X, Y)))


def test_double_layer_variant_converges_to_the_continuum_and_to_the_single_layer_form():
    # (-1/2 I + K) mu = -(V f)|_Gamma, z = V f + D mu: another boundary correction with the same
    # continuum limit, so P_dl^{-1} f -> u and P_dl^{-1} f - P^{-1} f -> 0 as h -> 0
    e_u, e_sl = [], []
    for n in (16, 32, 64):
        f, u = S.manufactured_sin(n)
        R = O.Problem(n, p=10)
        zdl = R.apply_dl(f, "fmm")
        e_u.append(rel_l2(zdl, u))
        e_sl.append(rel_l2(zdl, R.apply(f, "fmm")))
    print("double-layer variant: vs continuum", e_u, "vs single layer", e_sl)
    assert e_u[0] / e_u[1] > 1.5 and e_u[1] / e_u[2] > 1.5 and e_u[2] < 1e-2
    assert e_sl[0] / e_sl[1] > 1.5 and e_sl[1] / e_sl[2] > 1.5


def test_double_layer_variant_direct_equals_fmm_and_preconditions():
    n = 32
    r = S.random_field(n, 5)
    R = O.Problem(n, p=12)
    assert rel_l2(R.apply_dl(r, "fmm"), R.apply_dl(r, "direct")) < 1e-8
    f = S.gaussian_mixture(n, 2)
    _, it_sl, _, c1 = R.solve(f, "fgmres", 30, 100, 1e-8, "fmm")
    _, it_dl, _, c2 = R.solve(f, "fgmres", 30, 100, 1e-8, "fmm_dl")
    print("fgmres iterations: single layer", it_sl, "double layer", it_dl)
    assert c1 and c2 and abs(it_sl - it_dl) <= 3


# ---------------------------------------------------------------- the transpose of P^{-1}
def test_lu_solves_and_transpose_solves_match_numpy():
    # pins orc_lu / orc_lu_solve_transpose directly (and so the BEM solves)
    rng = np.random.default_rng(8)
    A = rng.standard_normal((40, 40)) + 8 * np.eye(40)
    b = rng.standard_normal(40)
    LU, piv = O.lu(A)
    assert np.max(np.abs(O.lu_solve_transpose(LU, piv, b) - np.linalg.solve(A.T, b))) < 1e-13
    S_, _ = O.bem_matrices(8, 0.0, 0.0, 1.0)
    LU, piv = O.lu(S_)
    assert rel_l2(O.lu_solve_transpose(LU, piv, b[:32]), np.linalg.solve(S_.T, b[:32])) < 1e-12


@pytest.mark.parametrize("n", [8, 16])
def test_transpose_is_the_adjoint_of_the_preconditioner(n):
    # <P^{-1} a, b> = <a, P^{-T} b> for the direct form, to rounding; the FMM forms within
    # the FMM truncation
    rng = np.random.default_rng(n)
    a, b = rng.standard_normal(n * n), rng.standard_normal(n * n)
    R = O.Problem(n, p=12)
    lhs = R.apply(a, "direct") @ b
    rhs = a @ R.apply_transpose(b, "direct")
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # and the dense transpose, column by column
    if n == 8:
        Pm = np.stack([R.apply(e, "direct") for e in np.eye(n * n)], 1)
        assert np.max(np.abs(R.apply_transpose(b, "direct") - Pm.T @ b)) < 1e-12 * np.max(np.abs(Pm.T @ b))
    assert rel_l2(R.apply_transpose(b, "fmm"), R.apply_transpose(b, "direct")) < 1e-8
