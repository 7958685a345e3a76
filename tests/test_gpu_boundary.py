"""Boundary data and the double-layer correction on the GPU against the oracle.

fmmpc_apply_bc: the boundary-integral solution of -lap u = f, u = g (Sec. 4.1, Eq. e:ubound
with its (1/2 I + K) g term, Eq. e:uinter with its -D g term).  The oracle evaluates the
boundary integrals in closed form and sums them directly; the GPU takes the far part of
both layers through the boundary FMM tree (the double layer as complex point weights at
the element ends), so the FP64 form agrees to the FMM truncation (p = 10), the single-
precision forms to the FP32 bar.  Tables t:p2 (harmonic u) and t:p3 (u = x^2 + y^2) are
reproduced at (at least) first order in h.

fmmpc_set_bem_form(DOUBLE_LAYER): the second-kind correction (-1/2 I + K) mu = -(V r)|_Gamma,
z = V r + D mu, against the oracle's, and as a preconditioner inside FGMRES (iterations
within one of the oracle's, in the host-driven and the graph solve)."""
import numpy as np
import pytest

import oracle as O
import synth_inputs as S
from conftest import check_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = {"fp64": 1e-7, "fp32": 1e-5, "mixed_tf32": 3e-5}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda").contiguous()


def midpoint_data(n, fn, x0=0.0, y0=0.0, side=1.0):
    _, _, _, _, cx, cy = O.elements(n, x0, y0, side)
    return fn(cx, cy)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed_tf32"])
@pytest.mark.parametrize("n,leaf_max", [(64, 64), (128, 64), (64, 16)])
def test_apply_bc_matches_oracle(prec, n, leaf_max):
    from paper_1308_3339_gb300 import FmmPreconditioner
    f = S.gaussian_mixture(n, 30)
    g = midpoint_data(n, lambda x, y: np.cos(3 * x) * np.exp(y) + x * y)
    P = FmmPreconditioner(n, p=10, leaf_max=leaf_max, precision=prec)
    u = P.apply_bc(dev(f), dev(g)).cpu().numpy()
    uo = O.Problem(n, p=10, leaf_max=leaf_max).apply_bc(f, g, "fmm")
    tol = GATE[prec]
    check_close(f"apply_bc {prec} n={n} leaf={leaf_max}", u, uo, tol, tol)
    # with g = 0 it is the preconditioner itself
    z0 = P.apply_bc(dev(f), dev(np.zeros(4 * n))).cpu().numpy()
    check_close(f"apply_bc g=0 vs apply {prec} n={n}", z0, P.apply(dev(f)).cpu().numpy(), 1e-6 if prec != "fp64" else 1e-12,
                1e-6 if prec != "fp64" else 1e-12)


@pytest.mark.parametrize("case", ["harmonic", "quadratic"])
def test_apply_bc_reproduces_tables_t_p2_t_p3(case):
    from paper_1308_3339_gb300 import FmmPreconditioner
    if case == "harmonic":
        fn, fval = (lambda x, y: 2 * (1 + y) / ((3 + x) ** 2 + (1 + y) ** 2)), 0.0
    else:
        fn, fval = (lambda x, y: x * x + y * y), -4.0
    errs = []
    for n in (32, 64, 128):
        X, Y, _ = S.grid_coords(n, -1.0, -1.0, 2.0)
        g = midpoint_data(n, fn, -1.0, -1.0, 2.0)
        P = FmmPreconditioner(n, p=10, precision="mixed_tf32", x0=-1.0, y0=-1.0, side=2.0)
        u = P.apply_bc(dev(np.full(n * n, fval)), dev(g)).cpu().numpy()
        uo = O.Problem(n, p=10, x0=-1.0, y0=-1.0, side=2.0).apply_bc(np.full(n * n, fval), g, "fmm")
        check_close(f"apply_bc table {case} n={n} vs oracle", u, uo, 3e-5, 3e-5)
        errs.append(np.max(np.abs(u - fn(X, Y))))
        P.close()
    print(f"apply_bc {case}: max errors against the exact solution {errs}")
    assert errs[0] / errs[1] > 1.5 and errs[1] / errs[2] > 1.5


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed_tf32"])
@pytest.mark.parametrize("n", [64, 256])
def test_double_layer_form_matches_oracle(prec, n):
    from paper_1308_3339_gb300 import FmmPreconditioner
    r = S.random_field(n, 44)
    P = FmmPreconditioner(n, p=10, precision=prec)
    P.set_bem_form("double_layer")
    rd = dev(r)
    z = P.apply(rd).cpu().numpy()
    mu = P.apply_part("q", rd).cpu().numpy()[0]
    zo, muo = O.Problem(n, p=10).apply_dl(r, "fmm", with_mu=True)
    tol = GATE[prec]
    check_close(f"double-layer z {prec} n={n}", z, zo, tol, tol)
    check_close(f"double-layer mu {prec} n={n}", mu, muo, 10 * tol, 10 * tol)
    assert P.query("device_errors") == 0


@pytest.mark.parametrize("graphs", [0, 2])
def test_double_layer_form_preconditions_fgmres(graphs):
    from paper_1308_3339_gb300 import FmmPreconditioner
    n = 128
    f = S.gaussian_mixture(n, 8)
    P = FmmPreconditioner(n, p=10, precision="mixed_tf32")
    P.set_bem_form("double_layer")
    u, info = P.solve(dev(f), rtol=1e-8, use_graphs=graphs)
    R = O.Problem(n, p=10)
    _, it_o, _, _ = R.solve(f, "fgmres", 30, 100, 1e-8, "fmm_dl")
    print(f"ITERS double-layer fgmres graphs={graphs}: gpu {info['iters']} oracle {it_o}")
    assert info["status"] == 0 and abs(info["iters"] - it_o) <= 1
    u10, _ = P.solve(dev(f), rtol=1e-11, use_graphs=graphs)
    x10, *_ = R.solve(f, "fgmres", 30, 100, 1e-11, "fmm_dl")
    check_close(f"double-layer fgmres solution graphs={graphs}", u10.cpu().numpy(), x10, 1e-8, 1e-8)
    P.set_bem_form("single_layer")
    _, info_sl = P.solve(dev(f), rtol=1e-8, use_graphs=graphs)
    assert abs(info_sl["iters"] - info["iters"]) <= 3
