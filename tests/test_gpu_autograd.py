"""Gradient of the source-inversion loss L(f) = ||u(f) - u_obs||^2, u = A^{-1} f, through
the adjoint FMM-preconditioned solve: against central finite differences of L and against
the oracle's FP64 gradient 2 A^{-1} (u - u_obs), on a 32 x 32 grid."""
import numpy as np
import pytest

import oracle as O
import synth_inputs as S
from conftest import check_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _setup(n=32):
    from paper_1308_3339_gb300 import FmmPreconditioner
    P = FmmPreconditioner(n, p=10, leaf_max=64)
    f_true = S.gaussian_mixture(n, 3)
    R = O.Problem(n, p=10)
    u_true, *_ = R.solve(f_true, "fgmres", rtol=1e-13, prec="fmm")
    u_obs = u_true + np.random.default_rng(7).normal(0.0, 0.01, n * n)
    return P, R, u_obs


def test_gradient_matches_finite_differences():
    from paper_1308_3339_gb300.autograd import fmm_solve
    n = 32
    P, R, u_obs = _setup(n)
    uo = torch.tensor(u_obs, dtype=torch.float64, device="cuda")
    f0 = torch.tensor(S.gaussian_mixture(n, 5), dtype=torch.float64, device="cuda", requires_grad=True)

    def loss(f):
        u = fmm_solve(f, P, rtol=1e-13, maxit=300)
        return ((u - uo) ** 2).sum()

    L = loss(f0)
    L.backward()
    g = f0.grad.detach().cpu().numpy()
    rng = np.random.default_rng(1)
    delta = 1e-4 * float(f0.detach().abs().max())
    for _ in range(3):
        d = rng.standard_normal(n * n)
        d /= np.linalg.norm(d)
        dt = torch.tensor(d, dtype=torch.float64, device="cuda")
        with torch.no_grad():
            fd = (loss(f0 + delta * dt) - loss(f0 - delta * dt)).item() / (2 * delta)
        assert abs(fd - g @ d) <= 1e-6 * max(abs(fd), 1e-30) + 1e-12 * np.linalg.norm(g)


def test_gradient_matches_oracle_fp64():
    from paper_1308_3339_gb300.autograd import fmm_solve
    n = 32
    P, R, u_obs = _setup(n)
    f = S.gaussian_mixture(n, 5)
    ft = torch.tensor(f, dtype=torch.float64, device="cuda", requires_grad=True)
    u = fmm_solve(ft, P, rtol=1e-13, maxit=300)
    ((u - torch.tensor(u_obs, device="cuda")) ** 2).sum().backward()
    u_o, *_ = R.solve(f, "fgmres", rtol=1e-13, prec="fmm")
    g_o, *_ = R.solve(2.0 * (u_o - u_obs), "fgmres", rtol=1e-13, prec="fmm")
    g = ft.grad.cpu().numpy()
    check_close("autograd gradient n=32 vs oracle", g, g_o, 1e-9, 1e-9)
