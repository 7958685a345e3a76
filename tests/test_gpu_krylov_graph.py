"""The whole Krylov solve as one CUDA graph (fmmpc_solve_opts.use_graphs = 2): set-up,
a conditional WHILE loop of Arnoldi steps (or CG iterations) whose convergence test,
Givens rotations and back substitution run on the device, and the final true residual.
It must follow the host-driven loop (use_graphs = 0) of the same method: the same
iteration counts within one (the graph form always orthogonalises twice, the host form
only when cancellation is detected), solutions within the solve tolerance of each other,
the same status codes, every right-hand side of a batch handled, and a loop that stops at
maxit or on a NaN."""
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


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float64, device="cuda").contiguous()


# restart 40 takes the unfused orthogonalisation (the fused kernels hold 32 basis vectors)
@pytest.mark.parametrize("method,prec,restart", [("fgmres", "mixed_tf32", 30), ("fgmres", "fp32", 4),
                                                 ("gmres", "fp64", 30), ("cg", "fp32", 30),
                                                 ("fgmres", "mixed_bf16", 40)])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_graph_solve_follows_host_loop(method, prec, restart, nrhs):
    from paper_1308_3339_gb300 import FmmPreconditioner
    n = 128
    fs = np.stack([S.gaussian_mixture(n, 60 + k) for k in range(nrhs)])
    P = FmmPreconditioner(n, p=10, precision=prec, n_rhs=nrhs)
    f = dev(fs if nrhs > 1 else fs[0])
    u0, i0 = P.solve(f, method=method, restart=restart, rtol=1e-9, use_graphs=0)
    u2, i2 = P.solve(f, method=method, restart=restart, rtol=1e-9, use_graphs=2)
    u2b, i2b = P.solve(f, method=method, restart=restart, rtol=1e-9, use_graphs=2)  # replay
    torch.cuda.synchronize()
    print(f"ITERS graph-vs-host {method} {prec} m={restart} nrhs={nrhs}: host {i0['iters']} graph {i2['iters']}")
    assert i0["status"] == 0 and i2["status"] == 0 and i2["rel_res"] <= 1e-9
    assert abs(i0["iters"] - i2["iters"]) <= 1
    assert torch.equal(u2, u2b) and i2b["iters"] == i2["iters"]
    check_close(f"graph vs host solve {method} {prec} nrhs={nrhs}", u2.cpu().numpy(), u0.cpu().numpy(), 1e-7, 1e-7)
    P.close()


def test_graph_solve_matches_oracle_and_closed_form():
    from paper_1308_3339_gb300 import FmmPreconditioner
    n = 64
    f, u = S.manufactured_sin(n)
    h = 1 / 65
    lam = 8 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    P = FmmPreconditioner(n, p=8, precision="mixed_tf32")
    x, info = P.solve(dev(f), method="fgmres", rtol=1e-8, use_graphs=2)
    _, it_o, _, _ = O.Problem(n, p=8).solve(f, "fgmres", 30, 100, 1e-8, "fmm")
    assert info["status"] == 0 and abs(info["iters"] - it_o) <= 1
    check_close("graph fgmres n=64 vs closed form", x.cpu().numpy(), (2 * np.pi ** 2 / lam) * u, 1e-7, 1e-7)


def test_graph_solve_stops_at_maxit_and_on_nan():
    from paper_1308_3339_gb300 import FmmPreconditioner
    n = 64
    P = FmmPreconditioner(n, p=8)
    f = dev(S.gaussian_mixture(n, 1))
    for method in ("fgmres", "cg"):
        _, info = P.solve(f, method=method, maxit=2, rtol=1e-14, use_graphs=2, raise_on_fail=False)
        assert info["status"] == -4 and info["iters"] == 2
    from paper_1308_3339_gb300 import FmmpcError
    for method in ("fgmres", "cg"):
        # an exact initial iterate needs no iteration
        u, info = P.solve(f, method=method, rtol=1e-8, use_graphs=2)
        _, info2 = P.solve(f, method=method, u0=u, rtol=1e-6, use_graphs=2)
        assert info2["status"] == 0 and info2["iters"] == 0
        bad = S.gaussian_mixture(n, 1)
        bad[100] = np.nan
        with pytest.raises(FmmpcError):
            P.solve(dev(bad), method=method, rtol=1e-8, use_graphs=2)
        _, info3 = P.solve(f, method=method, rtol=1e-8, use_graphs=2)  # the handle still works afterwards
        assert info3["status"] == 0


@pytest.mark.parametrize("method", ["fgmres", "cg"])
def test_graph_solve_right_hand_side_done_at_set_up(method):
    # a zero right-hand side is done before the first iteration; its neighbours in the
    # batch must still converge, to the same solutions as when solved alone
    from paper_1308_3339_gb300 import FmmPreconditioner
    n = 64
    fs = np.stack([S.gaussian_mixture(n, 7), np.zeros(n * n), S.gaussian_mixture(n, 8)])
    P = FmmPreconditioner(n, p=8, precision="fp32", n_rhs=3)
    u, info = P.solve(dev(fs), method=method, rtol=1e-9, use_graphs=2)
    assert info["status"] == 0 and info["rel_res"] <= 1e-9
    un = u.cpu().numpy().reshape(3, -1)
    assert np.all(un[1] == 0.0)
    for k in (0, 2):
        P1 = FmmPreconditioner(n, p=8, precision="fp32")
        u1, i1 = P1.solve(dev(fs[k]), method=method, rtol=1e-9, use_graphs=2)
        check_close(f"graph {method} rhs {k} in a batch with a zero rhs", un[k], u1.cpu().numpy(), 1e-7, 1e-7)
        P1.close()
    P.close()


def test_graph_solve_with_boundary_data():
    # u = x^2 + y^2, f = -4 (Table t:p3's problem): the FD solution is exact
    from paper_1308_3339_gb300 import FmmPreconditioner
    n = 64
    X, Y, h = S.grid_coords(n, -1.0, -1.0, 2.0)
    g = S.boundary_values(n, lambda x, y: x * x + y * y, -1.0, -1.0, 2.0)
    P = FmmPreconditioner(n, p=10, x0=-1.0, y0=-1.0, side=2.0)
    x, info = P.solve(dev(-4.0 * np.ones(n * n)), g=dev(g), rtol=1e-12, maxit=100, use_graphs=2)
    check_close("graph solve x^2+y^2", x.cpu().numpy(), X ** 2 + Y ** 2, 1e-10, 1e-10)
