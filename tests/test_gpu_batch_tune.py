"""Batched uneven problems and the autotuner (GPU).

The batch of independent grids solved together must give each problem the same
solution and iteration count as its own fmmpc_solve; the autotuner must return a
candidate within its accuracy gate whose solve converges, and its report must cover the
candidate grid (leaf_max x p)."""
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


def test_batched_solve_matches_individual_solves():
    from paper_1308_3339_gb300 import FmmBatch, FmmPreconditioner
    sides = [64, 128, 32, 256, 64]
    fs = [dev(S.gaussian_mixture(n, 1000 + k)) for k, n in enumerate(sides)]
    B = FmmBatch(sides, p=10)
    us, infos = B.solve(fs, rtol=1e-8)
    torch.cuda.synchronize()
    for k, n in enumerate(sides):
        assert infos[k]["status"] == 0 and infos[k]["rel_res"] <= 1e-8
        P = FmmPreconditioner(n, p=10)
        u1, inf1 = P.solve(fs[k], rtol=1e-8)
        assert abs(inf1["iters"] - infos[k]["iters"]) <= 1
        ub = us[k].cpu().numpy()
        check_close(f"batched problem {k} (n={n}) vs single", ub, u1.cpu().numpy(), 1e-7, 1e-7)
        # against the FP64 oracle solved tightly
        xo, *_ = O.Problem(n, p=10).solve(S.gaussian_mixture(n, 1000 + k), "fgmres", rtol=1e-13, prec="fmm")
        check_close(f"batched problem {k} (n={n}) vs oracle", ub, xo, 5e-8, 5e-8)  # measured <= 5.5e-9


def test_autotune_meets_gate_and_reports_all_candidates():
    from paper_1308_3339_gb300 import FmmPreconditioner, autotune
    n = 256
    f = dev(S.gaussian_mixture(n, 7))
    best, rep = autotune(f, n, tol=1e-5)
    assert len(rep) == 12
    assert {(e["leaf_max"], e["p"]) for e in rep} == {(l, p) for l in (16, 64, 256) for p in (6, 8, 10, 12)}
    chosen = [e for e in rep if e["leaf_max"] == best["leaf_max"] and e["p"] == best["p"]][0]
    assert chosen["ok"] and chosen["rel_err"] <= 1e-5
    assert chosen["solve_ms"] == min(e["solve_ms"] for e in rep if e["ok"])
    # higher p never raises the error at a fixed leaf size (geometric decay in p)
    for leaf in (16, 64, 256):
        errs = [e["rel_err"] for e in sorted((e for e in rep if e["leaf_max"] == leaf), key=lambda e: e["p"])]
        assert all(b <= max(a * 1.5, 2e-6) for a, b in zip(errs, errs[1:]))  # FP32 floor ~1e-7
    P = FmmPreconditioner(n, p=best["p"], leaf_max=best["leaf_max"])
    u, info = P.solve(f, rtol=1e-8)
    assert info["status"] == 0


def test_batched_autotuned_create():
    from paper_1308_3339_gb300 import FmmBatch
    sides = [128, 64]
    B = FmmBatch(sides, autotune=True)
    for i in range(len(sides)):
        cfg = B.config(i)
        assert cfg["leaf_side"] in (4, 8, 16) and cfg["p"] in (6, 8, 10, 12)
    us, infos = B.solve([dev(S.gaussian_mixture(n, 5)) for n in sides], rtol=1e-8)
    assert all(i["status"] == 0 for i in infos)
