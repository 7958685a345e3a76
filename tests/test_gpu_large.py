"""The multi-right-hand-side configuration at full size: 4096 x 4096 interior nodes
(16.8M), 32 right-hand sides of seeded Gaussian mixtures, p = 10, the mixed form with the
M2L on the tensor cores and FP64 Krylov around it.

The oracle's full FMM at this size takes minutes per right-hand side, so the checks are:
every right-hand side of the batch equals its own single-right-hand-side apply bit for bit
(each is an independent slice of every kernel); V r at sampled nodes matches the oracle's
direct sum within the FP32 gate; and the tensor-core kernels report no bounded wait that
gave up."""
import numpy as np
import pytest

import oracle as O
import synth_inputs as S
from conftest import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_4096_with_32_right_hand_sides():
    from paper_1308_3339_gb300 import FmmPreconditioner
    n, R = 4096, 32
    rs = np.stack([S.gaussian_mixture(n, k) for k in range(R)])
    P = FmmPreconditioner(n, p=10, n_rhs=R, precision="mixed_tf32")
    assert P.query("tc_m2l") == 1 and P.query("tc_p2p") == 1
    rd = torch.tensor(rs, dtype=torch.float64, device="cuda")
    z = P.apply(rd)
    torch.cuda.synchronize()
    assert P.query("device_errors") == 0
    for k in (0, R - 1):
        zk = P.apply(rd[k].contiguous())
        torch.cuda.synchronize()
        assert torch.equal(z[k], zk)
    idx = np.random.default_rng(1).choice(n * n, 96, replace=False).astype(np.int32)
    for k in (0, R - 1):
        vr = P.apply_part("vr", rd[k].contiguous())
        torch.cuda.synchronize()
        assert rel_l2(vr.cpu().numpy()[idx], O.direct_V_nodes(n, 0.0, 0.0, 1.0, rs[k], idx)) < 1e-5
    assert bool(torch.isfinite(z).all())


def test_64_uneven_problems_batched():
    # 64 grids with sides drawn from {128, 256, 512, 1024, 2048} (seed 0), each with its own
    # Gaussian mixture (seed 1000 + k), solved together by lockstep FGMRES(30), mixed TF32
    from paper_1308_3339_gb300 import FmmBatch, FmmPreconditioner
    sides = [int(v) for v in S.batched_sides(0, 64)]
    assert sum(n * n for n in sides) > 5e7
    fs = [torch.tensor(S.gaussian_mixture(n, 1000 + k), dtype=torch.float64, device="cuda")
          for k, n in enumerate(sides)]
    B = FmmBatch(sides, p=10, precision="mixed_tf32")
    us, infos = B.solve(fs, rtol=1e-8)
    torch.cuda.synchronize()
    assert all(i["status"] == 0 and i["rel_res"] <= 1e-8 for i in infos)
    for k in (int(np.argmin(sides)), int(np.argmax(sides))):
        P = FmmPreconditioner(sides[k], p=10, precision="mixed_tf32")
        u1, inf1 = P.solve(fs[k], rtol=1e-8)
        assert abs(inf1["iters"] - infos[k]["iters"]) <= 1
        assert rel_l2(us[k].cpu().numpy(), u1.cpu().numpy()) < 1e-7
        P.close()
    k = int(np.argmin(sides))
    xo, *_ = O.Problem(sides[k], p=10).solve(S.gaussian_mixture(sides[k], 1000 + k), "fgmres", rtol=1e-12,
                                              prec="fmm")
    assert rel_l2(us[k].cpu().numpy(), xo) < 1e-6  # ours stops at 1e-8, the oracle at 1e-12
    B.close()
