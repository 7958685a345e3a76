"""The multi-right-hand-side configuration at full size: 4096 x 4096 interior nodes
(16.8M), 32 right-hand sides of seeded Gaussian mixtures, p = 10, the mixed form with the
M2L on the tensor cores and FP64 Krylov around it.

The oracle's full FMM at this size needs the dense LU of the N_Gamma = 16384 boundary
matrix, so the checks sample outputs the oracle computes one by one: every right-hand side
of the batch equals its own single-right-hand-side apply bit for bit (each is an independent
slice of every kernel); V r at sampled nodes and at sampled collocation points matches the
oracle's direct sum; the GPU's boundary density q satisfies the boundary system
S q = -(V r)|_Gamma of Eq. e:ubound at sampled rows of S formed by the oracle; and z at
sampled nodes equals the oracle's direct V r plus the single layer of that q (Eq. e:uinter),
which checks the boundary tree, the boundary-to-volume M2L at L = 9 and the near-boundary
element integrals.  The tensor-core kernels must report no bounded wait that gave up."""
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
    rng = np.random.default_rng(1)
    idx = rng.choice(n * n, 96, replace=False).astype(np.int32)
    # nodes within two leaves of the boundary, where the boundary correction is largest
    band = np.concatenate([rng.integers(0, n, 16) + n * rng.integers(0, 16, 16),
                           rng.integers(0, 16, 16) + n * rng.integers(0, n, 16)]).astype(np.int32)
    rows = rng.choice(4 * n, 64, replace=False).astype(np.int32)
    Srows, _ = O.bem_rows(n, 0.0, 0.0, 1.0, rows)
    _, _, _, _, cx, cy = O.elements(n, 0.0, 0.0, 1.0)
    h = 1.0 / (n + 1)
    for k in (0, R - 1):
        rk = rd[k].contiguous()
        vr = P.apply_part("vr", rk).cpu().numpy()
        vcol = P.apply_part("vcol", rk).cpu().numpy()[0]
        q = P.apply_part("q", rk).cpu().numpy()[0]
        check_close(f"C3 vr rhs{k} (96 nodes) vs direct", vr[idx], O.direct_V_nodes(n, 0.0, 0.0, 1.0, rs[k], idx),
                    1e-5, 1e-5)
        check_close(f"C3 vcol rhs{k} (64 points) vs direct", vcol[rows],
                    O.direct_V_at(n, 0.0, 0.0, 1.0, rs[k], cx[rows], cy[rows]), 1e-5, 1e-5)
        # S q + vcol = 0 at the sampled rows, relative to |vcol|
        check_close(f"C3 BEM system rhs{k} (64 rows)", Srows @ q, -vcol[rows], 1e-10, 1e-10)  # measured 4e-12
        sel = np.concatenate([idx, band])
        zk = z[k].cpu().numpy()[sel]
        sl, _ = O.layers_at(n, 0.0, 0.0, 1.0, (sel % n + 1) * h, (sel // n + 1) * h, q=q)
        check_close(f"C3 z rhs{k} (128 nodes) vs direct V r + single layer of q", zk,
                    O.direct_V_nodes(n, 0.0, 0.0, 1.0, rs[k], sel) + sl, 1e-5, 1e-5)
    assert bool(torch.isfinite(z).all())


def test_64_uneven_problems_batched():
    # 64 grids with sides drawn from {128, 256, 512, 1024, 2048} (seed 0), each with its own
    # Gaussian mixture (seed 1000 + k), solved together by FGMRES(30) in one CUDA graph
    # (one chain per problem, each stopping at its own convergence), mixed TF32
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
        check_close(f"C4 problem {k} batched vs single", us[k].cpu().numpy(), u1.cpu().numpy(), 1e-7, 1e-7)
        P.close()
    k = int(np.argmin(sides))
    xo, *_ = O.Problem(sides[k], p=10).solve(S.gaussian_mixture(sides[k], 1000 + k), "fgmres", rtol=1e-12,
                                              prec="fmm")
    # ours stops at 1e-8, the oracle at 1e-12
    check_close(f"C4 problem {k} vs oracle", us[k].cpu().numpy(), xo, 5e-8, 5e-8)
    B.close()
