"""The full apply forks the tensor-core near field, the volume M2L and the near-boundary
correction onto three further streams (in the captured graph and in eager mode alike) and
joins them before the downward pass; with stage timing on it runs every stage on one stream
in order.  Every kernel computes the same sums either way (the two parts of a split M2L
tile add onto zeros, which is order-independent), so the results must be bitwise equal: a
missing dependency between the streams would show as a difference, or as a run-to-run
change."""
import numpy as np
import pytest

import synth_inputs as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("prec,n,nrhs", [("mixed_tf32", 256, 1), ("mixed_bf16", 512, 3), ("fp32", 256, 2)])
def test_overlapped_apply_equals_serial_apply(prec, n, nrhs):
    from paper_1308_3339_gb300 import FmmPreconditioner
    rs = np.stack([S.gaussian_mixture(n, 40 + k) for k in range(nrhs)])
    rd = torch.tensor(rs if nrhs > 1 else rs[0], dtype=torch.float64, device="cuda").contiguous()
    P = FmmPreconditioner(n, p=10, n_rhs=nrhs, precision=prec)
    P.set_timing(1)  # one stream, stages in order
    z_serial = P.apply(rd).clone()
    P.set_timing(0)
    outs = []
    for graphs in (True, False, True):
        P.set_graphs(graphs)
        for _ in range(2):
            outs.append(P.apply(rd).clone())
    torch.cuda.synchronize()
    assert P.query("device_errors") == 0
    for z in outs:
        assert torch.equal(z, z_serial)
    assert bool(torch.isfinite(z_serial).all())
    P.close()
