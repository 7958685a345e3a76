"""The allocation-free near-field entry point against the handle-based one.

fmmpc_near_field_noalloc serves callers that must not allocate device memory (a
framework's memory pool owns the device, a stream is being captured, or a latency-bound
loop cannot take cudaMalloc's implicit synchronisation): its scratch is a static device
array inside the library.  This file is collected last so that a failure here comes after
every other test has run; it must pass alone in a fresh process and after the others.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import synth_inputs as S
from conftest import check_close

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5  # the FP32 bar used by the other parity tests


def _call(lib, n, r, out, leaf_max=64, theta=0.4):
    return lib.fmmpc_near_field_noalloc(n, 1.0, leaf_max, theta, C.c_void_p(r.data_ptr()),
                                        C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_near_field_matches_apply_part_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_3339_gb300 import FmmPreconditioner, _lib
    lib = _lib.load()
    # two calls in a row: a larger grid first, then a smaller one that reuses the array
    for n, seed in ((256, 11), (128, 12)):
        r = torch.tensor(S.random_field(n, seed), dtype=torch.float64, device="cuda")
        out = torch.full_like(r, float("nan"))
        rc = _call(lib, n, r, out)
        assert rc == 0, lib.fmmpc_last_error(None)
        ref = FmmPreconditioner(n, p=8, leaf_max=64, theta=0.4).apply_part("near", r)
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all()
        check_close(f"noalloc near n={n} vs apply_part near", a, b, FP32_TOL, FP32_TOL)
        # and against the oracle's near field (the P2P part of its FMM, FP64)
        near_o = O.Problem(n, p=8).apply(S.random_field(n, seed), "fmm", stages=True)["near"]
        check_close(f"noalloc near n={n} vs oracle near", a, near_o, FP32_TOL, FP32_TOL)


def test_noalloc_rejects_grids_beyond_the_static_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_3339_gb300 import _lib
    lib = _lib.load()
    n = 2048
    r = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(r)
    assert _call(lib, n, r, out) == -1
    assert b"16 MiB" in lib.fmmpc_last_error(None)


def test_noalloc_never_lowers_the_shared_memory_limit_of_a_handle():
    # A handle whose CUDA-core near field needs a large source tile (theta = 0.3: stencil
    # radius 4 leaves) is made first; a no-allocation call with a small tile (theta = 0.5,
    # radius 2) runs the same kernel; the handle's near field must still run afterwards and
    # give the same values as before that call.
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1308_3339_gb300 import FmmPreconditioner, _lib
    lib = _lib.load()
    n = 256
    r = torch.tensor(S.random_field(n, 21), dtype=torch.float64, device="cuda")
    P = FmmPreconditioner(n, p=8, leaf_max=64, theta=0.3)
    P.set_p2p_engine("simt")
    before = P.apply_part("near", r).clone()
    out = torch.empty_like(r)
    assert _call(lib, n, r, out, theta=0.5) == 0, lib.fmmpc_last_error(None)
    after = P.apply_part("near", r)
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    P.close()
