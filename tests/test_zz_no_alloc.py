"""rlobpcg_gram_noalloc: the Gram pass for callers that cannot let the library allocate.

A serving process that has budgeted all of HBM at start-up, or a loop that must not call
cudaMalloc/cudaFree (they synchronise the whole device), cannot hand the library a workspace
or let it allocate one. The allocation-free entry point keeps its split-m scratch in a fixed
device buffer inside the library. These tests call it through the C ABI and check that two
calls in a row (different inputs, so the second cannot pass by reusing the first one's scratch)
give the same results as rlobpcg_gram with a caller-provided workspace, within the bounds the
other Gram tests use, that warm calls leave the device's free memory and torch's reserved pool
unchanged, and that an oversized problem is refused cleanly.

The file sorts last so that a run stopping at the first failure has already run everything else.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_16797_gb300 import rlobpcg as rl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _run(A, W, noalloc):
    m, n = A.shape
    b = W.shape[1]
    dt = rl.RLOBPCG_C128 if np.iscomplexobj(A) else rl.RLOBPCG_F64
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    Wd = torch.from_numpy(np.ascontiguousarray(W)).cuda()
    AW = torch.empty((m, b), dtype=Ad.dtype, device="cuda")
    G = torch.empty((n, b), dtype=Ad.dtype, device="cuda")
    if noalloc:
        rl.rlobpcg_gram_noalloc(Ad.data_ptr(), m, n, n, dt, Wd.data_ptr(), b, b, AW.data_ptr(), b, G.data_ptr(), b,
                                _stream())
    else:
        ws = rl.rlobpcg_gram_workspace_size(m, n, b, dt)
        work = torch.empty(max(ws, 16), dtype=torch.uint8, device="cuda")
        rl.rlobpcg_gram(Ad.data_ptr(), m, n, n, dt, Wd.data_ptr(), b, b, AW.data_ptr(), b, G.data_ptr(), b,
                        work.data_ptr(), ws, _stream())
    torch.cuda.synchronize()
    return AW.cpu().numpy(), G.cpu().numpy()


def _bounds(A, W, AW):
    """Componentwise dot-product error bounds of A W and A^H (A W) (as in the other Gram tests)."""
    m, n = A.shape
    f = 4.0 if np.iscomplexobj(A) else 1.0
    absA = np.abs(A)
    b1 = f * (n + 2) * U * (absA @ np.abs(W))
    b2 = absA.T @ b1 + f * (m + 2) * U * (absA.T @ np.abs(AW))
    return b1, b2


@pytest.mark.parametrize("m,n,b,cplx", [(50_000, 500, 5, False), (7_001, 301, 3, True), (4_000, 50, 1, False)])
def test_noalloc_matches_gram_on_two_consecutive_calls(m, n, b, cplx):
    rng = np.random.default_rng(m + n + b)
    for call in range(2):
        A = rng.standard_normal((m, n))
        W = rng.standard_normal((n, b))
        if cplx:
            A = A + 1j * rng.standard_normal((m, n))
            W = W + 1j * rng.standard_normal((n, b))
        AW1, G1 = _run(A, W, noalloc=True)
        AW0, G0 = _run(A, W, noalloc=False)
        b1, b2 = _bounds(A, W, AW0)
        assert np.all(np.abs(AW1 - AW0) <= b1), f"call {call}: A W differs"
        assert np.all(np.abs(G1 - G0) <= b2), f"call {call}: A^H A W differs"


def test_noalloc_refuses_problems_beyond_its_buffer():
    """A problem whose partials exceed the fixed buffer is refused before any device work (the
    tiny placeholder buffers below are never touched)."""
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    m, n, b = 10_000_000, 4000, 20
    rc = rl.load().rlobpcg_gram_noalloc(p, m, n, n, rl.RLOBPCG_F64, p, b, b, p, b, p, b, None)
    assert rc == rl.RLOBPCG_ERR_UNSUPPORTED
    assert "16 MiB" in rl.rlobpcg_last_error()
    assert rl.load().rlobpcg_gram_noalloc(None, 10, 10, 10, 0, p, 1, 1, p, 1, p, 1, None) == rl.RLOBPCG_ERR_INVALID_ARG


def test_noalloc_calls_leave_device_memory_unchanged():
    """After one warm-up call (which may load the kernels), further calls allocate nothing: the
    driver's free-memory count and torch's reserved pool are the same before and after them."""
    rng = np.random.default_rng(5)
    m, n, b = 20_000, 200, 4
    Ad = torch.from_numpy(rng.standard_normal((m, n))).cuda()
    Wd = torch.from_numpy(rng.standard_normal((n, b))).cuda()
    AW = torch.empty((m, b), dtype=torch.float64, device="cuda")
    G = torch.empty((n, b), dtype=torch.float64, device="cuda")

    def call():
        rl.rlobpcg_gram_noalloc(Ad.data_ptr(), m, n, n, rl.RLOBPCG_F64, Wd.data_ptr(), b, b, AW.data_ptr(), b,
                                G.data_ptr(), b, _stream())

    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(4):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0
