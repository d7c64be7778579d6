"""The split-bf16 Gram pass for complex128 A (rlobpcg_gram_split_c128) against the oracle's
products, and complex solves on it against the oracle.

The pass runs the real tensor-core pass on the real view B of A (m x 2n, interleaved Re/Im) with
each entry w of W expanded to the 2 x 2 block [Re w, Im w; -Im w, Re w]. Its bounds are therefore
the real pass's bounds (tests/test_gpu_split_gram.py) for B and that expanded W, entry by entry of
the real view of A W, and for G = A^H A W the sum of the two real bounds that make up each of
Re G and Im G plus one FP64 rounding of their sum.
"""
import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl
from tests.parity import check_sigma, check_truth
from tests.test_gpu_split_gram import bounds

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def split_gram_c(A, W, ldaw=None, ldg=None):
    """AW, G through the C ABI: prepare on the real view, one complex pass."""
    m, n = A.shape
    b = W.shape[1]
    ldaw = ldaw or b
    ldg = ldg or b
    Ad, Wd = _dev(A), _dev(W)
    ps = rl.rlobpcg_gram_split_prepare_size(m, 2 * n)
    ws = rl.rlobpcg_gram_split_c128_workspace_size(m, n, b)
    prep = torch.empty(ps, dtype=torch.uint8, device="cuda")
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    nan = complex(np.nan, np.nan)
    AW = torch.full((m, ldaw), nan, dtype=torch.complex128, device="cuda")
    G = torch.full((n, ldg), nan, dtype=torch.complex128, device="cuda")
    rl.rlobpcg_gram_split_prepare(Ad.data_ptr(), m, 2 * n, 2 * n, prep.data_ptr(), ps, _stream())
    rl.rlobpcg_gram_split_c128(prep.data_ptr(), m, n, Wd.data_ptr(), b, b, AW.data_ptr(), ldaw, G.data_ptr(), ldg,
                               work.data_ptr(), ws, _stream())
    torch.cuda.synchronize()
    AW, G = AW.cpu().numpy(), G.cpu().numpy()
    # columns beyond b are never written
    assert np.all(np.isnan(AW[:, b:].real)) and np.all(np.isnan(G[:, b:].real))
    return AW[:, :b], G[:, :b]


def _blocks(W):
    n, b = W.shape
    Wr = np.empty((2 * n, 2 * b))
    Wr[0::2, 0::2] = W.real
    Wr[0::2, 1::2] = W.imag
    Wr[1::2, 0::2] = -W.imag
    Wr[1::2, 1::2] = W.real
    return Wr


def _real_view(X):
    return np.ascontiguousarray(X).view(np.float64)


def check_against_oracle(A, W, **kw):
    AW, G = split_gram_c(A, W, **kw)
    AW0, G0 = oracle.gram_pass(A, W)
    B, Wr, Y0 = _real_view(A), _blocks(W), _real_view(AW0)
    tY, tGr = bounds(B, Wr, Y0)
    aGp = np.abs(B).T @ (np.abs(Y0) + tY)          # bounds |entries| of the real products B^T Y
    tre = tGr[0::2, 0::2] + tGr[1::2, 1::2] + U * (aGp[0::2, 0::2] + aGp[1::2, 1::2])
    tim = tGr[0::2, 1::2] + tGr[1::2, 0::2] + U * (aGp[0::2, 1::2] + aGp[1::2, 0::2])
    eY = np.abs(_real_view(AW) - Y0)
    assert np.all(eY <= tY), (np.max(eY / tY), np.unravel_index(np.argmax(eY / tY), eY.shape))
    ere, eim = np.abs(G.real - G0.real), np.abs(G.imag - G0.imag)
    assert np.all(ere <= tre), np.max(ere / tre)
    assert np.all(eim <= tim), np.max(eim / tim)
    return AW, G, AW0, G0


def _crand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_gaussian_integers_give_exact_products():
    # Re and Im with at most 10 significant bits: every real product of the pass is exact in
    # FP64 and held in two digits, so A W is bit-exact; G = A^H (A W) within the pass's bound
    rng = np.random.default_rng(11)
    m, n, b = 2500, 300, 5
    A = rng.integers(-512, 513, (m, n)) + 1j * rng.integers(-512, 513, (m, n))
    W = rng.integers(-512, 513, (n, b)) + 1j * rng.integers(-512, 513, (n, b))
    AW, G = split_gram_c(A, W)
    Ai = (A.real.astype(np.int64), A.imag.astype(np.int64))
    Wi = (W.real.astype(np.int64), W.imag.astype(np.int64))
    re = Ai[0] @ Wi[0] - Ai[1] @ Wi[1]
    im = Ai[0] @ Wi[1] + Ai[1] @ Wi[0]
    assert np.array_equal(AW.real, re.astype(np.float64)) and np.array_equal(AW.imag, im.astype(np.float64))
    gre = Ai[0].T @ re + Ai[1].T @ im                # conj(A)^T Z, exact in int64 (|.| < 2^53)
    gim = Ai[0].T @ im - Ai[1].T @ re
    tol = 64 * U * (np.abs(A).T @ np.abs(AW)) * 2
    assert np.all(np.abs(G.real - gre) <= tol) and np.all(np.abs(G.imag - gim) <= tol)


@pytest.mark.parametrize("m,n,b", [(1, 1, 1), (129, 17, 2), (2999, 300, 3), (4097, 500, 4), (3000, 257, 6),
                                   (1500, 64, 8), (2000, 130, 12)])
def test_products_against_oracle(m, n, b):
    rng = np.random.default_rng(m * 3 + n + b)
    check_against_oracle(_crand(rng, (m, n)), _crand(rng, (n, b)))


def test_leading_dimensions_and_scaled_rows():
    rng = np.random.default_rng(12)
    m, n, b = 1700, 150, 5
    A = _crand(rng, (m, n)) * np.exp2(rng.integers(-200, 201, (m, 1)))
    W = _crand(rng, (n, b)) * np.exp2(np.array([-100, -20, 0, 30, 150]))[None, :]
    check_against_oracle(A, W, ldaw=3 * b, ldg=3 * b + 1)


def test_purely_real_and_purely_imaginary():
    rng = np.random.default_rng(13)
    m, n, b = 1200, 90, 3
    Ar = rng.standard_normal((m, n)).astype(np.complex128)
    W = _crand(rng, (n, b))
    AW, G, AW0, G0 = check_against_oracle(Ar, W)
    check_against_oracle(1j * Ar, W)
    check_against_oracle(_crand(rng, (m, n)), 1j * rng.standard_normal((n, b)))


def test_workspace_and_block_limits():
    assert rl.rlobpcg_gram_split_c128_workspace_size(100, 10, 13) == 0
    assert rl.rlobpcg_gram_split_c128_workspace_size(100, 10, 12) > 0
    m, n = 300, 40
    A = _dev(np.ones((m, n), dtype=np.complex128))
    ps = rl.rlobpcg_gram_split_prepare_size(m, 2 * n)
    prep = torch.empty(ps, dtype=torch.uint8, device="cuda")
    rl.rlobpcg_gram_split_prepare(A.data_ptr(), m, 2 * n, 2 * n, prep.data_ptr(), ps, _stream())
    ws = rl.rlobpcg_gram_split_c128_workspace_size(m, n, 4)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    W = np.ones((n, 13), dtype=np.complex128)
    W[5, 1] = complex(0, np.inf)
    Wd = _dev(W)
    AW = torch.empty((m, 13), dtype=torch.complex128, device="cuda")
    G = torch.empty((n, 13), dtype=torch.complex128, device="cuda")
    with pytest.raises(rl.RlobpcgError) as e:
        rl.rlobpcg_gram_split_c128(prep.data_ptr(), m, n, Wd.data_ptr(), 13, 13, AW.data_ptr(), 13, G.data_ptr(), 13,
                                   work.data_ptr(), ws, _stream())
    assert e.value.code == rl.RLOBPCG_ERR_INVALID_ARG
    with pytest.raises(rl.RlobpcgError) as e:
        rl.rlobpcg_gram_split_c128(prep.data_ptr(), m, n, Wd.data_ptr(), 4, 13, AW.data_ptr(), 13, G.data_ptr(), 13,
                                   work.data_ptr(), ws - 1, _stream())
    assert e.value.code == rl.RLOBPCG_ERR_INVALID_ARG
    with pytest.raises(rl.RlobpcgError) as e:
        rl.rlobpcg_gram_split_c128(prep.data_ptr(), m, n, Wd.data_ptr(), 4, 13, AW.data_ptr(), 13, G.data_ptr(), 13,
                                   work.data_ptr(), ws, _stream())
    assert e.value.code == rl.RLOBPCG_ERR_NONFINITE


# ------------------------------------------------------------------------------- whole solves

def _solve(A, k, split, **kw):
    o = rl.rlobpcg_default_opts()
    o.seed = 931
    o.d = 3 * A.shape[1]
    o.zeta = 8
    o.gram_split = split
    o.exact_sketch_svd = 1      # the oracle's start block: V~(:, n-b+1:n) of the full sketch SVD
    for key, v in kw.items():
        setattr(o, key, v)
    sig, V, U_, res, info = rl.solve(_dev(A), k, opts=o)
    return sig.cpu().numpy(), V.cpu().numpy(), info


@pytest.mark.parametrize("b", [3, 12])
def test_complex_solve_fixed_iterations_split_and_fp64(b):
    rng = np.random.default_rng(14)
    sigma = np.concatenate([np.logspace(0, -8, 117), [1e-12, 3e-12, 1e-11]])
    A = wl.planted(rng, 15_000, sigma, complex_=True)[0]
    n, k = A.shape[1], 3
    ref = oracle.rlobpcg(A, k=k, b=b, d=3 * n, zeta=8, seed=931, fixed_iters=10)
    for split in (1, 0):
        sig, V, info = _solve(A, k, split, block=b, fixed_iters=10)
        assert info["iters"] == 10
        check_sigma(sig, ref["sigma"], ref["sigma11"], n)
        np.testing.assert_allclose(V.conj().T @ V, np.eye(k), atol=1e3 * np.sqrt(n) * U)


def test_complex_solve_with_residual_refresh():
    rng = np.random.default_rng(15)
    sigma = np.concatenate([np.logspace(0, -6, 97), [1e-10, 2e-10, 4e-10]])
    A, s, V = wl.planted(rng, 12_000, sigma, complex_=True)
    n, k = A.shape[1], 3
    sig, Vg, info = _solve(A, k, 1, residual_refresh_every=3)
    ref = oracle.rlobpcg(A, k=k, d=3 * n, zeta=8, seed=931)
    check_sigma(sig, ref["sigma"], ref["sigma11"], n)
    check_truth(sig, ref["sigma"], np.sort(s)[:k], ref["sigma11"], n)
