"""The split-bf16 Gram pass on the tensor cores (rlobpcg_gram_split) against the oracle's products.

The products are those of the Gram pass of Alg. 2 (A W and A^T (A W)). Bounds: a split operand
is exact to 2^-56 of its group maximum (E of the group, |x| < 2^E, error <= 2^(E-56) <= 2^-55
max), so a product term a w carries at most 2^-55 (max_a |w| + |a| max_w) plus FP64 rounding of
the recombination; the digit pairs of levels above 8, which the pass does not form, weigh below
2^-58 of max_a max_w per term; the oracle's own product adds the usual n u |A||W|. Block widths
cover every digit-block width of the pass (8, 12, 16, 24).
"""
import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl
from tests.parity import check_angle, check_sigma, check_truth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def split_gram(A, W):
    """AW, G from the tensor-core path through the C ABI (prepare + one pass)."""
    m, n = A.shape
    b = W.shape[1]
    Ad, Wd = _dev(A), _dev(W)
    ps = rl.rlobpcg_gram_split_prepare_size(m, n)
    ws = rl.rlobpcg_gram_split_workspace_size(m, n, b)
    prep = torch.empty(ps, dtype=torch.uint8, device="cuda")
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    AW = torch.full((m, b), np.nan, dtype=torch.float64, device="cuda")
    G = torch.full((n, b), np.nan, dtype=torch.float64, device="cuda")
    rl.rlobpcg_gram_split_prepare(Ad.data_ptr(), m, n, n, prep.data_ptr(), ps, _stream())
    rl.rlobpcg_gram_split(prep.data_ptr(), m, n, Wd.data_ptr(), b, b, AW.data_ptr(), b, G.data_ptr(), b,
                          work.data_ptr(), ws, _stream())
    torch.cuda.synchronize()
    return AW.cpu().numpy(), G.cpu().numpy()


def bounds(A, W, AW0):
    """Elementwise error bounds for AW and G = A^T AW (see module docstring); chunk maxima are
    bounded by global column maxima."""
    m, n = A.shape
    aA, aW = np.abs(A), np.abs(W)
    rowmax, rowsum = aA.max(axis=1), aA.sum(axis=1)
    wmax, wsum = aW.max(axis=0), aW.sum(axis=0)
    tAW = 2.0 ** -53 * (np.outer(rowmax, wsum) + np.outer(rowsum, wmax)) + (n + 32) * U * (aA @ aW)
    aY = np.abs(AW0) + tAW
    colmax, colsum = aA.max(axis=0), aA.sum(axis=0)
    ymax, ysum = aY.max(axis=0), aY.sum(axis=0)
    tG = aA.T @ tAW + 2.0 ** -53 * (np.outer(colmax, ysum) + np.outer(colsum, ymax)) + (m + 32) * U * (aA.T @ aY)
    return tAW, tG


def check_against_oracle(A, W):
    AW, G = split_gram(A, W)
    AW0, G0 = oracle.gram_pass(A, W)
    tAW, tG = bounds(A, W, AW0)
    eAW, eG = np.abs(AW - AW0), np.abs(G - G0)
    assert np.all(eAW <= tAW), (np.max(eAW / tAW), np.unravel_index(np.argmax(eAW / tAW), eAW.shape))
    assert np.all(eG <= tG), (np.max(eG / tG), np.unravel_index(np.argmax(eG / tG), eG.shape))
    return AW, G, AW0, G0


def test_integer_operands_give_exact_products():
    # entries with at most 11 significant bits: the first product is exact in FP64, the split
    # holds them in two digits, and levels 0..2 recombine exactly, so A W must be bit-exact.
    rng = np.random.default_rng(1)
    m, n, b = 3000, 500, 5
    A = rng.integers(-1024, 1025, (m, n)).astype(np.float64)
    W = rng.integers(-1024, 1025, (n, b)).astype(np.float64)
    AW, G = split_gram(A, W)
    exact = A.astype(np.int64) @ W.astype(np.int64)
    assert np.array_equal(AW, exact.astype(np.float64))
    Gx = A.astype(np.int64).T @ exact          # |entries| < 2^53: exact in int64 and in the bound
    assert np.all(np.abs(G - Gx.astype(np.float64)) <= 64 * U * np.abs(A).T @ np.abs(exact))


@pytest.mark.parametrize("m,n,b", [(1, 1, 1), (127, 16, 3), (129, 17, 5), (2999, 500, 5), (5000, 700, 10),
                                   (3001, 300, 8), (2048, 128, 9), (4097, 1000, 16), (1000, 40, 2),
                                   (3000, 257, 11), (2500, 600, 12), (129, 33, 13), (4097, 300, 17),
                                   (3000, 1030, 20), (1500, 96, 24)])
def test_products_against_oracle(m, n, b):
    rng = np.random.default_rng(m * 7 + n + b)
    A = rng.standard_normal((m, n))
    W = rng.standard_normal((n, b))
    check_against_oracle(A, W)


def test_row_scales_are_kept_per_row():
    # rows 2^(+-300) apart: a single global scale would flush the small rows to zero digits
    rng = np.random.default_rng(2)
    m, n, b = 1500, 200, 4
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-300, 301, (m, 1)))
    W = rng.standard_normal((n, b))
    AW, G, AW0, G0 = check_against_oracle(A, W)
    rel = np.abs(AW - AW0) / (np.abs(A) @ np.abs(W))
    assert rel.max() < 1e-14


def test_column_scales_of_w_and_chunks():
    rng = np.random.default_rng(3)
    m, n, b = 1300, 150, 6
    A = rng.standard_normal((m, n)) * np.exp2(rng.integers(-40, 41, (1, n)))
    W = rng.standard_normal((n, b)) * np.exp2(np.array([-200, -50, 0, 10, 100, 250]))[None, :]
    check_against_oracle(A, W)


def test_loewner_and_planted_rows():
    A = wl.loewner(70001, 4000, 120)
    W = np.linalg.qr(np.random.default_rng(4).standard_normal((120, 5)))[0]
    check_against_oracle(A, W)
    Ap = wl.planted(np.random.default_rng(5), 3000, np.logspace(0, -12, 90))[0]
    check_against_oracle(Ap, np.random.default_rng(6).standard_normal((90, 3)))


def test_invalid_and_nonfinite():
    m, n = 300, 40
    A = _dev(np.ones((m, n)))
    ps = rl.rlobpcg_gram_split_prepare_size(m, n)
    prep = torch.empty(ps, dtype=torch.uint8, device="cuda")
    rl.rlobpcg_gram_split_prepare(A.data_ptr(), m, n, n, prep.data_ptr(), ps, _stream())
    assert rl.rlobpcg_gram_split_workspace_size(m, n, 25) == 0
    ws = rl.rlobpcg_gram_split_workspace_size(m, n, 4)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    W = np.ones((n, 4))
    W[3, 2] = np.nan
    Wd = _dev(W)
    AW = torch.empty((m, 25), dtype=torch.float64, device="cuda")
    G = torch.empty((n, 25), dtype=torch.float64, device="cuda")
    with pytest.raises(rl.RlobpcgError) as e:
        rl.rlobpcg_gram_split(prep.data_ptr(), m, n, Wd.data_ptr(), 25, 25, AW.data_ptr(), 25, G.data_ptr(), 25,
                              work.data_ptr(), ws, _stream())
    assert e.value.code == rl.RLOBPCG_ERR_INVALID_ARG
    with pytest.raises(rl.RlobpcgError) as e:
        rl.rlobpcg_gram_split(prep.data_ptr(), m, n, Wd.data_ptr(), 4, 4, AW.data_ptr(), 4, G.data_ptr(), 4,
                              work.data_ptr(), ws, _stream())
    assert e.value.code == rl.RLOBPCG_ERR_NONFINITE
    with pytest.raises(rl.RlobpcgError) as e:
        rl.rlobpcg_gram_split_prepare(A.data_ptr(), m, n, n, prep.data_ptr(), ps - 1, _stream())
    assert e.value.code == rl.RLOBPCG_ERR_INVALID_ARG
    for bad in (np.nan, np.inf, -np.inf):
        Ab = np.ones((m, n))
        Ab[m - 1, n - 1] = bad
        with pytest.raises(rl.RlobpcgError) as e:
            rl.rlobpcg_gram_split_prepare(_dev(Ab).data_ptr(), m, n, n, prep.data_ptr(), ps, _stream())
        assert e.value.code == rl.RLOBPCG_ERR_NONFINITE


# ------------------------------------------------------------------------------- whole solves

def _opts(seed, d, **kw):
    o = rl.rlobpcg_default_opts()
    o.seed = seed
    o.d = d
    o.zeta = 8
    o.gram_split = 1
    for k_, v in kw.items():
        setattr(o, k_, v)
    return o


@pytest.mark.parametrize("case", ["small", "nullspace", "cluster", "loewner"])
def test_solve_with_split_gram_matches_oracle(case):
    if case == "small":
        A, s, V = wl.planted_small_gap_free()
        k, d, tau = 1, 200, 1e-12
        truth = s[::-1][:k]
    elif case == "nullspace":
        A, C = wl.exact_nullspace(m=20000, n=200, rank=195, seed=81)
        k, d, tau = 5, 600, -1.0
        truth = np.zeros(k)
    elif case == "cluster":
        A, s, V = wl.planted_bottom_cluster(m=20000, n=200, k=5, seed=82)
        k, d, tau = 5, 600, -1.0
        truth = s[::-1][:k]
    else:
        A = wl.loewner(83, 20000, 150)
        k, d, tau = 2, 600, -1.0
        truth = None
    n = A.shape[1]
    o = _opts(900, d, tau=tau, use_stagnation=0 if case == "small" else 1)
    sig, Vg, _, _, info = rl.solve(_dev(A), k, opts=o)
    sig, Vg = sig.cpu().numpy(), Vg.cpu().numpy()
    ref = oracle.rlobpcg(A, k=k, d=d, zeta=8, seed=900, tau=None if tau < 0 else tau,
                         use_stagnation=case != "small")
    check_sigma(sig, ref["sigma"], ref["sigma11"], n)
    if truth is not None:
        check_truth(sig, ref["sigma"], truth, ref["sigma11"], n)
    if case in ("small", "cluster"):
        gap = (s[-k - 1] - s[-k]) / s[0]
        check_angle(Vg, ref["V"], gap, n)
    if case == "loewner":
        # singular values at rounding level: the stop test sees noise; check the backward error
        assert np.linalg.norm(A @ Vg, 2) <= 50 * np.sqrt(n) * 2.0 ** -53 * np.linalg.norm(A)
        assert np.allclose(Vg.T @ Vg, np.eye(k), atol=1e-12)
        return
    if ref["stop_reason"] == "converged":
        # the products differ from the oracle's by rounding only: the stop rule fires within a few
        # iterations of the oracle's (when the oracle stops at all: with the stagnation checks a
        # target at rounding level can run to max_iter on one side and stop on the other)
        assert info["stop_reason"] == rl.RLOBPCG_STOP_CONVERGED
        assert abs(info["iters"] - ref["iters"]) <= max(5, ref["iters"] // 5), (info["iters"], ref["iters"])


def test_split_and_fp64_paths_agree_fixed_iterations():
    A, s, V = wl.planted_bottom_cluster(m=12000, n=160, k=4, seed=84)
    k, d = 4, 480
    out = {}
    for split in (0, 1):
        o = _opts(901, d, fixed_iters=12, gram_split=split)
        sig, Vg, _, _, _ = rl.solve(_dev(A), k, opts=o)
        out[split] = (sig.cpu().numpy(), Vg.cpu().numpy())
    ref = oracle.rlobpcg(A, k=k, d=d, zeta=8, seed=901, fixed_iters=12)
    for split in (0, 1):
        check_sigma(out[split][0], ref["sigma"], ref["sigma11"], 160)


def test_split_with_residual_refresh():
    A, s, V = wl.planted_bottom_cluster(m=15000, n=180, k=3, seed=85)
    k, d = 3, 540
    o = _opts(902, d, residual_refresh_every=3)
    sig, Vg, _, _, info = rl.solve(_dev(A), k, opts=o)
    ref = oracle.rlobpcg(A, k=k, d=d, zeta=8, seed=902)
    check_sigma(sig.cpu().numpy(), ref["sigma"], ref["sigma11"], 180)
    check_truth(sig.cpu().numpy(), ref["sigma"], s[::-1][:k], ref["sigma11"], 180)
