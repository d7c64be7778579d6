"""Full-size configurations, in the launch configuration bench.py times.

- complex128 2e5 x 300, k = 3: parity with the oracle at full size.
- 1e6 x 1000 (8 GB) Gram pass, FP64 and split-bf16 tensor-core forms, b = 10 (the block the
  1e6 x 1000, k = 10 solve uses): the oracle's products A W and A^H (A W), elementwise.
- 1e6 x 1000, k = 10 solves, FP64 sketch and FP32 sketch/R: the oracle is too slow at this size,
  so the results are checked against what holds at any size: the planted singular values and
  subspace (within the backward-stable floors of Sec. 4), ||A v_j|| = sigma_j and V^H V = I.
"""
import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl
from tests.parity import U, c_of, check_angle, check_sigma, check_truth, sub_sin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _opts(seed, d, prec=0, **kw):
    o = rl.rlobpcg_default_opts()
    o.seed = seed
    o.d = d
    o.zeta = 8
    o.sketch_prec = prec
    for k_, v in kw.items():
        setattr(o, k_, v)
    return o


def test_complex_full_size_refined_sketch():
    """The complex 2e5 x 300, k = 3 configuration with its FP32 factor (refined once in FP64 so
    that kappa = 1e13 is resolved): converges (no max_iter) and matches the oracle's refined run
    and the planted truth at full size."""
    A, s, V = wl.planted_complex()
    n, k = 300, 3
    sig, Vg, _, _, info = rl.solve(torch.from_numpy(A).cuda(), k,
                                   opts=_opts(1003, 4 * n, rl.RLOBPCG_SKETCH_F32_REFINE))
    assert info["stop_reason"] == rl.RLOBPCG_STOP_CONVERGED
    sig, Vg = sig.cpu().numpy(), Vg.cpu().numpy()
    o = oracle.rlobpcg(A, k=k, d=4 * n, zeta=8, seed=1003, sketch_precision="f32_refine")
    gap = (s[-4] - s[-3]) / s[0]
    check_sigma(sig, o["sigma"], o["sigma11"], n)
    check_angle(Vg, o["V"], gap, n)
    check_truth(sig, o["sigma"], s[::-1][:k], o["sigma11"], n)


def test_complex_full_size_parity():
    A, s, V = wl.planted_complex()
    n, k = 300, 3
    sig, Vg, _, _, info = rl.solve(torch.from_numpy(A).cuda(), k, opts=_opts(1003, 4 * n))
    sig, Vg = sig.cpu().numpy(), Vg.cpu().numpy()
    o = oracle.rlobpcg(A, k=k, d=4 * n, zeta=8, seed=1003)
    gap = (s[-4] - s[-3]) / s[0]
    check_sigma(sig, o["sigma"], o["sigma11"], n)
    check_angle(Vg, o["V"], gap, n)
    check_truth(sig, o["sigma"], s[::-1][:k], o["sigma11"], n)


@pytest.fixture(scope="module")
def large():
    A, s, V = wl.planted_large_device()
    yield A, s, V
    del A
    torch.cuda.empty_cache()


def test_large_gram_pass_against_oracle_products(large):
    A, s, V = large
    m, n = A.shape
    b = 10
    rng = np.random.default_rng(11)
    W = rng.standard_normal((n, b))
    Wd = torch.from_numpy(W).cuda()
    AW = torch.empty((m, b), dtype=torch.float64, device="cuda")
    G = torch.empty((n, b), dtype=torch.float64, device="cuda")
    ws = rl.rlobpcg_gram_workspace_size(m, n, b, rl.RLOBPCG_F64)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    rl.rlobpcg_gram(A.data_ptr(), m, n, n, rl.RLOBPCG_F64, Wd.data_ptr(), b, b, AW.data_ptr(), b, G.data_ptr(), b,
                    work.data_ptr(), ws, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    Ah = A.cpu().numpy()
    AW_h, G_h = AW.cpu().numpy(), G.cpu().numpy()
    rows = rng.choice(m, 2000, replace=False)
    AW0 = Ah[rows] @ W
    b1 = (n + 2) * U * (np.abs(Ah[rows]) @ np.abs(W))
    assert np.all(np.abs(AW_h[rows] - AW0) <= b1)
    AWfull, G0 = oracle.gram_pass(Ah, W)
    absA = np.abs(Ah)
    b2 = absA.T @ ((n + 2) * U * (absA @ np.abs(W))) + (m + 2) * U * (absA.T @ np.abs(AWfull))
    assert np.all(np.abs(G_h - G0) <= b2)


def test_large_split_gram_pass_against_oracle_products(large):
    """The tensor-core Gram pass at the full 1e6 x 1000 size with b = 10, in the launch
    configuration a solve of that matrix uses, against the oracle's products elementwise under
    the split's error bound (tests/test_gpu_split_gram.py)."""
    from tests.test_gpu_split_gram import bounds
    A, s, V = large
    m, n = A.shape
    b = 10
    rng = np.random.default_rng(12)
    W = np.linalg.qr(rng.standard_normal((n, b)))[0]
    Wd = torch.from_numpy(W).cuda()
    st = torch.cuda.current_stream().cuda_stream
    ps = rl.rlobpcg_gram_split_prepare_size(m, n)
    ws = rl.rlobpcg_gram_split_workspace_size(m, n, b)
    prep = torch.empty(ps, dtype=torch.uint8, device="cuda")
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    AW = torch.full((m, b), np.nan, dtype=torch.float64, device="cuda")
    G = torch.full((n, b), np.nan, dtype=torch.float64, device="cuda")
    rl.rlobpcg_gram_split_prepare(A.data_ptr(), m, n, n, prep.data_ptr(), ps, st)
    rl.rlobpcg_gram_split(prep.data_ptr(), m, n, Wd.data_ptr(), b, b, AW.data_ptr(), b, G.data_ptr(), b,
                          work.data_ptr(), ws, st)
    torch.cuda.synchronize()
    del prep, work
    Ah = A.cpu().numpy()
    AW_h, G_h = AW.cpu().numpy(), G.cpu().numpy()
    AW0, G0 = oracle.gram_pass(Ah, W)
    tAW, tG = bounds(Ah, W, AW0)
    assert np.all(np.abs(AW_h - AW0) <= tAW)
    assert np.all(np.abs(G_h - G0) <= tG)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_large_solve_against_planted_truth(large, prec):
    A, s, V = large
    m, n = A.shape
    k = 10
    sig, Vg, _, resid, info = rl.solve(A, k, opts=_opts(1004, 4 * n, prec))
    sig, Vg = sig.cpu().numpy(), Vg.cpu().numpy()
    floor = c_of(n) * U * s[0]
    # planted values and subspace within the floors u sigma_1 (value) and u / gap_abs (subspace)
    assert np.all(np.abs(sig - s[::-1][:k]) <= max(floor, 0)), (sig, s[::-1][:k])
    gap = (s[-k - 1] - s[-k]) / s[0]
    assert sub_sin(Vg, V[:, -k:]) <= max(1e-8, c_of(n) * U / gap)
    # invariants at full size: orthonormal V, ||A v_j|| = sigma_j
    assert np.allclose(Vg.T @ Vg, np.eye(k), atol=100 * n * U)
    AV = (A @ torch.from_numpy(Vg).cuda()).cpu().numpy()
    assert np.all(np.abs(np.linalg.norm(AV, axis=0) - sig) <= 100 * np.sqrt(n) * U * s[0])
    assert info["stop_reason"] in (rl.RLOBPCG_STOP_CONVERGED, rl.RLOBPCG_STOP_MAX_ITER)
