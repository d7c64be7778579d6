"""Block sizes b in {1, 3, 5, 10, 20} on the clustered spectrum of the block tests (Sec. 4.2),
one wanted triplet (k = 1), on a row-reduced copy that the oracle runs in seconds.

Per block size, in fixed-iteration mode: the smallest Ritz value after every iteration (the
history the study reports, read back with rlobpcg_history) against the oracle's, the final
triplet against the oracle's (bars of tests/parity.py), the matrix-vector count b (iterations + 1)
of Sec. 4.2's cost model, and the history's last row against the returned sigma. Every block size
runs the Gram products on the tensor cores (digit-block widths 8, 12 and 24).
"""
import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl
from tests.parity import check_sigma, check_truth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clustered_small():
    return wl.clustered(1006, 20_000, 200)


@pytest.mark.parametrize("b", [1, 3, 5, 10, 20])
def test_block_size_history_and_parity(clustered_small, b):
    A, s, V = clustered_small
    m, n = A.shape
    iters = 8
    o = rl.rlobpcg_default_opts()
    o.seed = 11
    o.block = b
    o.fixed_iters = iters
    o.exact_sketch_svd = 1        # the oracle's start block: V~(:, n-b+1:n) of the full sketch SVD
    st = torch.cuda.current_stream().cuda_stream
    plan = rl.rlobpcg_plan(m, n, 1, rl.RLOBPCG_F64, o, st)
    Ad = torch.from_numpy(A).cuda()
    sig = torch.empty(1, dtype=torch.float64, device="cuda")
    Vg = torch.empty((n, 1), dtype=torch.float64, device="cuda")
    res = torch.empty(1, dtype=torch.float64, device="cuda")
    info = rl.rlobpcg_info()
    try:
        rl.rlobpcg_solve(plan, Ad.data_ptr(), n, -1.0, sig.data_ptr(), Vg.data_ptr(), None, res.data_ptr(), info)
        th, rs = rl.rlobpcg_history(plan)
    finally:
        rl.rlobpcg_plan_destroy(plan)
    ora = oracle.rlobpcg(A, k=1, b=b, seed=11, fixed_iters=iters)
    assert info.iters == iters and info.block == b
    assert info.matvecs == b * (iters + 1) == ora["matvecs"]
    assert th.shape == (iters + 1, b) and rs.shape == (iters + 1, b)
    # the last row's smallest Ritz value is the returned sigma, bit for bit
    assert th[-1, -1] == sig.item()
    # per-iteration smallest Ritz value against the oracle's (row 0: the start block's)
    th_ora = np.vstack([ora["theta0"][None, :], ora["theta_hist"][1:]])
    rel = np.abs(th[:, -1] - th_ora[:, -1]) / th_ora[:, -1]
    print("per-iteration relative difference of the smallest Ritz value:", rel)
    for t in range(iters + 1):
        check_sigma(th[t, -1:], th_ora[t, -1:], ora["sigma11"], n)
    check_sigma(sig.cpu().numpy(), ora["sigma"], ora["sigma11"], n)
    np.testing.assert_allclose(rs[1:, -1], ora["res_hist"][1:, -1], rtol=5e-2,
                               atol=100 * np.sqrt(n) * 2.0 ** -53 * ora["sigma11"] ** 2)


@pytest.mark.parametrize("b", [1, 5])
def test_block_size_adaptive_against_truth(clustered_small, b):
    """With the paper's stopping rule: the smallest singular value within the backward-stable
    floor of the planted one (Sec. 4), whatever the block size."""
    A, s, V = clustered_small
    o = rl.rlobpcg_default_opts()
    o.seed = 11
    o.block = b
    sig, Vg, _, _, info = rl.solve(torch.from_numpy(A).cuda(), 1, opts=o)
    ora = oracle.rlobpcg(A, k=1, b=b, seed=11)
    check_truth(sig.cpu().numpy(), ora["sigma"], s[-1:], ora["sigma11"], A.shape[1])
