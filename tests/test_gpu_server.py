"""Serving with continuous batching (rlobpcg_server_*): each result is the same alone and in the
mix, the HBM budget is respected, and requests beyond it are refused."""
import numpy as np
import pytest

from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests(count=10, max_m=30_000):
    """Mixed stream shaped like the serving workload (half Loewner, half planted; uneven m, n, k),
    with m capped to keep the test short."""
    out = []
    rng = np.random.default_rng(7)
    for r in range(count):
        n = int(rng.integers(20, 201))
        k = int(rng.choice([1, 2, 4]))
        m = int(max(4 * n, np.exp(rng.uniform(np.log(2e3), np.log(max_m)))))
        if r % 2 == 0:
            A = wl.loewner(50000 + r, m, n)
        else:
            sig = np.concatenate([np.logspace(0, -6, n - k), np.logspace(-9, -10, k)])
            A = wl.planted(np.random.default_rng(50000 + r), m, sig)[0]
        out.append((np.ascontiguousarray(A), k, 900 + r))
    return out


def _opts(seed):
    o = rl.rlobpcg_default_opts()
    o.seed = seed
    o.max_iter = 60
    return o


def test_server_results_equal_solo_and_budget_holds():
    reqs = _requests()
    solo = []
    for A, k, seed in reqs:
        sig, V, _, _, info = rl.solve(torch.from_numpy(A).cuda(), k, opts=_opts(seed))
        solo.append((sig.cpu().numpy(), V.cpu().numpy()))
    sizes = sorted((rl.rlobpcg_plan_workspace_size(A.shape[0], A.shape[1], k, rl.RLOBPCG_F64, _opts(s)) +
                    A.nbytes for A, k, s in reqs), reverse=True)
    budget = sum(sizes[:3])                      # at most ~3 of the largest at once: requests queue
    srv = rl.rlobpcg_server_create(budget, 4, 0)
    try:
        tickets = [rl.rlobpcg_server_submit(srv, A.ctypes.data, A.shape[0], A.shape[1], A.shape[1], k,
                                            rl.RLOBPCG_F64, _opts(seed)) for A, k, seed in reqs]
        for (A, k, seed), t, (s0, V0) in zip(reqs, tickets, solo):
            sig = np.zeros(k)
            V = np.zeros((A.shape[1], k))
            info = rl.rlobpcg_info()
            rl.rlobpcg_server_wait(srv, t, sig.ctypes.data, V.ctypes.data, None, info)
            # same deterministic kernels on the same input: identical results
            assert np.array_equal(sig, s0) and np.array_equal(V, V0)
        st = rl.rlobpcg_server_stats(srv)
    finally:
        rl.rlobpcg_server_destroy(srv)
    assert st["completed"] == len(reqs)
    assert st["peak_bytes"] <= budget
    assert 1 <= st["peak_running"] <= 4
    assert 0 < st["p50_ms"] <= st["p99_ms"]


def test_server_refuses_request_beyond_budget():
    A = np.random.default_rng(0).standard_normal((5000, 40))
    srv = rl.rlobpcg_server_create(1 << 20, 2, 0)
    try:
        with pytest.raises(rl.RlobpcgError) as e:
            rl.rlobpcg_server_submit(srv, A.ctypes.data, 5000, 40, 40, 1, rl.RLOBPCG_F64, None)
        assert e.value.code == rl.RLOBPCG_ERR_OOM
    finally:
        rl.rlobpcg_server_destroy(srv)
