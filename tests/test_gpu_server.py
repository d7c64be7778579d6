"""Serving with continuous batching (rlobpcg_server_*): each result is the same alone and in the
mix, the HBM budget is respected, requests beyond it are refused, queued requests are cancelled
(and their waiters woken) by destroy, and one ticket has one waiter."""
import threading

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


def _waiter(srv, ticket, n, k, out):
    """Wait for one ticket on a thread; records the status code (0, 1 or the error raised)."""
    sig = np.zeros(k)
    V = np.zeros((n, k))
    try:
        rc, _ = rl.rlobpcg_server_wait(srv, ticket, sig.ctypes.data, V.ctypes.data, None)
        out.append(rc)
    except rl.RlobpcgError as e:
        out.append(e.code)


def test_destroy_cancels_queued_requests_and_wakes_waiters():
    reqs = _requests(count=5, max_m=60_000)
    srv = rl.rlobpcg_server_create(1 << 36, 1, 0)    # one slot: all but the first request queue
    tickets = [rl.rlobpcg_server_submit(srv, A.ctypes.data, A.shape[0], A.shape[1], A.shape[1], k,
                                        rl.RLOBPCG_F64, _opts(seed)) for A, k, seed in reqs]
    results = [[] for _ in reqs]
    threads = [threading.Thread(target=_waiter, args=(srv, t, A.shape[1], k, res))
               for (A, k, _), t, res in zip(reqs, tickets, results)]
    for th in threads:
        th.start()
    rl.rlobpcg_server_destroy(srv)                   # returns only after every waiter has left
    for th in threads:
        th.join(timeout=60)
        assert not th.is_alive()
    codes = [r[0] for r in results]
    assert all(c in (rl.RLOBPCG_OK, rl.RLOBPCG_NOT_CONVERGED, rl.RLOBPCG_ERR_CANCELLED) for c in codes), codes
    # the last request cannot have started before destroy (one slot, four ahead of it)
    assert codes[-1] == rl.RLOBPCG_ERR_CANCELLED


def test_one_waiter_per_ticket():
    reqs = _requests(count=3, max_m=60_000)
    srv = rl.rlobpcg_server_create(1 << 36, 1, 0)
    try:
        tickets = [rl.rlobpcg_server_submit(srv, A.ctypes.data, A.shape[0], A.shape[1], A.shape[1], k,
                                            rl.RLOBPCG_F64, _opts(seed)) for A, k, seed in reqs]
        A, k, _ = reqs[-1]
        out = []
        th = [threading.Thread(target=_waiter, args=(srv, tickets[-1], A.shape[1], k, out)) for _ in range(2)]
        for t in th:
            t.start()
        for t in th:
            t.join(timeout=120)
            assert not t.is_alive()
        # whichever thread claimed the ticket first gets the result; the other is refused
        assert len(out) == 2 and out.count(rl.RLOBPCG_ERR_INVALID_ARG) == 1, out
        assert all(c in (rl.RLOBPCG_OK, rl.RLOBPCG_NOT_CONVERGED, rl.RLOBPCG_ERR_INVALID_ARG) for c in out), out
        for t, (A, k, _) in zip(tickets[:-1], reqs[:-1]):
            rl.rlobpcg_server_wait(srv, t, None, None, None)
    finally:
        rl.rlobpcg_server_destroy(srv)


def _batch_alone(A, k, opts):
    """rlobpcg_solve_batch with this request alone (the reference for the batched server, which
    plans a request it hands to the batch engine without a split of A: gram_split = 0)."""
    m, n = A.shape
    opts.gram_split = 0
    st = torch.cuda.current_stream().cuda_stream
    Ad = torch.from_numpy(A).cuda()
    plan = rl.rlobpcg_plan(m, n, k, rl.RLOBPCG_F64, opts, st)
    sig = torch.empty(k, dtype=torch.float64, device="cuda")
    V = torch.empty((n, k), dtype=torch.float64, device="cuda")
    try:
        rc, infos, status = rl.rlobpcg_solve_batch([plan], [Ad.data_ptr()], [n], [sig.data_ptr()], [V.data_ptr()],
                                                   None, None, st)
    finally:
        rl.rlobpcg_plan_destroy(plan)
    assert rc >= 0
    return sig.cpu().numpy(), V.cpu().numpy(), infos[0].iters


def test_batched_server_results_equal_the_batch_alone_and_budget_holds():
    """Batched serving: the iterations of every admitted small solve (m n b <= 2^23) run together
    in the batch engine, solves joining and leaving between replays, and each such result is
    bit-identical to rlobpcg_solve_batch of that request alone; larger requests and a complex one
    (not batchable) run whole on their worker and equal rlobpcg_solve."""
    reqs = _requests(12)
    limit = 1 << 23                                # rlobpcg_server_set_batch_limit's default
    routed = [A.shape[0] * A.shape[1] * k <= limit for A, k, _ in reqs]
    assert any(routed) and not all(routed)         # both paths are exercised
    alone = []
    for (A, k, seed), eng in zip(reqs, routed):
        if eng:
            alone.append(_batch_alone(A, k, _opts(seed)))
        else:                                      # larger requests run whole, as rlobpcg_solve
            sig, V, _, _, info = rl.solve(torch.from_numpy(A).cuda(), k, opts=_opts(seed))
            alone.append((sig.cpu().numpy(), V.cpu().numpy(), info["iters"]))
    rng = np.random.default_rng(77)
    Ac = wl.planted(rng, 6000, np.concatenate([np.logspace(0, -6, 37), np.logspace(-9, -10, 3)]), complex_=True)[0]
    Ac = np.ascontiguousarray(Ac)
    sc, Vc, _, _, _ = rl.solve(torch.from_numpy(Ac).cuda(), 3, opts=_opts(5))
    srv = rl.rlobpcg_server_create(4 << 30, 16, 0, rl.RLOBPCG_SERVE_BATCHED)
    try:
        tickets = [rl.rlobpcg_server_submit(srv, A.ctypes.data, A.shape[0], A.shape[1], A.shape[1], k,
                                            rl.RLOBPCG_F64, _opts(seed)) for A, k, seed in reqs]
        tc = rl.rlobpcg_server_submit(srv, Ac.ctypes.data, Ac.shape[0], Ac.shape[1], Ac.shape[1], 3,
                                      rl.RLOBPCG_C128, _opts(5))
        for (A, k, seed), t, (s0, V0, it0) in zip(reqs, tickets, alone):
            sig = np.zeros(k)
            V = np.zeros((A.shape[1], k))
            info = rl.rlobpcg_info()
            rl.rlobpcg_server_wait(srv, t, sig.ctypes.data, V.ctypes.data, None, info)
            assert info.iters == it0
            assert np.array_equal(sig, s0) and np.array_equal(V, V0)
        sig = np.zeros(3)
        V = np.zeros((Ac.shape[1], 3), dtype=np.complex128)
        rl.rlobpcg_server_wait(srv, tc, sig.ctypes.data, V.ctypes.data, None, rl.rlobpcg_info())
        assert np.array_equal(sig, sc.cpu().numpy()) and np.array_equal(V, Vc.cpu().numpy())
        st = rl.rlobpcg_server_stats(srv)
        assert st["completed"] == len(reqs) + 1 and st["peak_bytes"] <= 4 << 30 and st["peak_running"] >= 2
    finally:
        rl.rlobpcg_server_destroy(srv)
