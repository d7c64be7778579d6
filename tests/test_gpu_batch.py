"""Batched solves (rlobpcg_solve_batch): many small solves iterating together in two persistent
kernels per iteration, replayed from a captured CUDA graph.

- fixed-iteration parity with the oracle per solve: the Ritz values after every iteration (bars of
  tests/parity.py), the final triplets, orthonormal V and U = A V / sigma;
- bit-identity: each solve alone (a batch of one) and in the mixed batch give the same bits;
- the device stopping rule: adaptive solves reach the planted values within the floors of Sec. 4;
- a Loewner-type nullspace (sigma_min at noise level): backward error only;
- the autotuner's table and the argument checks.
Shapes follow the serving stream's recipe on a small scale: n from 20 to 120, k in {1, 2, 4}.
"""
import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl
from tests.parity import U as U64, check_sigma, check_truth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(3000, 20, 1), (8000, 60, 2), (5000, 100, 4), (12000, 40, 4), (2500, 120, 1), (20000, 80, 2)]


def _problem(i, m, n, k):
    rng = np.random.default_rng(7100 + i)
    sigma = np.concatenate([np.logspace(0, -6, n - k), np.logspace(-9, -10, k)])
    A, s, V = wl.planted(rng, m, sigma)
    return A, s


@pytest.fixture(scope="module")
def problems():
    return [_problem(i, *sh) for i, sh in enumerate(SHAPES)]


def _opts(k, fixed=None, seed=11):
    o = rl.rlobpcg_default_opts()
    o.seed = seed
    o.block = k
    o.exact_sketch_svd = 1
    o.gram_split = 0
    if fixed:
        o.fixed_iters = fixed
    return o


def _run_batch(mats, ks, fixed=None, want_u=True):
    """mats: device tensors; returns per-solve dicts with numpy outputs, infos and histories."""
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in mats]
    plans, outs = [], []
    for A, k, s in zip(mats, ks, streams):
        m, n = A.shape
        plans.append(rl.rlobpcg_plan(m, n, k, rl.RLOBPCG_F64, _opts(k, fixed), s.cuda_stream))
        outs.append(dict(sigma=torch.empty(k, dtype=torch.float64, device="cuda"),
                         V=torch.empty((n, k), dtype=torch.float64, device="cuda"),
                         U=torch.empty((m, k), dtype=torch.float64, device="cuda") if want_u else None,
                         resid=torch.empty(k, dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    try:
        rc, infos, st = rl.rlobpcg_solve_batch(
            plans, [A.data_ptr() for A in mats], [A.shape[1] for A in mats],
            [o["sigma"].data_ptr() for o in outs], [o["V"].data_ptr() for o in outs],
            [o["U"].data_ptr() for o in outs] if want_u else None, [o["resid"].data_ptr() for o in outs],
            torch.cuda.current_stream().cuda_stream)
        hist = [rl.rlobpcg_history(p) for p in plans]
    finally:
        for p in plans:
            rl.rlobpcg_plan_destroy(p)
    assert rc >= 0, (rc, rl.rlobpcg_last_error())
    res = []
    for o, info, s, h in zip(outs, infos, st, hist):
        res.append(dict(sigma=o["sigma"].cpu().numpy(), V=o["V"].cpu().numpy(),
                        U=o["U"].cpu().numpy() if want_u else None, resid=o["resid"].cpu().numpy(),
                        info=info, status=s, theta=h[0], res=h[1]))
    return res


def test_batch_fixed_iterations_parity(problems):
    iters = 6
    mats = [torch.from_numpy(A).cuda() for A, _ in problems]
    ks = [sh[2] for sh in SHAPES]
    out = _run_batch(mats, ks, fixed=iters)
    for (A, s), k, r in zip(problems, ks, out):
        n = A.shape[1]
        ora = oracle.rlobpcg(A, k=k, b=k, seed=11, fixed_iters=iters)
        assert r["status"] == rl.RLOBPCG_OK and r["info"].iters == iters
        assert r["info"].matvecs == k * (iters + 1) == ora["matvecs"]
        assert r["info"].stop_reason == rl.RLOBPCG_STOP_FIXED
        th_ora = np.vstack([ora["theta0"][None, :], ora["theta_hist"][1:]])
        assert r["theta"].shape == th_ora.shape
        for t in range(iters + 1):
            check_sigma(r["theta"][t], th_ora[t], ora["sigma11"], n)
        check_sigma(r["sigma"], ora["sigma"], ora["sigma11"], n)
        V, U = r["V"], r["U"]
        np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e3 * np.sqrt(n) * U64)
        np.testing.assert_allclose(U * r["sigma"][None, :], A @ V, atol=1e2 * np.sqrt(n) * U64 * ora["sigma11"])


def test_batch_results_are_the_same_alone_and_in_the_mix(problems):
    mats = [torch.from_numpy(A).cuda() for A, _ in problems]
    ks = [sh[2] for sh in SHAPES]
    mixed = _run_batch(mats, ks)
    for i in [0, 2, 5]:
        alone = _run_batch([mats[i]], [ks[i]])[0]
        for key in ("sigma", "V", "U", "resid", "theta", "res"):
            assert np.array_equal(alone[key], mixed[i][key]), key
        assert alone["info"].iters == mixed[i]["info"].iters
        assert alone["info"].stop_reason == mixed[i]["info"].stop_reason


def test_batch_adaptive_reaches_the_planted_values(problems):
    mats = [torch.from_numpy(A).cuda() for A, _ in problems]
    ks = [sh[2] for sh in SHAPES]
    out = _run_batch(mats, ks)
    for (A, s), k, r in zip(problems, ks, out):
        n = A.shape[1]
        ora = oracle.rlobpcg(A, k=k, b=k, seed=11)
        print("n", n, "k", k, "gpu iters", r["info"].iters, "stop", r["info"].stop_reason,
              "oracle iters", ora["iters"], ora["stop_reason"])
        assert r["status"] in (rl.RLOBPCG_OK, rl.RLOBPCG_NOT_CONVERGED)
        check_truth(r["sigma"], ora["sigma"], np.sort(s)[:k], ora["sigma11"], n)
        # the history's last row holds the returned values
        np.testing.assert_array_equal(r["theta"][-1][::-1][:k], r["sigma"])


def test_batch_loewner_nullspace_backward_error():
    """Half of the serving stream is Loewner-type: sigma_min sits at noise level, so only the
    backward error ||L v|| and orthonormality are defined (Sec. 4)."""
    mats, ks = [], []
    for j, (m, n, k) in enumerate([(4000, 40, 1), (6000, 90, 2), (3000, 30, 4)]):
        L = wl.loewner(9100 + j, m, n)
        mats.append(torch.from_numpy(np.ascontiguousarray(L)).cuda())
        ks.append(k)
    out = _run_batch(mats, ks, want_u=False)
    for A, k, r in zip(mats, ks, out):
        L = A.cpu().numpy()
        n = L.shape[1]
        assert r["status"] in (rl.RLOBPCG_OK, rl.RLOBPCG_NOT_CONVERGED)
        V = r["V"]
        np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e3 * np.sqrt(n) * U64)
        bw = np.linalg.norm(L @ V, axis=0)
        assert np.all(bw <= 1e3 * np.sqrt(n) * U64 * np.linalg.norm(L, "fro")), bw


def test_batch_tile_table_and_pinning():
    t1 = rl.rlobpcg_batch_tile(100, 4)
    assert t1[0] in (256, 512, 1024, 2048) and t1[1] in (8, 16)
    assert rl.rlobpcg_batch_tile(70, 4) == t1          # same class (n in (64, 128])
    with pytest.raises(rl.RlobpcgError):
        rl.rlobpcg_batch_set_tile(100, 4, 300, 16)     # not a candidate
    with pytest.raises(rl.RlobpcgError):
        rl.rlobpcg_batch_tile(600, 4)                  # n above the batched path


def test_batch_rejects_what_it_does_not_run():
    A = torch.randn(2000, 30, dtype=torch.float64, device="cuda")
    sig = torch.empty(1, dtype=torch.float64, device="cuda")
    V = torch.empty((30, 1), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    o = _opts(1)
    o.locking = 1
    p = rl.rlobpcg_plan(2000, 30, 1, rl.RLOBPCG_F64, o, st)
    try:
        rc, _, _ = rl.rlobpcg_solve_batch([p], [A.data_ptr()], [30], [sig.data_ptr()], [V.data_ptr()], None, None, st)
        assert rc == rl.RLOBPCG_ERR_UNSUPPORTED
    finally:
        rl.rlobpcg_plan_destroy(p)
    p = rl.rlobpcg_plan(2000, 30, 1, rl.RLOBPCG_F64, _opts(1), st)
    try:
        Ah = A.cpu().numpy()
        rc, _, _ = rl.rlobpcg_solve_batch([p], [Ah.ctypes.data], [30], [sig.data_ptr()], [V.data_ptr()], None, None, st)
        assert rc == rl.RLOBPCG_ERR_INVALID_ARG        # A must be on the device
    finally:
        rl.rlobpcg_plan_destroy(p)
