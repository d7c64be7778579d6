"""rlobpcg_solve_async / rlobpcg_solve_wait: the solve runs on a library thread and gives the same
results, bit for bit, as rlobpcg_solve on the same plan; the plan refuses other calls while a
solve is in flight; errors come back through the wait; destroying the plan waits for the solve."""
import time

import numpy as np
import pytest

from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _buffers(m, n, k, dtype=torch.float64):
    return dict(sigma=torch.empty(k, dtype=torch.float64, device="cuda"),
                V=torch.empty((n, k), dtype=dtype, device="cuda"),
                U=torch.empty((m, k), dtype=dtype, device="cuda"),
                resid=torch.empty(k, dtype=torch.float64, device="cuda"))


def _plan(m, n, k, dtype=rl.RLOBPCG_F64):
    o = rl.rlobpcg_default_opts()
    o.seed = 41
    return rl.rlobpcg_plan(m, n, k, dtype, o, torch.cuda.current_stream().cuda_stream)


def _run(plan, A, out, asynchronous):
    info = rl.rlobpcg_info()
    args = (plan, A.data_ptr(), A.shape[1], -1.0, out["sigma"].data_ptr(), out["V"].data_ptr(),
            out["U"].data_ptr(), out["resid"].data_ptr(), info)
    if asynchronous:
        rl.rlobpcg_solve_async(*args)
        rc = rl.rlobpcg_solve_wait(plan)
    else:
        rc = rl.rlobpcg_solve(*args)
    torch.cuda.synchronize()
    return rc, info, {key: v.cpu().numpy() for key, v in out.items()}


@pytest.mark.parametrize("cplx", [False, True])
def test_async_results_equal_sync(cplx):
    rng = np.random.default_rng(5)
    sigma = np.concatenate([np.logspace(0, -6, 77), np.logspace(-9, -10, 3)])
    A = wl.planted(rng, 20_000, sigma, complex_=cplx)[0]
    Ad = torch.from_numpy(A).cuda()
    m, n, k = A.shape[0], A.shape[1], 3
    tdt = torch.complex128 if cplx else torch.float64
    plan = _plan(m, n, k, rl.RLOBPCG_C128 if cplx else rl.RLOBPCG_F64)
    try:
        rc0, info0, r0 = _run(plan, Ad, _buffers(m, n, k, tdt), False)
        rc1, info1, r1 = _run(plan, Ad, _buffers(m, n, k, tdt), True)
    finally:
        rl.rlobpcg_plan_destroy(plan)
    assert rc0 == rc1 and info0.iters == info1.iters and info0.stop_reason == info1.stop_reason
    for key in r0:
        assert np.array_equal(r0[key], r1[key]), key


def test_async_returns_before_the_solve_ends_and_guards_the_plan():
    A, s, V = wl.planted_complex(m=100_000)
    Ad = torch.from_numpy(A).cuda()
    m, n, k = A.shape[0], A.shape[1], 3
    plan = _plan(m, n, k, rl.RLOBPCG_C128)
    out = _buffers(m, n, k, torch.complex128)
    try:
        t0 = time.perf_counter()
        _run(plan, Ad, out, False)
        t_sync = time.perf_counter() - t0
        info = rl.rlobpcg_info()
        t0 = time.perf_counter()
        rl.rlobpcg_solve_async(plan, Ad.data_ptr(), n, -1.0, out["sigma"].data_ptr(), out["V"].data_ptr(), None,
                               out["resid"].data_ptr(), info)
        t_async = time.perf_counter() - t0
        # while in flight, the plan takes no other call
        with pytest.raises(rl.RlobpcgError) as e:
            rl.rlobpcg_solve(plan, Ad.data_ptr(), n, -1.0, out["sigma"].data_ptr(), out["V"].data_ptr())
        assert e.value.code == rl.RLOBPCG_ERR_INVALID_ARG
        with pytest.raises(rl.RlobpcgError):
            rl.rlobpcg_solve_async(plan, Ad.data_ptr(), n, -1.0, out["sigma"].data_ptr(), out["V"].data_ptr())
        assert rl.rlobpcg_solve_wait(plan) in (rl.RLOBPCG_OK, rl.RLOBPCG_NOT_CONVERGED)
        assert info.iters > 0
        with pytest.raises(rl.RlobpcgError):
            rl.rlobpcg_solve_wait(plan)            # nothing in flight any more
        print("sync solve %.1f ms, async call %.2f ms" % (t_sync * 1e3, t_async * 1e3))
        assert t_async < 0.5 * t_sync
    finally:
        rl.rlobpcg_plan_destroy(plan)


def test_async_error_comes_back_through_the_wait_and_destroy_waits():
    m, n, k = 5000, 60, 2
    A = np.random.default_rng(6).standard_normal((m, n))
    A[17, 3] = np.nan
    Ad = torch.from_numpy(A).cuda()
    plan = _plan(m, n, k)
    out = _buffers(m, n, k)
    try:
        rl.rlobpcg_solve_async(plan, Ad.data_ptr(), n, -1.0, out["sigma"].data_ptr(), out["V"].data_ptr())
        with pytest.raises(rl.RlobpcgError) as e:
            rl.rlobpcg_solve_wait(plan)
        assert e.value.code == rl.RLOBPCG_ERR_NONFINITE
        # a solve left in flight: the plan's destruction waits for it
        A2 = torch.from_numpy(np.random.default_rng(7).standard_normal((m, n))).cuda()
        rl.rlobpcg_solve_async(plan, A2.data_ptr(), n, -1.0, out["sigma"].data_ptr(), out["V"].data_ptr())
    finally:
        rl.rlobpcg_plan_destroy(plan)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out["sigma"].cpu().numpy()))
