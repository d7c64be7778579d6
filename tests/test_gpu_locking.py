"""SVQB orthonormalisation (Sec. 2.1) and locking of converged columns (Sec. 2.3) on the GPU,
against the oracle run with the same options.

SVQB: in fixed-iteration mode the per-iteration Ritz values and the final triplets match the
oracle's SVQB run (bars of tests/parity.py) and the returned V is orthonormal.

Locking: a column whose residual norm meets sigma11^2 tau is moved out of the active block; the
solve then runs Rayleigh-Ritz on the active columns only and keeps W orthogonal to the locked
ones. The cases below are chosen so that every lock decision of the oracle sits at least 1.5 %
(in relative residual) away from the threshold -- far more than the GPU's rounding moves a
residual that large -- so the GPU must take the same decisions: the same iterations and the same
matrix-vector count b + sum of the active widths, the same locked slots frozen in the history from
the iteration they locked, and sigma within the parity bars.
"""
import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl
from tests.parity import check_sigma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


def _run(A, k, b, *, fixed=None, tau=None, d=None, zeta=None, svqb=False, locking=False, split=1):
    m, n = A.shape
    o = rl.rlobpcg_default_opts()
    o.seed = 11
    o.block = b
    o.exact_sketch_svd = 1      # the oracle's start block: V~(:, n-b+1:n) of the full sketch SVD
    o.gram_split = split
    o.orth_mode = rl.RLOBPCG_ORTH_SVQB if svqb else rl.RLOBPCG_ORTH_HOUSEHOLDER
    o.locking = 1 if locking else 0
    if fixed:
        o.fixed_iters = fixed
    if tau is not None:
        o.tau = tau
        o.use_stagnation = 0
        o.check_every = 1
    if d is not None:
        o.d = d
    if zeta is not None:
        o.zeta = zeta
    cplx = np.iscomplexobj(A)
    st = torch.cuda.current_stream().cuda_stream
    plan = rl.rlobpcg_plan(m, n, k, rl.RLOBPCG_C128 if cplx else rl.RLOBPCG_F64, o, st)
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    sig = torch.empty(k, dtype=torch.float64, device="cuda")
    Vg = torch.empty((n, k), dtype=Ad.dtype, device="cuda")
    Ug = torch.empty((m, k), dtype=Ad.dtype, device="cuda")
    res = torch.empty(k, dtype=torch.float64, device="cuda")
    info = rl.rlobpcg_info()
    try:
        rl.rlobpcg_solve(plan, Ad.data_ptr(), n, -1.0, sig.data_ptr(), Vg.data_ptr(), Ug.data_ptr(),
                         res.data_ptr(), info)
        th, rs = rl.rlobpcg_history(plan)
    finally:
        rl.rlobpcg_plan_destroy(plan)
    ora = oracle.rlobpcg(A, k=k, b=b, seed=11, fixed_iters=fixed, tau=tau, d=d, zeta=8 if zeta is None else zeta,
                         use_stagnation=tau is None, check_every=1 if tau is not None else None,
                         orth_mode="svqb" if svqb else "householder", locking=locking)
    return info, sig.cpu().numpy(), Vg.cpu().numpy(), Ug.cpu().numpy(), res.cpu().numpy(), th, rs, ora


def _check_triplets(A, sig, V, Uo, sigma11):
    n = A.shape[1]
    assert np.all(np.diff(sig) >= 0)
    np.testing.assert_allclose(V.conj().T @ V, np.eye(V.shape[1]), atol=1e3 * U * np.sqrt(n))
    # U = A V diag(sigma)^{-1}
    np.testing.assert_allclose(Uo * sig[None, :], A @ V, atol=1e2 * np.sqrt(n) * U * sigma11)


@pytest.fixture(scope="module")
def clustered_small():
    return wl.clustered(1006, 20_000, 200)[0]


@pytest.mark.parametrize("b,split", [(5, 1), (5, 0), (10, 1)])
def test_svqb_fixed_iterations_parity(clustered_small, b, split):
    A = clustered_small
    iters = 6
    info, sig, V, Uo, res, th, rs, ora = _run(A, 3, b, fixed=iters, svqb=True, split=split)
    assert info.iters == iters and info.matvecs == b * (iters + 1) == ora["matvecs"]
    th_ora = np.vstack([ora["theta0"][None, :], ora["theta_hist"][1:]])
    for t in range(iters + 1):
        check_sigma(th[t, -3:], th_ora[t, -3:], ora["sigma11"], A.shape[1])
    check_sigma(sig, ora["sigma"], ora["sigma11"], A.shape[1])
    _check_triplets(A, sig, V, Uo, ora["sigma11"])


def _lock_case(name):
    if name == "condition_1e8":
        return wl.condition_sweep(7, 1e8)[0], dict(tau=1e-10, d=110, zeta=1)
    if name == "gap_1e-2":
        return wl.gap_sweep(7, 1e-2)[0], dict(tau=1e-10, d=120, zeta=1)
    if name == "clustered":
        return wl.clustered(1006, 20_000, 200)[0], dict(tau=1e-12, d=220, zeta=1)
    if name == "complex":
        A = wl.planted(np.random.default_rng(21), 10_000, np.geomspace(1.0, 1e-6, 100), complex_=True)[0]
        return A, dict(tau=1e-12)
    raise KeyError(name)


def _first_lock(rh, thr):
    return [int(np.argmax(rh[:, j] <= thr)) if (rh[:, j] <= thr).any() else -1 for j in range(rh.shape[1])]


@pytest.mark.parametrize("name,svqb", [("condition_1e8", False), ("gap_1e-2", False), ("clustered", False),
                                       ("complex", False), ("condition_1e8", True)])
def test_locking_parity(name, svqb):
    A, kw = _lock_case(name)
    b, k = 5, 3
    info, sig, V, Uo, res, th, rs, ora = _run(A, k, b, svqb=svqb, locking=True, **kw)
    thr = ora["sigma11"] ** 2 * kw["tau"]
    margin = np.min(np.abs(np.log(ora["res_hist"][1:] / thr)))
    assert margin > 0.015, margin          # the case's decisions are well away from the threshold
    print(name, "iters", info.iters, "matvecs", info.matvecs, "locked", ora["locked"])
    assert ora["locked"].any()
    assert info.iters == ora["iters"] and info.matvecs == ora["matvecs"]
    assert rs.shape == ora["res_hist"].shape
    # the same slots lock at the same iterations; a locked slot's history is frozen from then on
    assert _first_lock(rs, thr) == _first_lock(ora["res_hist"], thr)
    for j, t0 in enumerate(_first_lock(rs, thr)):
        if 0 < t0 < rs.shape[0] - 1 and ora["locked"][j]:
            assert np.all(rs[t0:, j] == rs[t0, j]) and np.all(th[t0:, j] == th[t0, j])
    check_sigma(sig, ora["sigma"], ora["sigma11"], A.shape[1])
    _check_triplets(A, sig, V, Uo, ora["sigma11"])


def test_locking_ends_fixed_iterations_once_every_column_locked(clustered_small):
    """A tolerance every column meets after the first iteration: the fixed-iteration solve ends
    there (Sec. 2.3: nothing is left to iterate on), with the oracle's count."""
    A = clustered_small
    info, sig, V, Uo, res, th, rs, ora = _run(A, 3, 5, fixed=8, tau=1e-9, locking=True)
    assert ora["iters"] == 1 and ora["locked"].all()
    assert info.iters == 1 and info.matvecs == ora["matvecs"] == 10
    assert info.stop_reason == rl.RLOBPCG_STOP_FIXED
    check_sigma(sig, ora["sigma"], ora["sigma11"], A.shape[1])
    _check_triplets(A, sig, V, Uo, ora["sigma11"])
