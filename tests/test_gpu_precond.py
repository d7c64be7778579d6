"""The preconditioner variants of Sec. 1.1 on the GPU: the diagonally preconditioned LOBPCG
(P = diag(||A(:, i)||^{-1})) and LOBPCG without a preconditioner (P = I), both from the
sketch-and-solve start, against the oracle run with the same variant: the Ritz values after every
iteration in fixed-iteration mode (bars of tests/parity.py), real and complex, and the easy
(coherent) case of Sec. 1.1 where the diagonal preconditioner is far ahead of none."""
import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl
from tests.parity import check_sigma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = {rl.RLOBPCG_PRECOND_DIAG: "diag", rl.RLOBPCG_PRECOND_NONE: "none", rl.RLOBPCG_PRECOND_SKETCH: "sketch"}


def _solve(A, k, b, precond, fixed, split=1):
    m, n = A.shape
    o = rl.rlobpcg_default_opts()
    o.seed = 5
    o.block = b
    o.exact_sketch_svd = 1
    o.fixed_iters = fixed
    o.precond = precond
    o.gram_split = split
    cplx = np.iscomplexobj(A)
    st = torch.cuda.current_stream().cuda_stream
    plan = rl.rlobpcg_plan(m, n, k, rl.RLOBPCG_C128 if cplx else rl.RLOBPCG_F64, o, st)
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    sig = torch.empty(k, dtype=torch.float64, device="cuda")
    V = torch.empty((n, k), dtype=Ad.dtype, device="cuda")
    info = rl.rlobpcg_info()
    try:
        rl.rlobpcg_solve(plan, Ad.data_ptr(), n, -1.0, sig.data_ptr(), V.data_ptr(), None, None, info)
        th, rs = rl.rlobpcg_history(plan)
    finally:
        rl.rlobpcg_plan_destroy(plan)
    return sig.cpu().numpy(), th, info


@pytest.mark.parametrize("precond", [rl.RLOBPCG_PRECOND_DIAG, rl.RLOBPCG_PRECOND_NONE])
@pytest.mark.parametrize("cplx,split", [(False, 1), (False, 0), (True, 0)])
def test_variant_fixed_iterations_parity(precond, cplx, split):
    rng = np.random.default_rng(71)
    n = 60
    sigma = np.concatenate([np.geomspace(1.0, 1e-3, n - 2), [1e-6, 5e-7]])
    A = wl.planted(rng, 6000, sigma, complex_=cplx)[0]
    A = A * np.linspace(0.5, 2.0, n)[None, :]          # uneven column norms: diag != none
    iters = 6
    sig, th, info = _solve(A, 2, 2, precond, iters, split)
    ora = oracle.rlobpcg(A, k=2, b=2, seed=5, fixed_iters=iters, precond=NAMES[precond])
    assert info.iters == iters
    th_ora = np.vstack([ora["theta0"][None, :], ora["theta_hist"][1:]])
    for t in range(iters + 1):
        check_sigma(th[t], th_ora[t], ora["sigma11"], n)
    check_sigma(sig, ora["sigma"], ora["sigma11"], n)


def test_easy_problem_both_preconditioners_beat_none():
    """Sec. 1.1's easy problem on a small scale (coherent V, sigma geometric 1 -> 0.1 and
    sigma_n = 1e-7): after 4 iterations both preconditioners are far ahead of none. With V this
    close to the identity the columns of A are nearly orthogonal and the diagonal P P^* is nearly
    (A^* A)^{-1} (the coherent case where Sec. 1.1 notes a diagonal preconditioner works)."""
    A, s, V = wl.easy_coherent(73, 20_000, 200)
    err = {}
    for pc in (rl.RLOBPCG_PRECOND_SKETCH, rl.RLOBPCG_PRECOND_DIAG, rl.RLOBPCG_PRECOND_NONE):
        sig, th, info = _solve(A, 1, 1, pc, 4)
        err[NAMES[pc]] = abs(sig[0] - s[-1]) / s[-1]
    print(err)
    assert err["diag"] < 1e-2 * err["none"]
    assert err["sketch"] < 1e-1 * err["none"]
