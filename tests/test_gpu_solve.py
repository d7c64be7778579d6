"""End-to-end parity of rlobpcg_solve (through the C ABI) with the CPU oracle.

Each case runs the same seeded matrix and the same SparseStack seed on both sides, in adaptive
stopping mode and in fixed-iteration mode (so that a stop decision taken one check apart on the
two sides is told apart from a numerical disagreement), and checks both results against the
planted truth. Bars: see tests/parity.py.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl
from tests.parity import U, check_angle, check_sigma, check_truth, sub_sin

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu_solve(A, k, *, seed, d=None, zeta=8, b=None, tau=None, stagnation=True, fixed=0, prec="f64",
              max_iter=0, refresh=0, want_u=False, exact_svd=False, gram=None):
    o = rl.rlobpcg_default_opts()
    if gram is not None:
        o.gram_split = 1 if gram == "split" else 0
    o.exact_sketch_svd = 1 if exact_svd else 0
    o.seed = seed
    o.zeta = zeta
    o.d = d or 0
    o.block = b or 0
    o.use_stagnation = 1 if stagnation else 0
    o.fixed_iters = fixed
    o.max_iter = max_iter
    o.residual_refresh_every = refresh
    o.sketch_prec = {"f32": rl.RLOBPCG_SKETCH_F32, "f64": rl.RLOBPCG_SKETCH_F64,
                     "f32_refine": rl.RLOBPCG_SKETCH_F32_REFINE}[prec]
    if tau is not None:
        o.tau = tau
    Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    sigma, V, U_, resid, info = rl.solve(Ad, k, opts=o, want_u=want_u)
    torch.cuda.synchronize()
    return (sigma.cpu().numpy(), V.cpu().numpy(), None if U_ is None else U_.cpu().numpy(), resid.cpu().numpy(),
            info)


def ora_solve(A, k, *, seed, d=None, zeta=8, b=None, tau=None, stagnation=True, fixed=None, prec="f64",
              max_iter=None):
    return oracle.rlobpcg(A, k=k, b=b, d=d, zeta=zeta, seed=seed, tau=tau, use_stagnation=stagnation,
                          fixed_iters=fixed, sketch_precision=prec, max_iter=max_iter)


def compare(A, k, s_true, V_true, *, n, gap_abs, **kw):
    g = gpu_solve(A, k, **kw)
    okw = dict(kw)
    okw["fixed"] = kw.get("fixed") or None
    if okw.get("max_iter") == 0:
        okw["max_iter"] = None
    okw.pop("refresh", None)
    okw.pop("want_u", None)
    okw.pop("exact_svd", None)
    okw.pop("gram", None)
    o = ora_solve(A, k, **okw)
    sig, V, _, resid, info = g
    print(f"gpu: iters={info['iters']} stop={info['stop_reason']} sigma11={info['sigma11']!r} sigma={sig!r}")
    print(f"ora: iters={o['iters']} stop={o['stop_reason']} sigma11={o['sigma11']!r} sigma={o['sigma']!r}")
    print(f"ora res_hist max: {o['res_hist'].max(axis=1)[:12]!r}")
    check_sigma(sig, o["sigma"], o["sigma11"], n)
    check_angle(V, o["V"], gap_abs, n)
    if s_true is not None:
        check_truth(sig, o["sigma"], s_true, o["sigma11"], n)
    if V_true is not None:
        # both sides sit at the same distance from the planted subspace, up to the floor
        assert sub_sin(V, V_true) <= max(1e-8, 4 * sub_sin(o["V"], V_true), 10 * np.sqrt(n) * U / gap_abs)
    # invariants: orthonormal V, ||A v_j|| = sigma_j (to c u ||A||)
    assert np.allclose(V.conj().T @ V, np.eye(k), atol=100 * n * U)
    nA = o["sigma11"]
    assert np.all(np.abs(np.linalg.norm(A @ V, axis=0) - sig) <= 100 * np.sqrt(n) * U * nA + 1e-6 * sig)
    return g, o


# ---------------------------------------------------------------------------------------------
# small planted problem: m = 4000, n = 50, sigma_50 = 1e-10, k = 1, d = 4n, zeta = 8
# ---------------------------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_planted():
    return wl.planted_small_gap_free()


def test_small_planted_tau_1e12(small_planted):
    A, s, V = small_planted
    gap = (s[-2] - s[-1]) / s[0]
    g, o = compare(A, 1, s[-1:], V[:, -1:], n=50, gap_abs=gap, seed=1001, tau=1e-12, stagnation=False)
    assert g[4]["iters"] == o["iters"]


def test_small_planted_default_stop(small_planted):
    A, s, V = small_planted
    gap = (s[-2] - s[-1]) / s[0]
    g, o = compare(A, 1, s[-1:], V[:, -1:], n=50, gap_abs=gap, seed=1001)
    assert g[4]["stop_reason"] == rl.RLOBPCG_STOP_CONVERGED


@pytest.mark.parametrize("exact_svd", [False, True])
@pytest.mark.parametrize("iters", [1, 3, 12])
def test_small_planted_fixed_iterations(small_planted, iters, exact_svd):
    A, s, V = small_planted
    gap = (s[-2] - s[-1]) / s[0]
    g, o = compare(A, 1, None, None, n=50, gap_abs=gap, seed=1001, fixed=iters, exact_svd=exact_svd)
    assert g[4]["iters"] == iters and g[4]["stop_reason"] == rl.RLOBPCG_STOP_FIXED


def test_well_conditioned_literal_bars():
    """cfg1 shape with sigma_min = 1e-3 (kappa = 1e3): the literal 1e-10 sigma bar holds."""
    rng = np.random.default_rng(77)
    sigma = np.concatenate([np.logspace(0, -2, 49), [1e-3]])
    A, s, V = wl.planted(rng, 4000, sigma)
    g = gpu_solve(A, 1, seed=3)
    o = ora_solve(A, 1, seed=3)
    assert abs(g[0][0] - o["sigma"][0]) <= 1e-10 * o["sigma"][0]
    assert abs(g[0][0] - s[-1]) <= 1e-10 * s[-1]
    assert sub_sin(g[1], o["V"]) <= 1e-8


# ---------------------------------------------------------------------------------------------
# exact nullspace and planted bottom cluster, n = 500, k = 5, d = 3n (reduced m for speed)
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("gram", ["split", "fp64"])
@pytest.mark.parametrize("m", [20_000, 100_000])
def test_exact_nullspace(m, gram):
    A, C = wl.exact_nullspace(m=m)
    _, _, Vh = np.linalg.svd(C)
    null = Vh.conj().T[:, 495:]
    g = gpu_solve(A, 5, seed=1002, d=1500, gram=gram)
    o = ora_solve(A, 5, seed=1002, d=1500)
    nA = o["sigma11"]
    # sigma is at rounding level: absolute bar only
    assert np.all(np.abs(g[0] - o["sigma"]) <= 10 * np.sqrt(500) * U * nA)
    assert sub_sin(g[1], null) <= 1e-8
    assert sub_sin(g[1], o["V"]) <= 1e-8
    assert np.linalg.norm(A @ g[1], 2) <= 100 * np.sqrt(500) * U * nA


@pytest.mark.parametrize("gram", ["split", "fp64"])
@pytest.mark.parametrize("m", [20_000, 100_000])
def test_planted_bottom_cluster(m, gram):
    A, s, V = wl.planted_bottom_cluster(m=m)
    gap = (s[-6] - s[-5]) / s[0]
    compare(A, 5, s[::-1][:5], V[:, ::-1][:, :5], n=500, gap_abs=gap, seed=1002, d=1500, gram=gram)


@pytest.mark.parametrize("exact_svd", [False, True])
def test_planted_bottom_cluster_fixed_iterations(exact_svd):
    A, s, V = wl.planted_bottom_cluster(m=20_000)
    gap = (s[-6] - s[-5]) / s[0]
    compare(A, 5, None, None, n=500, gap_abs=gap, seed=1002, d=1500, fixed=8, exact_svd=exact_svd)


def test_start_block_matches_exact_sketch_svd():
    """The start block by inverse iteration + Rayleigh-Ritz spans the sketch's bottom-b right
    singular subspace (the exact V~(:, n-b+1:n)), so one iteration from either start gives the
    same block. Sigma~(1,1) by block power iteration is within 2% (it only scales the stop
    tolerance, and it estimates ||A|| only up to the sketch's distortion anyway)."""
    A, s, V = wl.planted_bottom_cluster(m=20_000)
    g0 = gpu_solve(A, 5, seed=1002, d=1500, fixed=1, exact_svd=False)
    g1 = gpu_solve(A, 5, seed=1002, d=1500, fixed=1, exact_svd=True)
    assert g0[4]["sigma11"] <= g1[4]["sigma11"] * (1 + 1e-12)
    assert abs(g0[4]["sigma11"] - g1[4]["sigma11"]) <= 2e-2 * g1[4]["sigma11"]
    assert sub_sin(g0[1], g1[1]) <= 1e-8


# ---------------------------------------------------------------------------------------------
# complex128 with the FP32 sketch (reduced m), and the mixed-precision form in general
# ---------------------------------------------------------------------------------------------

def test_complex_planted_fp64_sketch():
    """complex128, sigma logspaced 1 -> 1e-8 with the three smallest 1e-12, 3e-13, 1e-13."""
    A, s, V = wl.planted_complex(m=20_000)
    gap = (s[-4] - s[-3]) / s[0]
    compare(A, 3, s[::-1][:3], None, n=300, gap_abs=gap, seed=1003)


def test_complex_fp32_sketch_resolvable():
    """The FP32 sketch/R/R^{-1} (applied in FP64) where FP32 resolves the spectrum (kappa = 1e5):
    same answer as the oracle's FP32-sketch run."""
    rng = np.random.default_rng(1003)
    n = 120
    sigma = np.concatenate([np.logspace(0, -3, n - 3), [3e-5, 2e-5, 1e-5]])
    A, s, V = wl.planted(rng, 20_000, sigma, complex_=True)
    gap = (s[-4] - s[-3]) / s[0]
    compare(A, 3, s[::-1][:3], V[:, ::-1][:, :3], n=n, gap_abs=gap, seed=7, prec="f32")


def test_complex_fp64_sketch_fixed():
    A, s, V = wl.planted_complex(m=20_000)
    gap = (s[-4] - s[-3]) / s[0]
    compare(A, 3, None, None, n=300, gap_abs=gap, seed=1003, fixed=10)


@pytest.mark.parametrize("fixed", [0, 3, 12])
def test_refined_sketch_small(small_planted, fixed):
    """FP32 factor refined once in FP64, kappa = 1e10: parity with the oracle's refined run, in
    adaptive and fixed-iteration mode; adaptive stops after as many iterations as the oracle."""
    A, s, V = small_planted
    gap = (s[-2] - s[-1]) / s[0]
    g, o = compare(A, 1, None if fixed else s[-1:], None if fixed else V[:, -1:], n=50, gap_abs=gap, seed=1001,
                   prec="f32_refine", fixed=fixed, tau=1e-12, stagnation=False)
    if not fixed:
        assert g[4]["iters"] == o["iters"]


@pytest.mark.parametrize("fixed", [0, 10])
def test_complex_refined_sketch(fixed):
    """complex128 with the three smallest singular values 1e-13..1e-12 (kappa = 1e13), FP32
    factor refined in FP64: parity with the oracle's refined run and with the planted truth."""
    A, s, V = wl.planted_complex(m=20_000)
    gap = (s[-4] - s[-3]) / s[0]
    compare(A, 3, None if fixed else s[::-1][:3], None, n=300, gap_abs=gap, seed=1003, prec="f32_refine",
            fixed=fixed)


def test_refined_nullspace():
    """Exactly rank-deficient sketch (A = B C): the shifted Cholesky keeps the refined factor
    defined; the nullspace is found like with the FP64 factor."""
    A, C = wl.exact_nullspace(m=20_000)
    Q = np.linalg.svd(C)[2].T[:, -5:]
    sig, V, _, _, info = gpu_solve(A, 5, seed=2002, d=1500, prec="f32_refine")
    assert info["stop_reason"] == rl.RLOBPCG_STOP_CONVERGED
    assert np.all(sig <= 100 * np.sqrt(500) * U * info["sigma11"])
    assert sub_sin(V, Q) <= 1e-8


def test_mixed_precision_sketch_small(small_planted):
    A, s, V = small_planted
    gap = (s[-2] - s[-1]) / s[0]
    compare(A, 1, s[-1:], V[:, -1:], n=50, gap_abs=gap, seed=1001, prec="f32")


# ---------------------------------------------------------------------------------------------
# API behaviour: host pointers, U, determinism, block larger than k, refresh, edge sizes, errors
# ---------------------------------------------------------------------------------------------

def test_host_pointers_match_device(small_planted):
    A, s, V = small_planted
    m, n = A.shape
    o = rl.rlobpcg_default_opts()
    o.seed = 5
    plan = rl.rlobpcg_plan(m, n, 1, rl.RLOBPCG_F64, o, 0)
    try:
        Ah = np.ascontiguousarray(A)
        sig = np.zeros(1)
        Vh = np.zeros((n, 1))
        Uh = np.zeros((m, 1))
        res = np.zeros(1)
        info = rl.rlobpcg_info()
        rl.rlobpcg_solve(plan, Ah.ctypes.data, n, -1.0, sig.ctypes.data, Vh.ctypes.data, Uh.ctypes.data,
                         res.ctypes.data, info)
    finally:
        rl.rlobpcg_plan_destroy(plan)
    g = gpu_solve(A, 1, seed=5, want_u=True)
    assert np.array_equal(sig, g[0]) and np.array_equal(Vh, g[1]) and np.array_equal(Uh, g[2])
    # U = A V / sigma, up to the absolute rounding of A V (u ||A||) magnified by 1 / sigma
    assert np.linalg.norm(Uh - A @ Vh / sig[None, :]) <= 100 * np.sqrt(n) * U * s[0] / sig[0]
    assert abs(np.linalg.norm(Uh) - 1.0) <= 100 * np.sqrt(n) * U * s[0] / sig[0]


def test_deterministic(small_planted):
    A, _, _ = small_planted
    g1 = gpu_solve(A, 1, seed=9)
    g2 = gpu_solve(A, 1, seed=9)
    assert np.array_equal(g1[0], g2[0]) and np.array_equal(g1[1], g2[1]) and g1[4]["iters"] == g2[4]["iters"]


def test_block_larger_than_k():
    rng = np.random.default_rng(4)
    n = 60
    sigma = np.concatenate([np.logspace(0, -5, n - 3), [3e-9, 2e-9, 1e-9]])
    A, s, V = wl.planted(rng, 5000, sigma)
    gap = (s[-2] - s[-1]) / s[0]
    g = gpu_solve(A, 1, seed=2, b=3, max_iter=40)
    o = ora_solve(A, 1, seed=2, b=3, max_iter=40)
    check_sigma(g[0], o["sigma"], o["sigma11"], n)
    check_angle(g[1], o["V"], gap, n)


def test_residual_refresh_does_not_change_the_answer(small_planted):
    A, s, V = small_planted
    g0 = gpu_solve(A, 1, seed=1, fixed=15)
    g1 = gpu_solve(A, 1, seed=1, fixed=15, refresh=3)
    assert abs(g0[0][0] - g1[0][0]) <= 10 * np.sqrt(50) * U
    assert sub_sin(g0[1], g1[1]) <= 1e-8


@pytest.mark.parametrize("m,n,k", [(3, 3, 1), (64, 6, 2), (1000, 3, 1), (200, 199, 1)])
def test_edge_shapes(m, n, k):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)) @ np.diag(np.logspace(0, -3, n))
    g = gpu_solve(A, k, seed=1, d=max(4 * n, 8), max_iter=50)
    _, s, Vh = np.linalg.svd(A, full_matrices=False)
    assert np.allclose(np.sort(g[0]), np.sort(s[-k:]), rtol=1e-8, atol=10 * np.sqrt(n) * U * s[0])


def test_loewner_backward_error():
    L = wl.loewner(seed=50000, m=20000, n=120)
    g = gpu_solve(L, 2, seed=3, max_iter=60)
    nL = np.linalg.norm(L)
    assert np.linalg.norm(L @ g[1], 2) <= 50 * U * nL * np.sqrt(120)
    assert np.allclose(g[1].T @ g[1], np.eye(2), atol=1e-12)


@pytest.mark.parametrize("gram", ["split", "fp64"])
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_input_is_reported(gram, bad):
    A = np.random.default_rng(0).standard_normal((500, 20))
    A[123, 7] = bad
    with pytest.raises(rl.RlobpcgError) as e:
        gpu_solve(A, 1, seed=1, gram=gram)
    assert e.value.code == rl.RLOBPCG_ERR_NONFINITE


def test_invalid_arguments():
    h = ctypes.c_void_p()
    lib = rl.load()
    assert lib.rlobpcg_plan(ctypes.byref(h), 100, 30, 11, 0, None, None) == rl.RLOBPCG_ERR_INVALID_ARG
    assert lib.rlobpcg_solve(None, None, 0, -1.0, None, None, None, None, None) == rl.RLOBPCG_ERR_INVALID_ARG
