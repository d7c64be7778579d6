"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the passage of arXiv 2602.16797 (section, algorithm, fact or theorem) or the
external definition it checks against. All run on the CPU (no GPU marker).
"""
import os

import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = 2.0 ** -53


def _subspace_sin(V1, V2):
    """Largest principal angle (its sine) between span(V1) and span(V2), both orthonormal."""
    Q1, _ = np.linalg.qr(V1)
    Q2, _ = np.linalg.qr(V2)
    # ||(I - Q2 Q2^H) Q1||_2; sqrt(1 - cos^2) would lose half the digits
    return float(np.linalg.norm(Q1 - Q2 @ (Q2.conj().T @ Q1), 2))


def _distortion(A, S):
    """Distortion eta of S on range(A) (Definition of a subspace embedding, Sec. 1.2):
    the extreme squared singular values of S Q_A are 1 -+ eta."""
    Q, _ = np.linalg.qr(A)
    s = np.linalg.svd(S @ Q, compute_uv=False)
    return float(max(s.max() ** 2 - 1.0, 1.0 - s.min() ** 2))


# ---------------------------------------------------------------------------------------------
# The two products of one iteration: A W and A^H (A W) (Alg. 2)
# ---------------------------------------------------------------------------------------------

def _int_matrix(rng, rows, cols, complex_, lim=60):
    re = rng.integers(-lim, lim + 1, size=(rows, cols))
    if not complex_:
        return re.astype(np.int64)
    return re + 1j * rng.integers(-lim, lim + 1, size=(rows, cols))


def _exact_products(A, W):
    """A W and A^H (A W) by definition, in Python integers (Gaussian integers for complex data):
    (A W)_ij = sum_k a_ik w_kj and (A^H Y)_kj = sum_i conj(a_ik) y_ij, with no rounding at all."""
    m, n = A.shape
    b = W.shape[1]
    cplx = np.iscomplexobj(A)
    to = (lambda z: (int(z.real), int(z.imag))) if cplx else (lambda z: (int(z), 0))
    a = [[to(A[i, k]) for k in range(n)] for i in range(m)]
    w = [[to(W[k, j]) for j in range(b)] for k in range(n)]
    mul = lambda x, y: (x[0] * y[0] - x[1] * y[1], x[0] * y[1] + x[1] * y[0])  # noqa: E731
    Y = [[(sum(mul(a[i][k], w[k][j])[0] for k in range(n)), sum(mul(a[i][k], w[k][j])[1] for k in range(n)))
          for j in range(b)] for i in range(m)]
    G = [[(sum(mul((a[i][k][0], -a[i][k][1]), Y[i][j])[0] for i in range(m)),
           sum(mul((a[i][k][0], -a[i][k][1]), Y[i][j])[1] for i in range(m))) for j in range(b)] for k in range(n)]
    return Y, G


@pytest.mark.parametrize("complex_", [False, True])
def test_gram_pass_exact_on_integers(complex_):
    """On small integer (Gaussian-integer) data every product and partial sum of A W and
    A^H (A W) is an integer below 2^53, so float64 arithmetic is exact and the oracle must agree
    bit for bit with the definition of the two products (conjugate transpose in the second)."""
    rng = np.random.default_rng(31)
    A = _int_matrix(rng, 29, 11, complex_)
    W = _int_matrix(rng, 11, 3, complex_)
    Y, G = _exact_products(A, W)
    AW, GW = oracle.gram_pass(A.astype(np.complex128 if complex_ else np.float64),
                              W.astype(np.complex128 if complex_ else np.float64))
    assert max(abs(v) for row in Y for c in row for v in c) < 2 ** 53
    assert max(abs(v) for row in G for c in row for v in c) < 2 ** 53
    for i in range(A.shape[0]):
        for j in range(W.shape[1]):
            assert AW[i, j].real == Y[i][j][0] and np.imag(AW[i, j]) == Y[i][j][1], (i, j)
    for k in range(A.shape[1]):
        for j in range(W.shape[1]):
            assert GW[k, j].real == G[k][j][0] and np.imag(GW[k, j]) == G[k][j][1], (k, j)


def test_gram_pass_within_rounding_of_exact_rationals():
    """Non-integer data: the exact products in rational arithmetic (every float64 is a dyadic
    rational) against the oracle's float64 products, within the standard dot-product bound
    gamma_n |A| |W| (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 3.1), and for
    the second product gamma_m |A|^T |A W| plus the first product's error carried through A^T."""
    from fractions import Fraction
    rng = np.random.default_rng(32)
    m, n, b = 13, 7, 2
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-3, 3, (m, n)))
    W = rng.standard_normal((n, b))
    AW, GW = oracle.gram_pass(A, W)
    Af = [[Fraction(float(x)) for x in row] for row in A]
    Wf = [[Fraction(float(x)) for x in row] for row in W]
    Yf = [[sum(Af[i][k] * Wf[k][j] for k in range(n)) for j in range(b)] for i in range(m)]
    Gf = [[sum(Af[i][k] * Yf[i][j] for i in range(m)) for j in range(b)] for k in range(n)]
    u = 2.0 ** -53
    gam = lambda p: p * u / (1 - p * u)  # noqa: E731
    absA = np.abs(A)
    bY = gam(n) * (absA @ np.abs(W))
    bG = gam(m) * (absA.T @ np.abs(AW)) + absA.T @ bY * (1 + gam(m))
    for i in range(m):
        for j in range(b):
            assert abs(Fraction(float(AW[i, j])) - Yf[i][j]) <= Fraction(float(bY[i, j])) * Fraction(101, 100)
    for k in range(n):
        for j in range(b):
            assert abs(Fraction(float(GW[k, j])) - Gf[k][j]) <= Fraction(float(bG[k, j])) * Fraction(101, 100)


# ---------------------------------------------------------------------------------------------
# SplitMix64 and the SparseStack pattern (Sec. 2.2)
# ---------------------------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 8
    for seed, idx, out in rows:
        got = int(oracle.splitmix64(int(seed), int(idx)))
        assert got == int(out), (seed, idx)


@pytest.mark.parametrize("m,d,zeta", [(500, 200, 8), (777, 1500, 8), (300, 37, 4), (64, 8, 8)])
def test_sparse_stack_structure(m, d, zeta):
    """Each column of S has exactly one +-zeta^{-1/2} in each of its zeta pieces, the pieces are
    [floor(jd/zeta), floor((j+1)d/zeta)), and every column has unit norm (Sec. 2.2)."""
    dest, sign = oracle.sparse_stack(m, d, zeta, seed=11)
    b = np.array([(j * d) // zeta for j in range(zeta + 1)])
    for j in range(zeta):
        assert np.all(dest[:, j] >= b[j]) and np.all(dest[:, j] < b[j + 1])
    assert set(np.unique(sign)) <= {1.0, -1.0}
    S = oracle.sketch_dense_matrix(m, d, zeta, seed=11)
    assert np.all(np.count_nonzero(S, axis=0) == zeta)
    np.testing.assert_allclose(np.linalg.norm(S, axis=0), 1.0, rtol=0, atol=4 * U64)
    assert np.all(np.abs(S[S != 0]) == 1.0 / np.sqrt(zeta))


def test_sparse_stack_uniform_positions_and_signs():
    """Positions are uniform inside each piece and signs are fair coins (chi-square / binomial
    bounds at very small false-alarm probability); E[S^T S] = I off the diagonal."""
    m, d, zeta = 200_000, 40, 4
    dest, sign = oracle.sparse_stack(m, d, zeta, seed=3)
    for j in range(zeta):
        lo = (j * d) // zeta
        counts = np.bincount(dest[:, j] - lo, minlength=d // zeta)
        e = m / (d // zeta)
        chi2 = float(((counts - e) ** 2 / e).sum())
        assert chi2 < 60.0, chi2            # 9 dof: P(chi2 > 60) ~ 1e-9
    frac = (sign > 0).mean()
    assert abs(frac - 0.5) < 6 * 0.5 / np.sqrt(sign.size)
    S = oracle.sketch_dense_matrix(4000, 64, 8, seed=5)
    G = S.T @ S
    off = G[~np.eye(G.shape[0], dtype=bool)]
    assert abs(off.mean()) < 1e-3


def test_sketch_matches_dense_S_on_integers():
    """SA = S A exactly for small-integer A (all partial sums exact in float64)."""
    rng = np.random.default_rng(0)
    m, n, d, zeta = 700, 9, 40, 4
    A = rng.integers(-50, 50, size=(m, n)).astype(np.float64)
    S = oracle.sketch_dense_matrix(m, d, zeta, seed=9)
    got = oracle.sketch(A, d, zeta, seed=9) * np.sqrt(zeta)
    want = (S * np.sqrt(zeta)) @ A
    assert np.array_equal(np.round(want), got)
    Ac = A + 1j * rng.integers(-50, 50, size=(m, n))
    gotc = oracle.sketch(Ac, d, zeta, seed=9) * np.sqrt(zeta)
    assert np.array_equal(np.round((S * np.sqrt(zeta)) @ Ac.real), gotc.real)
    assert np.array_equal(np.round((S * np.sqrt(zeta)) @ Ac.imag), gotc.imag)


@pytest.mark.parametrize("precision,dt", [("f64", np.float64), ("f32", np.float32)])
def test_sketch_sums_in_ascending_source_order(precision, dt):
    """The documented summation order (ascending source row per destination, one scaling at the
    end) holds bit for bit: compared with an explicit sequential loop."""
    rng = np.random.default_rng(1)
    m, n, d, zeta = 300, 5, 24, 3
    A = rng.standard_normal((m, n)) * np.exp(rng.uniform(-20, 20, (m, 1)))
    dest, sign = oracle.sparse_stack(m, d, zeta, seed=4)
    acc = np.zeros((d, n), dtype=dt)
    Aw = A.astype(dt)
    for i in range(m):
        for j in range(zeta):
            acc[dest[i, j]] = acc[dest[i, j]] + dt(sign[i, j]) * Aw[i]
    want = acc * dt(1.0 / np.sqrt(zeta))
    got = oracle.sketch(A, d, zeta, seed=4, precision=precision)
    assert got.dtype == dt
    assert np.array_equal(got, want)


# ---------------------------------------------------------------------------------------------
# Sketch factorisation, preconditioner and start (Sec. 2.1, Sec. 3.1 Facts)
# ---------------------------------------------------------------------------------------------

def test_sketch_svd_is_svd_of_sketch():
    """Sigma~ and V~ reproduce (SA)^H (SA) = V~ Sigma~^2 V~^H and R^H R of a Householder QR."""
    rng = np.random.default_rng(2)
    SA = rng.standard_normal((160, 40)) @ np.diag(np.logspace(0, -5, 40))
    s, V = oracle.sketch_svd(SA)
    assert np.all(np.diff(s) <= 0)
    G = SA.T @ SA
    np.testing.assert_allclose(V @ np.diag(s ** 2) @ V.T, G, atol=50 * U64 * s[0] ** 2)
    R = oracle.householder_r(SA)
    assert np.all(np.diag(R) >= 0) and np.allclose(np.tril(R, -1), 0)
    np.testing.assert_allclose(R.T @ R, G, atol=50 * U64 * s[0] ** 2)


@pytest.mark.parametrize("complex_", [False, True])
def test_randomized_preconditioning_fact(complex_):
    """Fact (randomized preconditioning, Sec. 3.1): with P = V~ Sigma~^{-1} the squared singular
    values of A P lie in [1/(1+eta), 1/(1-eta)] for the measured distortion eta of S."""
    rng = np.random.default_rng(5)
    m, n, zeta = 3000, 40, 8
    sigma = np.logspace(0, -9, n)
    A, _, _ = wl.planted(rng, m, sigma, complex_=complex_)
    d = 16 * n        # d = 4n gives eta ~ 1 in this squared-norm definition; the Fact needs eta < 1
    S = oracle.sketch_dense_matrix(m, d, zeta, seed=21)
    eta = _distortion(A, S)
    assert 0 < eta < 1
    s, V = oracle.sketch_svd(oracle.sketch(A, d, zeta, seed=21))
    P = V / s[None, :]
    sv = np.linalg.svd(A @ P, compute_uv=False)
    slack = 1e-6      # the rounding of a kappa = 1e9 problem
    assert sv.max() ** 2 <= 1.0 / (1.0 - eta) + slack
    assert sv.min() ** 2 >= 1.0 / (1.0 + eta) - slack
    # sharper: the singular values of A P are exactly the reciprocals of those of S Q_A
    Q, _ = np.linalg.qr(A)
    ssq = np.linalg.svd(S @ Q, compute_uv=False)
    np.testing.assert_allclose(np.sort(sv), np.sort(1.0 / ssq), rtol=1e-6)


@pytest.mark.parametrize("complex_,kappa", [(False, 1e10), (True, 1e13)])
def test_refined_factor_is_a_qr_factor_of_the_sketch(complex_, kappa):
    """The FP32 factor corrected once in FP64 (sketch precision 'f32_refine') is an FP64-quality
    QR factor of the sketch: R^H R = (SA)^H (SA) up to the Cholesky shift s = n u max_i H_ii
    times ||R_32||^2 and FP64 rounding, where the FP32 factor alone is off by u_32 ||SA||^2."""
    rng = np.random.default_rng(41)
    m, n, zeta = 3000, 40, 8
    sigma = np.logspace(0, -np.log10(kappa), n)
    A, _, _ = wl.planted(rng, m, sigma, complex_=complex_)
    SA = oracle.sketch(A, 4 * n, zeta, seed=22)
    R = oracle.refined_factor(SA)
    G = SA.conj().T @ SA
    nrm = np.linalg.norm(SA, 2) ** 2
    assert np.allclose(np.tril(R, -1), 0)
    assert np.linalg.norm(R.conj().T @ R - G, 2) <= 100 * n * U64 * nrm
    low = np.complex64 if complex_ else np.float32
    R32 = np.linalg.qr(SA.astype(low), mode="r").astype(SA.dtype)
    assert np.linalg.norm(R32.conj().T @ R32 - G, 2) > 1000 * n * U64 * nrm   # what the FP64 step removes


@pytest.mark.parametrize("complex_", [False, True])
def test_refined_factor_satisfies_the_preconditioning_fact(complex_):
    """Fact (randomized preconditioning, Sec. 3.1) for P = R^{-1} with the refined factor, at
    kappa(A) = 1e10 where an FP32 factor alone leaves kappa(A R_32^{-1}) ~ u_32 kappa(A)."""
    rng = np.random.default_rng(42)
    m, n, zeta = 3000, 40, 8
    sigma = np.logspace(0, -10, n)
    A, _, _ = wl.planted(rng, m, sigma, complex_=complex_)
    d = 16 * n
    S = oracle.sketch_dense_matrix(m, d, zeta, seed=23)
    eta = _distortion(A, S)
    assert 0 < eta < 1
    R = oracle.refined_factor(oracle.sketch(A, d, zeta, seed=23))
    sv = np.linalg.svd(A @ np.linalg.inv(R), compute_uv=False)
    slack = 1e-4
    assert sv.max() ** 2 <= 1.0 / (1.0 - eta) + slack
    assert sv.min() ** 2 >= 1.0 / (1.0 + eta) - slack


def test_refined_solve_matches_the_fp64_solve():
    """The whole method with the refined factor behaves like the FP64 form on a kappa = 1e10
    planted problem (tolerance 1e-12 of the 4000 x 50 configuration): the same number of
    iterations and the same sigma to 1e-10 relative, where the FP32 factor alone needs more."""
    A, s, V = wl.planted_small_gap_free(m=4000, n=50)
    r64 = oracle.rlobpcg(A, k=1, seed=3, tau=1e-12, use_stagnation=False)
    rrf = oracle.rlobpcg(A, k=1, seed=3, tau=1e-12, use_stagnation=False, sketch_precision="f32_refine")
    r32 = oracle.rlobpcg(A, k=1, seed=3, tau=1e-12, use_stagnation=False, sketch_precision="f32")
    assert rrf["iters"] == r64["iters"]
    assert abs(rrf["sigma"][0] - r64["sigma"][0]) <= 1e-10 * r64["sigma"][0]
    assert rrf["iters"] < r32["iters"]


def test_sketch_and_solve_fact():
    """Fact (sketch-and-solve, Sec. 3.1): v0 = P e_n / ||P e_n|| satisfies
    ||A v0||^2 <= (1+eta)/(1-eta) sigma_min(A)^2."""
    rng = np.random.default_rng(6)
    m, n, zeta = 4000, 50, 8
    sigma = np.concatenate([np.logspace(0, -3, n - 1), [1e-5]])
    A, s_true, _ = wl.planted(rng, m, sigma)
    d = 16 * n
    S = oracle.sketch_dense_matrix(m, d, zeta, seed=8)
    eta = _distortion(A, S)
    assert eta < 1
    s, V = oracle.sketch_svd(oracle.sketch(A, d, zeta, seed=8))
    v0 = V[:, -1]
    lhs = np.linalg.norm(A @ v0) ** 2
    assert lhs <= (1 + eta) / (1 - eta) * s_true[-1] ** 2 * (1 + 1e-8)


# ---------------------------------------------------------------------------------------------
# The full method against closed forms and dense SVD
# ---------------------------------------------------------------------------------------------

def test_planted_small_workload():
    """4000 x 50, sigma_50 = 1e-10: converges to the planted sigma and vector within the
    backward-stable floors u sigma_1/sigma_min (value) and u/gap_abs (vector) (Sec. 4)."""
    A, s, V = wl.planted_small_gap_free()
    r = oracle.rlobpcg(A, k=1, zeta=8, seed=7)
    assert r["stop_reason"] == "converged"
    rel = abs(r["sigma"][0] - s[-1]) / s[-1]
    assert rel < 10 * U64 * s[0] / s[-1]
    gap_abs = (s[-2] - s[-1]) / s[0]
    assert _subspace_sin(r["V"], V[:, -1:]) < 10 * U64 / gap_abs
    # invariants: ||A v|| = sigma, unit v, residual below the sketched tolerance at stop
    np.testing.assert_allclose(np.linalg.norm(A @ r["V"][:, 0]), r["sigma"][0], rtol=1e-5)
    np.testing.assert_allclose(np.linalg.norm(r["V"][:, 0]), 1.0, atol=1e-14)
    assert r["resid"][0] <= r["sigma11"] ** 2 * oracle.default_tau(50)


@pytest.mark.parametrize("complex_", [False, True])
def test_block_planted_cluster(complex_):
    """Block version (Alg. 2), k = b = 3 with a clustered bottom: the 3-dim subspace and all three
    values match the planted ones; V^H V = I and ||A v_j|| = sigma_j."""
    rng = np.random.default_rng(12)
    n, k = 45, 3
    sigma = np.concatenate([np.logspace(0, -4, n - k), [3e-9, 2e-9, 1e-9]])
    A, s, V = wl.planted(rng, 3000, sigma, complex_=complex_)
    # the per-column stagnation checks rarely all hold at once for b = 3 (Sec. 4.2 notes that
    # larger blocks forestall termination), so cap the run; the accuracy is what is pinned
    r = oracle.rlobpcg(A, k=k, seed=3, max_iter=40)
    np.testing.assert_allclose(r["sigma"], s[::-1][:k], rtol=20 * U64 * s[0] / s[-1])
    gap_abs = (s[-k - 1] - s[-k]) / s[0]
    assert _subspace_sin(r["V"], V[:, -k:]) < 20 * U64 / gap_abs
    np.testing.assert_allclose(r["V"].conj().T @ r["V"], np.eye(k), atol=1e-13)
    np.testing.assert_allclose(np.linalg.norm(A @ r["V"], axis=0), r["sigma"], rtol=1e-5)


def test_dense_svd_agreement():
    """Well-conditioned small case: sigma to 1e-10 relative and the subspace to 1e-8 against
    LAPACK's dense SVD of A."""
    rng = np.random.default_rng(13)
    A = rng.standard_normal((1500, 36)) @ np.diag(np.linspace(1, 3, 36))
    r = oracle.rlobpcg(A, k=2, seed=1)
    _, s, Vh = np.linalg.svd(A, full_matrices=False)
    np.testing.assert_allclose(r["sigma"], s[::-1][:2], rtol=1e-10)
    assert _subspace_sin(r["V"], Vh.T[:, -2:]) < 1e-8


def test_exact_nullspace():
    """A = B C with B 3000 x 57, C 57 x 60: V spans null(C) and ||A V|| is at rounding level."""
    A, C = wl.exact_nullspace(seed=5, m=3000, n=60, rank=57)
    r = oracle.rlobpcg(A, k=3, d=3 * 60, seed=2)
    _, _, Vh = np.linalg.svd(C)
    null = Vh.conj().T[:, 57:]
    assert _subspace_sin(r["V"], null) < 1e-10
    nA = np.linalg.norm(A, 2)
    assert np.linalg.norm(A @ r["V"], 2) < 100 * U64 * nA * np.sqrt(60)


def test_loewner_backward_error():
    """Loewner matrix (Sec. 5 family): sigma_min is at noise level, so only the backward error
    ||L V|| <= c u ||L||_F and orthonormality are pinned (parity unpinned in sigma and V)."""
    L = wl.loewner(seed=4, m=2500, n=40)
    r = oracle.rlobpcg(L, k=2, seed=6)
    assert np.linalg.norm(L @ r["V"], 2) <= 50 * U64 * np.linalg.norm(L) * np.sqrt(40)
    np.testing.assert_allclose(r["V"].T @ r["V"], np.eye(2), atol=1e-13)


def test_theorem1_geometric_rate():
    """Theorem 1: when eta < gap/(2+gap), (||A v_k||^2 - sigma_n^2)/sigma_n^2 <= C gap q^{2k}
    with q = eta + (1-eta)/(1+gap) and C = 2 eta / ((1-eta) gap - 2 eta)."""
    rng = np.random.default_rng(21)
    m, n, zeta = 4000, 40, 8
    s_n, gap = 1e-2, 3.0
    sigma = np.concatenate([np.geomspace(1.0, 0.1, n - 2), [s_n * np.sqrt(1 + gap), s_n]])
    A, _, _ = wl.planted(rng, m, sigma)
    d = 12 * n
    S = oracle.sketch_dense_matrix(m, d, zeta, seed=14)
    eta = _distortion(A, S)
    assert eta < gap / (2 + gap)
    q = eta + (1 - eta) / (1 + gap)
    Cc = 2 * eta / ((1 - eta) * gap - 2 * eta)
    r = oracle.rlobpcg(A, k=1, d=d, zeta=zeta, seed=14, fixed_iters=12)
    thetas = np.concatenate([r["theta0"][-1:], r["theta_hist"][1:, -1]])
    floor = 100 * U64 * (sigma[0] / s_n) ** 2
    for kk, th in enumerate(thetas):
        lhs = (th ** 2 - s_n ** 2) / s_n ** 2
        assert lhs <= Cc * gap * q ** (2 * kk) + floor, (kk, lhs)


# ---------------------------------------------------------------------------------------------
# Stopping rule on hand-worked histories (Sec. 2.1)
# ---------------------------------------------------------------------------------------------

def _hist(vals_by_t):
    return [np.array([v]) for v in vals_by_t]


def test_stop_rule_hand_worked():
    inf = np.inf
    # residual norms r_0..r_11 and estimates theta_0 (= inf) .. theta_11
    r = _hist([1.0, .5, .4, .3, .2, .1, 1e-20, 1e-20, 1e-20, 1e-20, 1e-20, 1e-20])
    th_stag = _hist([inf, 4.0, 3.9, 3.5, 3.2, 3.1, 3.0, 2.8, 2.5, 2.2, 2.1, 2.0])
    th_conv = _hist([inf, 4.0, 3.0, 2.7, 2.4, 2.2, 2.0, 1.9, 1.8, 1.7, 1.6, 1.5])
    # i = 10: tol (1e-20 <= 1 * 1e-16), stag1 (1.1e-20 >= r_6 = 1e-20),
    # stag2: 1.1 (3.0 - 2.0)/2.0 = 0.55 >= (4.0 - 3.0)/3.0 = 0.333 -> stop
    assert oracle.stop_check(10, r, th_stag, 1.0, 1e-16, True) == (True, True, True)
    # stag2: 1.1 (2.0 - 1.5)/1.5 = 0.367 < (4.0 - 2.0)/2.0 = 1.0 -> keep going
    assert oracle.stop_check(10, r, th_conv, 1.0, 1e-16, True) == (True, True, False)
    # i = 5: theta_{-4} does not exist (+inf) -> stag2 false; r_1 = 0.5 > 1.1 r_6 -> stag1 false
    assert oracle.stop_check(5, r, th_stag, 1.0, 1e-16, True) == (True, False, False)
    # tolerance scaled by Sigma~(1,1)^2: 1e-20 > 1e-4^2 * 1e-16
    assert oracle.stop_check(10, r, th_stag, 1e-4, 1e-16, True)[0] is False
    # without stagnation checks only the tolerance counts
    assert oracle.stop_check(0, _hist([1.0, 1e-20]), _hist([inf, 1.0]), 1.0, 1e-16, False) == (True, True, True)


def test_earliest_stagnation_stop_is_iteration_10():
    """With stagnation checks on, no stop can happen before i = 10 (11 iterations)."""
    A, _, _ = wl.planted_small_gap_free(m=2000, n=30)
    r = oracle.rlobpcg(A, k=1, seed=1)
    assert r["iters"] >= 11 and (r["iters"] - 1) % 5 == 0


# ---------------------------------------------------------------------------------------------
# SVQB (Sec. 2.1) and locking (Sec. 2.3)
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("complex_", [False, True])
def test_svqb_orthonormalises_and_keeps_the_span(complex_):
    """SVQB (Stathopoulos & Wu 2002) returns orthonormal columns spanning those of W, to about
    u kappa(W D)^2 (D the column scaling); on columns that are already orthogonal, W D is
    orthonormal, so the result is W D times an orthogonal matrix."""
    rng = np.random.default_rng(51)
    n, b = 300, 6
    G = rng.standard_normal((n, b)) + (1j * rng.standard_normal((n, b)) if complex_ else 0)
    W = G @ np.diag(np.logspace(0, -3, b)) @ (rng.standard_normal((b, b)) + 3 * np.eye(b))
    Q = oracle.svqb(W)
    kap = np.linalg.cond(W / np.linalg.norm(W, axis=0))
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(b), 2) <= 100 * U64 * kap ** 2
    Qw, _ = np.linalg.qr(W)
    assert np.linalg.norm(Q - Qw @ (Qw.conj().T @ Q), 2) <= 100 * U64 * kap ** 2
    # already orthogonal columns of different norms
    Qo, _ = np.linalg.qr(G)
    Wo = Qo * np.array([1e-3, 1.0, 7.0, 1e5, 0.5, 2.0])[None, :]
    Z = (Wo / np.linalg.norm(Wo, axis=0)).conj().T @ oracle.svqb(Wo)
    assert np.allclose(Z.conj().T @ Z, np.eye(b), atol=50 * U64)


def test_svqb_threshold_keeps_a_zero_column_finite():
    rng = np.random.default_rng(52)
    W = rng.standard_normal((100, 4))
    W[:, 2] = 0.0
    Q = oracle.svqb(W)
    assert np.isfinite(Q).all()
    assert np.allclose(Q[:, np.linalg.norm(Q, axis=0) > 0.5].T @ Q[:, np.linalg.norm(Q, axis=0) > 0.5], np.eye(3),
                       atol=1e-12)


def _spread_bottom():
    rng = np.random.default_rng(5)
    n = 60
    sigma = np.concatenate([np.logspace(0, -3, n - 4), [1e-5, 3e-6, 1e-6, 2e-7]])
    return wl.planted(rng, 5000, sigma)


@pytest.mark.parametrize("orth_mode", ["householder", "svqb"])
def test_locking_deflates_converged_columns(orth_mode):
    """Locking (Sec. 2.3): converged columns keep their values while the rest iterate in the
    orthogonal complement; the result is the planted bottom triplets (within the backward-stable
    floors of Sec. 4), V stays orthonormal across locked and active columns, the iteration ends
    once every column is locked, and it spends fewer matrix-vector products (b per iteration
    without locking, the active count with it)."""
    A, s, V = _spread_bottom()
    k = 4
    r0 = oracle.rlobpcg(A, k=k, seed=3, orth_mode=orth_mode)
    r1 = oracle.rlobpcg(A, k=k, seed=3, orth_mode=orth_mode, locking=True, keep_iterates=True)
    truth = np.sort(s)[:k]
    floor = 10 * np.sqrt(A.shape[1]) * U64 * s[0]
    assert np.all(np.abs(r1["sigma"] - truth) <= np.maximum(1e-10 * truth, floor))
    assert np.all(np.abs(r0["sigma"] - truth) <= np.maximum(1e-10 * truth, floor))
    assert r1["locked"].all() and r1["stop_reason"] == "converged"
    assert r1["matvecs"] < r0["matvecs"]
    for Vi in r1["iterates"]:
        assert np.linalg.norm(Vi.conj().T @ Vi - np.eye(k), 2) <= 1e3 * A.shape[1] * U64
    # the locked residuals met the tolerance of Sec. 2.1 when they locked, and stay frozen
    tau = oracle.default_tau(A.shape[1])
    assert np.all(r1["resid"] <= r1["sigma11"] ** 2 * tau)


def test_locking_ends_a_fixed_iteration_solve_once_every_column_locked():
    """Sec. 2.3: with every column locked nothing is left to iterate on; a tolerance that the
    first iteration already meets ends a fixed-iteration solve after one iteration, with b + b
    matrix-vector products and the same triplets as the plain method's first iteration."""
    A, s, V = _spread_bottom()
    r = oracle.rlobpcg(A, k=2, b=3, seed=3, fixed_iters=8, tau=1e-2, locking=True)
    p = oracle.rlobpcg(A, k=2, b=3, seed=3, fixed_iters=1, tau=1e-2)
    assert r["iters"] == 1 and r["locked"].all() and r["matvecs"] == 6
    assert np.array_equal(r["sigma"], p["sigma"])


def test_locking_off_is_the_plain_method():
    A, s, V = _spread_bottom()
    a = oracle.rlobpcg(A, k=2, seed=3, fixed_iters=6)
    b = oracle.rlobpcg(A, k=2, seed=3, fixed_iters=6, locking=False, orth_mode="householder")
    assert np.array_equal(a["sigma"], b["sigma"]) and a["matvecs"] == 2 * 7


# ---------------------------------------------------------------------------------------------
# Preconditioner variants of Sec. 1.1 (diagonal, none) beside the randomized one
# ---------------------------------------------------------------------------------------------

def _small_planted(seed, m=3000, n=30, V=None, sigma=None):
    rng = np.random.default_rng(seed)
    sigma = np.concatenate([np.geomspace(1.0, 1e-3, n - 1), [1e-6]]) if sigma is None else sigma
    return wl.planted(rng, m, sigma, V=V)


def test_no_preconditioner_is_rotation_covariant():
    """LOBPCG without a preconditioner (P = I) and the sketch-and-solve start are covariant under
    A -> A Q for an orthogonal Q (S A Q = (S A) Q), so the Ritz values of every iteration are the
    same for A and A Q; a diagonal P is not (it depends on the columns' basis)."""
    A, s, V = _small_planted(61)
    Q = wl.haar_orthonormal(np.random.default_rng(62), A.shape[1], A.shape[1])
    r1 = oracle.rlobpcg(A, k=2, seed=5, fixed_iters=5, precond="none")
    r2 = oracle.rlobpcg(A @ Q, k=2, seed=5, fixed_iters=5, precond="none")
    np.testing.assert_allclose(r2["theta_hist"][1:], r1["theta_hist"][1:], rtol=1e-6)
    d1 = oracle.rlobpcg(A, k=2, seed=5, fixed_iters=5, precond="diag")
    d2 = oracle.rlobpcg(A @ Q, k=2, seed=5, fixed_iters=5, precond="diag")
    assert not np.allclose(d2["theta_hist"][1:], d1["theta_hist"][1:], rtol=1e-3)


def test_diagonal_preconditioner_equals_none_for_equal_column_norms():
    """P = diag(||A(:, i)||^{-1}) is a multiple of I when every column has the same norm; W is then
    a multiple of R, the trial space is the same, and so are the Ritz values."""
    A, s, V = _small_planted(63)
    A = A / np.linalg.norm(A, axis=0)[None, :] * 0.37
    r1 = oracle.rlobpcg(A, k=1, seed=5, fixed_iters=6, precond="none")
    r2 = oracle.rlobpcg(A, k=1, seed=5, fixed_iters=6, precond="diag")
    np.testing.assert_allclose(r2["theta_hist"][1:], r1["theta_hist"][1:], rtol=1e-9)


def test_diagonal_preconditioner_is_exact_for_orthogonal_columns():
    """For A = U diag(sigma) (orthogonal columns, coherent V = I) the diagonal P P^* equals
    (A^* A)^{-1}: each step is an inverse-iteration step, so the diagonally preconditioned method
    is far ahead of the unpreconditioned one after two iterations (Sec. 1.1's easy problem is the
    coherent case where a diagonal preconditioner works)."""
    n = 30
    sigma = np.concatenate([np.geomspace(1.0, 0.1, n - 1), [1e-7]])
    A, s, V = _small_planted(64, n=n, V=np.eye(n), sigma=sigma)
    rd = oracle.rlobpcg(A, k=1, seed=5, fixed_iters=2, precond="diag")
    rn = oracle.rlobpcg(A, k=1, seed=5, fixed_iters=2, precond="none")
    ed = abs(rd["sigma"][0] - 1e-7) / 1e-7
    en = abs(rn["sigma"][0] - 1e-7) / 1e-7
    assert ed < 1e-6 and ed < 1e-3 * en, (ed, en)
