"""Parity of each GPU step with the CPU oracle, through the C ABI.

sketch: bit for bit (same SplitMix64 stream, same summation order).
gram:   A W and A^H (A W) within the standard dot-product error bounds.
tsqr:   the R factor of a tall block against LAPACK's Householder R.
factor: R, Sigma~, V~ and R^{-1} of the sketch against LAPACK.
"""
import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _dtype_code(A):
    return rl.RLOBPCG_C128 if np.iscomplexobj(A) else rl.RLOBPCG_F64


def _rand(rng, shape, cplx):
    x = rng.standard_normal(shape)
    if cplx:
        x = x + 1j * rng.standard_normal(shape)
    return x


# ------------------------------------------------------------------------------------------- sketch

def gpu_sketch(A, d, zeta, seed, prec):
    m, n = A.shape
    cplx = np.iscomplexobj(A)
    tdt = {(False, "f64"): torch.float64, (False, "f32"): torch.float32,
           (True, "f64"): torch.complex128, (True, "f32"): torch.complex64}[(cplx, prec)]
    Ad = _dev(A)
    SA = torch.empty((n, d), dtype=tdt, device="cuda")      # column-major d x n == row-major n x d
    rl.rlobpcg_sketch(Ad.data_ptr(), m, n, n, _dtype_code(A), d, zeta, seed,
                      rl.RLOBPCG_SKETCH_F32 if prec == "f32" else rl.RLOBPCG_SKETCH_F64, SA.data_ptr(), _stream())
    torch.cuda.synchronize()
    return SA.cpu().numpy().T


@pytest.mark.parametrize("m,n,d,zeta", [(1, 1, 8, 8), (200, 7, 24, 3), (4000, 50, 200, 8), (1537, 33, 1500, 8),
                                        (3001, 70, 280, 4), (10007, 120, 360, 8)])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_sketch_bit_exact(m, n, d, zeta, cplx, prec):
    rng = np.random.default_rng(m + n)
    A = _rand(rng, (m, n), cplx) * np.exp(rng.uniform(-5, 5, (m, 1)))
    got = gpu_sketch(A, d, zeta, 12345, prec)
    want = oracle.sketch(A, d, zeta, 12345, precision=prec)
    assert got.dtype == want.dtype
    assert np.array_equal(got, want), np.max(np.abs(got - want))


def test_sketch_strided_lda():
    rng = np.random.default_rng(3)
    m, n, lda, d, zeta = 999, 20, 27, 80, 8
    Abig = rng.standard_normal((m, lda))
    Ad = _dev(Abig)
    SA = torch.empty((n, d), dtype=torch.float64, device="cuda")
    rl.rlobpcg_sketch(Ad.data_ptr(), m, n, lda, rl.RLOBPCG_F64, d, zeta, 77, rl.RLOBPCG_SKETCH_F64, SA.data_ptr(),
                      _stream())
    torch.cuda.synchronize()
    assert np.array_equal(SA.cpu().numpy().T, oracle.sketch(Abig[:, :n], d, zeta, 77))


# --------------------------------------------------------------------------------------------- gram

def gpu_gram(A, W):
    m, n = A.shape
    b = W.shape[1]
    dt = _dtype_code(A)
    Ad, Wd = _dev(A), _dev(W)
    AW = torch.empty((m, b), dtype=Ad.dtype, device="cuda")
    G = torch.empty((n, b), dtype=Ad.dtype, device="cuda")
    ws = rl.rlobpcg_gram_workspace_size(m, n, b, dt)
    work = torch.empty(max(ws, 16), dtype=torch.uint8, device="cuda")
    rl.rlobpcg_gram(Ad.data_ptr(), m, n, n, dt, Wd.data_ptr(), b, b, AW.data_ptr(), b, G.data_ptr(), b,
                    work.data_ptr(), ws, _stream())
    torch.cuda.synchronize()
    return AW.cpu().numpy(), G.cpu().numpy()


def gram_bounds(A, W, AW):
    """Componentwise bounds: |fl(A W) - A W| <= g_n |A||W|, and the error of A^H (A W) from both the
    rounding of A W and the second product (complex products carry a factor of about 2)."""
    m, n = A.shape
    f = 4.0 if np.iscomplexobj(A) else 1.0
    absA = np.abs(A)
    b1 = f * (n + 2) * U * (absA @ np.abs(W))
    b2 = absA.T @ b1 + f * (m + 2) * U * (absA.T @ np.abs(AW))
    return b1, b2


@pytest.mark.parametrize("m,n,b", [(1, 8, 1), (1000, 50, 1), (4097, 64, 5), (20011, 100, 10), (3000, 333, 3),
                                   (777, 31, 2), (50000, 500, 5), (5000, 1000, 10), (2048, 16, 16)])
@pytest.mark.parametrize("cplx", [False, True])
def test_gram_parity(m, n, b, cplx):
    rng = np.random.default_rng(m * 7 + n)
    A = _rand(rng, (m, n), cplx)
    W = _rand(rng, (n, b), cplx)
    AW, G = gpu_gram(A, W)
    AW0, G0 = oracle.gram_pass(A, W)
    b1, b2 = gram_bounds(A, W, AW0)
    assert np.all(np.abs(AW - AW0) <= b1 + 1e-300)
    assert np.all(np.abs(G - G0) <= b2 + 1e-300)


def test_gram_deterministic():
    rng = np.random.default_rng(9)
    A = rng.standard_normal((30011, 200))
    W = rng.standard_normal((200, 4))
    r1 = gpu_gram(A, W)
    r2 = gpu_gram(A, W)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])


def test_gram_planted_small_singular_directions():
    """Directions with A w ~ sigma_min: A^H (A w) stays accurate relative to |A|^H |A w| (the
    quantity the residual of the smallest triplets depends on)."""
    A, s, V = wl.planted_small_gap_free(m=4000, n=50)
    W = V[:, -3:]
    AW, G = gpu_gram(A, W)
    AW0, G0 = oracle.gram_pass(A, W)
    b1, b2 = gram_bounds(A, W, AW0)
    assert np.all(np.abs(AW - AW0) <= b1) and np.all(np.abs(G - G0) <= b2)


# --------------------------------------------------------------------------------------------- tsqr

def gpu_tsqr(X):
    m, c = X.shape
    dt = _dtype_code(X)
    Xd = _dev(X)
    R = torch.empty((c, c), dtype=Xd.dtype, device="cuda")
    ws = rl.rlobpcg_tsqr_workspace_size(m, c, dt)
    work = torch.empty(max(ws, 16), dtype=torch.uint8, device="cuda")
    rl.rlobpcg_tsqr(Xd.data_ptr(), m, c, c, dt, R.data_ptr(), work.data_ptr(), ws, _stream())
    torch.cuda.synchronize()
    return R.cpu().numpy()


@pytest.mark.parametrize("m,c", [(5, 3), (1000, 1), (4000, 3), (30000, 15), (100003, 30), (2000, 64), (257, 30)])
@pytest.mark.parametrize("cplx", [False, True])
def test_tsqr_parity(m, c, cplx):
    rng = np.random.default_rng(m + c)
    X = _rand(rng, (m, c), cplx) * np.logspace(0, -10, c)[None, :]
    R = gpu_tsqr(X)
    R0 = oracle.householder_r(X)
    assert np.allclose(np.tril(R, -1), 0)
    assert np.all(np.real(np.diag(R)) >= 0) and np.allclose(np.imag(np.diag(R)), 0)
    # backward-stable QR: R^H R = X^H X to u ||X||^2, and each row agrees with LAPACK's to
    # u ||X|| / (size of the trailing block)
    nX = np.linalg.norm(X, 2)
    assert np.allclose(R.conj().T @ R, X.conj().T @ X, rtol=0, atol=50 * c * U * nX ** 2)
    # singular values (the only thing Rayleigh-Ritz uses besides the right vectors)
    s, s0 = np.linalg.svd(R, compute_uv=False), np.linalg.svd(R0, compute_uv=False)
    assert np.all(np.abs(s - s0) <= 100 * c * U * nX)


# ------------------------------------------------------------------------------------------- factor

def gpu_factor(SA, prec):
    d, n = SA.shape
    cplx = np.iscomplexobj(SA)
    dt = rl.RLOBPCG_C128 if cplx else rl.RLOBPCG_F64
    sp = {"f32": rl.RLOBPCG_SKETCH_F32, "f64": rl.RLOBPCG_SKETCH_F64,
          "f32_refine": rl.RLOBPCG_SKETCH_F32_REFINE}[prec]
    low = prec == "f32"
    tdt = {(False, False): torch.float64, (False, True): torch.float32,
           (True, False): torch.complex128, (True, True): torch.complex64}[(cplx, low)]
    SAd = torch.from_numpy(np.ascontiguousarray(SA.T)).to(tdt).cuda()   # column-major d x n
    R = torch.empty((n, n), dtype=tdt, device="cuda")
    Vt = torch.empty((n, n), dtype=tdt, device="cuda")
    Rinv = torch.empty((n, n), dtype=tdt, device="cuda")
    sig = torch.empty(n, dtype=torch.float64, device="cuda")
    ws = rl.rlobpcg_factor_workspace_size(d, n, dt, sp)
    work = torch.empty(ws, dtype=torch.uint8, device="cuda")
    rl.rlobpcg_factor(SAd.data_ptr(), d, n, dt, sp, R.data_ptr(), sig.data_ptr(), Vt.data_ptr(), Rinv.data_ptr(),
                      work.data_ptr(), ws, _stream())
    torch.cuda.synchronize()
    # R and Vt are column-major: the row-major n x n tensors hold their transposes
    return R.cpu().numpy().T, sig.cpu().numpy(), Vt.cpu().numpy().T, Rinv.cpu().numpy()


def _sub_sin(V1, V2):
    Q1, _ = np.linalg.qr(V1)
    Q2, _ = np.linalg.qr(V2)
    return np.linalg.norm(Q1 - Q2 @ (Q2.conj().T @ Q1), 2)


# (1900, 700): more columns than resident CTAs, so CTAs own several; (2500, 300): 16 rows per
# thread; (4500, 120): taller than the register-resident QR, the grid-barrier kernel
@pytest.mark.parametrize("d,n", [(200, 50), (37, 36), (1500, 500), (400, 101), (1900, 700), (2500, 300),
                                 (4500, 120), (1, 1), (257, 257)])
@pytest.mark.parametrize("cplx", [False, True])
def test_factor_parity_f64(d, n, cplx):
    rng = np.random.default_rng(d + n)
    SA = _rand(rng, (d, n), cplx) @ np.diag(np.logspace(0, -8, n))
    R, sig, Vt, Rinv = gpu_factor(SA, "f64")
    R0 = oracle.householder_r(SA)
    ph = np.diag(R) / np.abs(np.diag(R))
    Rn = R * ph.conj()[:, None]
    s0, V0 = oracle.sketch_svd(SA)
    assert np.allclose(np.tril(R, -1), 0)
    assert np.allclose(Rn.conj().T @ Rn, SA.conj().T @ SA, rtol=0, atol=100 * n * U * s0[0] ** 2)
    assert np.allclose(Rn, R0, rtol=0, atol=1e3 * n * U * s0[0] * (s0[0] / s0[-1]))
    # singular values with high relative accuracy where the spectrum allows, absolute otherwise
    assert np.all(np.abs(sig - s0) <= 50 * n * U * s0[0])
    assert np.all(np.diff(sig) <= 0)
    # the bottom 3 right singular vectors (the start block) span the same subspace
    if n >= 4:
        gap = (s0[-4] - s0[-3]) / s0[0]
        assert _sub_sin(Vt[:, -3:], V0[:, -3:]) <= max(1e-10, 1e3 * n * U / gap)
    assert np.allclose(Vt.conj().T @ Vt, np.eye(n), atol=1e3 * n * U)
    # R^{-1} R = I to kappa u
    kappa = s0[0] / s0[-1]
    assert np.allclose(Rinv @ R, np.eye(n), atol=1e2 * n * U * kappa)


@pytest.mark.parametrize("cplx", [False, True])
def test_factor_rank_deficient_sketch(cplx):
    # exact zero columns keep tau = 0 and R(j, j) = 0 exactly; a repeated column gives a diagonal
    # entry at rounding level; R^H R = SA^H SA still holds to rounding
    rng = np.random.default_rng(11)
    d, n = 900, 300
    SA = _rand(rng, (d, n), cplx)
    SA[:, 5:9] = 0
    SA[:, 40] = SA[:, 3]
    R, sig, Vt, Rinv = gpu_factor(SA, "f64")
    s0 = np.linalg.svd(SA, compute_uv=False)
    assert np.all(np.tril(R, -1) == 0)
    assert np.all(R[5:9, 5:9] == 0) and np.all(R[:, 5:9] == 0)
    assert abs(R[40, 40]) <= 1e2 * n * U * s0[0]
    assert np.allclose(R.conj().T @ R, SA.conj().T @ SA, rtol=0, atol=100 * n * U * s0[0] ** 2)
    assert np.all(np.abs(sig - s0) <= 50 * n * U * s0[0])


@pytest.mark.parametrize("cplx", [False, True])
def test_factor_f32_graded_columns(cplx):
    """FP32 factor of a sketch whose columns fall to 1e-13 of the largest: every output finite
    (the complex reflector scalar is formed without squaring a product of two small numbers), and
    R^H R = SA^H SA to FP32 rounding of the column scales."""
    rng = np.random.default_rng(9)
    d, n = 1200, 300
    SA = (_rand(rng, (d, n), cplx) @ np.diag(np.logspace(0, -13, n))).astype(np.complex64 if cplx else np.float32)
    R, sig, Vt, Rinv = gpu_factor(SA, "f32")
    assert np.isfinite(R).all() and np.isfinite(sig).all() and np.isfinite(Rinv).all()
    SA64 = SA.astype(np.complex128 if cplx else np.float64)
    R64 = R.astype(SA64.dtype)
    G = SA64.conj().T @ SA64
    assert np.linalg.norm(R64.conj().T @ R64 - G, 2) <= 50 * n * 2.0 ** -24 * np.linalg.norm(G, 2)


@pytest.mark.parametrize("cplx", [False, True])
def test_factor_f32_sketch(cplx):
    rng = np.random.default_rng(5)
    d, n = 400, 100
    SA = (_rand(rng, (d, n), cplx) @ np.diag(np.logspace(0, -4, n))).astype(np.complex64 if cplx else np.float32)
    R, sig, Vt, Rinv = gpu_factor(SA, "f32")
    s0, V0 = oracle.sketch_svd(SA)
    u32 = 2.0 ** -24
    assert np.all(np.abs(sig - s0) <= 50 * n * u32 * s0[0])
    assert np.allclose(Vt.conj().T @ Vt, np.eye(n), atol=1e2 * n * u32)
    assert np.allclose(Rinv.astype(np.complex128 if cplx else np.float64) @ R, np.eye(n),
                       atol=1e2 * n * u32 * s0[0] / s0[-1])


@pytest.mark.parametrize("d,n,kappa", [(400, 100, 1e10), (1200, 300, 1e13), (4000, 1000, 1e10), (37, 36, 1e6),
                                       (257, 130, 1e12)])
@pytest.mark.parametrize("cplx", [False, True])
def test_factor_refined_parity(d, n, kappa, cplx):
    """FP32 QR of the FP64 sketch corrected once in FP64 (RLOBPCG_SKETCH_F32_REFINE): R^H R equals
    SA^H SA to FP64 rounding and the shift (where the FP32 factor alone is off by u_32 ||SA||^2),
    sigma~ matches the FP64 SVD of SA, and R^{-1} R = I; both the oracle's refined factor and the
    GPU's are QR factors of the same SA. Sizes span several Cholesky panels and ragged tiles."""
    rng = np.random.default_rng(d + n)
    SA = _rand(rng, (d, n), cplx) @ np.diag(np.logspace(0, -np.log10(kappa), n))
    R, sig, Vt, Rinv = gpu_factor(SA, "f32_refine")
    G = SA.conj().T @ SA
    s0, V0 = oracle.sketch_svd(SA)
    nrm = s0[0] ** 2
    assert np.allclose(np.tril(R, -1), 0)
    assert np.linalg.norm(R.conj().T @ R - G, 2) <= 100 * n * U * nrm
    Ro = oracle.refined_factor(SA)
    assert np.linalg.norm(Ro.conj().T @ Ro - G, 2) <= 100 * n * U * nrm
    assert np.all(np.abs(sig - s0) <= 50 * n * U * s0[0])
    assert np.all(np.diff(sig) <= 0)
    assert np.allclose(Rinv @ R, np.eye(n), atol=1e2 * n * U * s0[0] / s0[-1])
