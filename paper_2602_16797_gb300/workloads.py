"""Seeded synthetic test matrices shaped like the paper's workloads.

This module holds no arithmetic of the method itself: it only draws random matrices with
planted singular spectra (A = U diag(sigma) V^H with Haar-distributed singular vectors) and the
other matrix families the paper experiments on. Both the oracle-based tests and the GPU tests /
benchmark draw their inputs from here, so the two sides always see identical matrices.

Families (section / paragraph of arXiv 2602.16797 they follow):
  * planted spectra with Haar U, V                 -- Sec. 1.1 "hard" problem, Sec. 4.1
  * the "easy" problem with coherent V             -- Sec. 1.1
  * gap sweep (sigma_{n-1} set by gap)             -- Sec. 4.1.1
  * condition-number sweep                         -- Sec. 4.1.2
  * clustered spectrum for block tests             -- Sec. 4.2
  * exact nullspace A = B C                        -- problem statement (nullspace of a tall matrix)
  * Loewner matrices of f(x) = exp(x)/(1+25x^2)    -- Sec. 5 (AAA-Lawson needs Loewner-type matrices)

Seeds follow one convention: a generator gets an explicit integer seed and builds its own
``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import numpy as np

# Seeds of the named workloads: workload k uses 1000 + k; serving request r uses 50000 + r.
SEED_BASE = 1000
SERVE_SEED_BASE = 50000


def _gaussian(rng, shape, complex_=False):
    if complex_:
        return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    return rng.standard_normal(shape)


def haar_orthonormal(rng, rows: int, cols: int, complex_: bool = False) -> np.ndarray:
    """rows x cols matrix with orthonormal columns drawn from the Haar measure.

    QR of a Gaussian matrix with the phases of diag(R) folded back into Q (Mezzadri, "How to
    generate random matrices from the classical compact groups", Notices AMS 2007).
    """
    G = _gaussian(rng, (rows, cols), complex_)
    Q, R = np.linalg.qr(G)
    d = np.diagonal(R).copy()
    d[d == 0] = 1.0
    return Q * (d / np.abs(d))[None, :]


def planted(rng, m: int, sigma: np.ndarray, complex_: bool = False, V: np.ndarray | None = None):
    """A = U diag(sigma) V^H with Haar U (m x n) and Haar V (n x n) unless V is given.

    Returns (A, sigma_sorted_descending, V) so that callers know the exact singular triplets.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    n = sigma.size
    U = haar_orthonormal(rng, m, n, complex_)
    if V is None:
        V = haar_orthonormal(rng, n, n, complex_)
    A = (U * sigma[None, :]) @ V.conj().T
    order = np.argsort(-sigma, kind="stable")
    return np.ascontiguousarray(A), sigma[order], V[:, order]


# ---------------------------------------------------------------------------------------------
# Named workloads (sizes of the configurations this library is benchmarked on)
# ---------------------------------------------------------------------------------------------

def planted_small_gap_free(seed: int = SEED_BASE + 1, m: int = 4000, n: int = 50):
    """m=4000, n=50: sigma_1..sigma_49 logspaced 1 -> 1e-6 and sigma_50 = 1e-10 (FP64 real)."""
    rng = np.random.default_rng(seed)
    sigma = np.concatenate([np.logspace(0, -6, n - 1), [1e-10]])
    return planted(rng, m, sigma)


def exact_nullspace(seed: int = SEED_BASE + 2, m: int = 100_000, n: int = 500, rank: int = 495):
    """A = B C with B (m x rank), C (rank x n) N(0,1): an exact nullspace of dimension n - rank.

    Returns (A, C); the nullspace of A is the nullspace of C (B has full column rank a.s.).
    """
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((m, rank))
    C = rng.standard_normal((rank, n))
    return np.ascontiguousarray(B @ C), C


def planted_bottom_cluster(seed: int = SEED_BASE + 2, m: int = 100_000, n: int = 500, k: int = 5,
                           top_low: float = 1e-4, bottom_hi: float = 1e-9, bottom_lo: float = 1e-12):
    """sigma_1..sigma_{n-k} logspaced 1 -> top_low; the k smallest logspaced bottom_hi -> bottom_lo."""
    rng = np.random.default_rng(seed + 100)
    sigma = np.concatenate([np.logspace(0, np.log10(top_low), n - k),
                            np.logspace(np.log10(bottom_hi), np.log10(bottom_lo), k)])
    return planted(rng, m, sigma)


def planted_complex(seed: int = SEED_BASE + 3, m: int = 200_000, n: int = 300):
    """complex128: sigma logspaced 1 -> 1e-8 with the three smallest set to 1e-12, 3e-13, 1e-13."""
    rng = np.random.default_rng(seed)
    sigma = np.logspace(0, -8, n)
    sigma[-3:] = [1e-12, 3e-13, 1e-13]
    return planted(rng, m, sigma, complex_=True)


def planted_large(seed: int = SEED_BASE + 4, m: int = 1_000_000, n: int = 1000, k: int = 10):
    """sigma_1..sigma_{n-k} logspaced 1 -> 1e-4, sigma_{n-k+1}..sigma_n logspaced 1e-9 -> 1e-10."""
    rng = np.random.default_rng(seed)
    sigma = np.concatenate([np.logspace(0, -4, n - k), np.logspace(-9, -10, k)])
    return planted(rng, m, sigma)


# ---------------------------------------------------------------------------------------------
# The paper's own experiment families (Sec. 1.1, 4.1, 4.2)
# ---------------------------------------------------------------------------------------------

def gap_sweep(seed: int, gap: float, m: int = 10_000, n: int = 100):
    """Sec. 4.1.1: sigma_1..sigma_{n-2} geometric 1 -> 1e-9, sigma_n = 1e-10, and sigma_{n-1}
    chosen so that (sigma_{n-1}^2 - sigma_n^2) / sigma_n^2 = gap."""
    rng = np.random.default_rng(seed)
    s_n = 1e-10
    sigma = np.concatenate([np.geomspace(1.0, 1e-9, n - 2), [s_n * np.sqrt(1.0 + gap), s_n]])
    return planted(rng, m, sigma)


def condition_sweep(seed: int, kappa: float, m: int = 10_000, n: int = 100):
    """Sec. 4.1.2: sigma_2..sigma_n geometric 1e-8 -> 1e-10 and sigma_1 = kappa * sigma_n."""
    rng = np.random.default_rng(seed)
    tail = np.geomspace(1e-8, 1e-10, n - 1)
    sigma = np.concatenate([[kappa * tail[-1]], tail])
    return planted(rng, m, sigma)


def clustered_sigma(n: int, a: float = 1.0 / 256.0) -> np.ndarray:
    """Sec. 4.2: sigma_i = exp(-log(1e10) ((i-1)/(n-1))^a), i = 1..n (clustered near the bottom)."""
    i = np.arange(1, n + 1)
    return np.exp(-np.log(1e10) * ((i - 1) / (n - 1)) ** a)


def clustered(seed: int, m: int, n: int, a: float = 1.0 / 256.0):
    """Sec. 4.2 block-test matrix: Haar U, V and the clustered spectrum of clustered_sigma."""
    rng = np.random.default_rng(seed)
    return planted(rng, m, clustered_sigma(n, a))


def clustered_large_device(seed: int = SEED_BASE + 6, m: int = 1_000_000, n: int = 2000, device="cuda"):
    """The 1e6 x 2000 clustered block-test matrix of Sec. 4.2 (16 GB FP64), built on the GPU."""
    return planted_on_device(seed, m, clustered_sigma(n), device=device)


def easy_coherent(seed: int, m: int, n: int):
    """Sec. 1.1 "easy": V = orth(diag(randn(n)) + 1e-4 randn(n)), Haar U, sigma_1..sigma_{n-1}
    geometric 1 -> 0.1 and sigma_n = 1e-7."""
    rng = np.random.default_rng(seed)
    M = np.diag(rng.standard_normal(n)) + 1e-4 * rng.standard_normal((n, n))
    V, _ = np.linalg.qr(M)
    sigma = np.concatenate([np.geomspace(1.0, 0.1, n - 1), [1e-7]])
    return planted(rng, m, sigma, V=V)


def loewner(seed: int, m: int, n: int):
    """Loewner matrix L_ij = (f(x_i) - f(z_j)) / (x_i - z_j) with f(x) = exp(x) / (1 + 25 x^2),
    z_j Chebyshev points of the second kind cos(pi j / (n-1)) and x_i uniform on [-1, 1], redrawn
    when closer than 1e-12 to any z_j."""
    rng = np.random.default_rng(seed)
    z = np.cos(np.pi * np.arange(n) / (n - 1))
    x = rng.uniform(-1.0, 1.0, m)
    for _ in range(100):
        bad = np.min(np.abs(x[:, None] - z[None, :]), axis=1) < 1e-12
        if not bad.any():
            break
        x[bad] = rng.uniform(-1.0, 1.0, int(bad.sum()))
    f = lambda t: np.exp(t) / (1.0 + 25.0 * t * t)  # noqa: E731
    L = (f(x)[:, None] - f(z)[None, :]) / (x[:, None] - z[None, :])
    return np.ascontiguousarray(L)


def serve_request(r: int):
    """Request r of the serving stream: half Loewner, half planted; m log-uniform in [2e3, 5e5],
    n uniform in [20, 400], k in {1, 2, 4}. Returns (A, k, kind)."""
    rng = np.random.default_rng(SERVE_SEED_BASE + r)
    m = int(round(np.exp(rng.uniform(np.log(2e3), np.log(5e5)))))
    n = int(rng.integers(20, 401))
    k = int(rng.choice([1, 2, 4]))
    m = max(m, 4 * n)
    if r % 2 == 0:
        return loewner(SERVE_SEED_BASE + r, m, n), k, "loewner"
    sigma = np.concatenate([np.logspace(0, -6, n - k), np.logspace(-9, -10, k)])
    A, _, _ = planted(rng, m, sigma)
    return A, k, "planted"


def serve_shape(r: int):
    """(m, n, k, kind) of request r of the serving stream (the draws of serve_request)."""
    rng = np.random.default_rng(SERVE_SEED_BASE + r)
    m = int(round(np.exp(rng.uniform(np.log(2e3), np.log(5e5)))))
    n = int(rng.integers(20, 401))
    k = int(rng.choice([1, 2, 4]))
    return max(m, 4 * n), n, k, ("loewner" if r % 2 == 0 else "planted")


def loewner_on_device(seed: int, m: int, n: int, device="cuda"):
    """The Loewner matrix of `loewner` built with torch on a GPU (x_i drawn on the host with the same
    seeded generator, so the matrix equals loewner(seed, m, n) up to rounding of f)."""
    import torch
    rng = np.random.default_rng(seed)
    z = np.cos(np.pi * np.arange(n) / (n - 1))
    x = rng.uniform(-1.0, 1.0, m)
    for _ in range(100):
        bad = np.min(np.abs(x[:, None] - z[None, :]), axis=1) < 1e-12
        if not bad.any():
            break
        x[bad] = rng.uniform(-1.0, 1.0, int(bad.sum()))
    xd = torch.from_numpy(x).to(device)
    zd = torch.from_numpy(z).to(device)
    f = lambda t: torch.exp(t) / (1.0 + 25.0 * t * t)  # noqa: E731
    return ((f(xd)[:, None] - f(zd)[None, :]) / (xd[:, None] - zd[None, :])).contiguous()


def serve_pool(size: int, device="cuda"):
    """A pool of `size` matrices with the serving stream's shapes (entry j has request j's m, n, k
    and kind), built on a GPU and held in pinned host memory. The serving benchmark draws its
    requests from this pool, each request with its own sketch seed: the stream keeps the shape
    distribution (m log-uniform in [2e3, 5e5], n uniform in [20, 400], k in {1, 2, 4}, half
    Loewner, half planted) while the host holds `size` matrices instead of one per request.
    Returns a list of (A host tensor, k, kind)."""
    import torch
    out = []
    for j in range(size):
        m, n, k, kind = serve_shape(j)
        if kind == "loewner":
            Ad = loewner_on_device(SERVE_SEED_BASE + j, m, n, device)
        else:
            sigma = np.concatenate([np.logspace(0, -6, n - k), np.logspace(-9, -10, k)])
            Ad = planted_on_device(SERVE_SEED_BASE + j, m, sigma, device)[0]
        Ah = torch.empty(Ad.shape, dtype=Ad.dtype, pin_memory=True)
        Ah.copy_(Ad)
        del Ad
        out.append((Ah, k, kind))
    torch.cuda.synchronize()
    return out


def fig1_device(m: int = 2_000_000, n: int = 4000, seed: int = SEED_BASE + 7, device="cuda", kinds=("easy", "hard")):
    """Sec. 1.1's two m x n problems A = U diag(sigma) V^T, built on a GPU one at a time (a
    generator: each A is dropped before the next is made, and U is dropped before A is handed
    out, so that a solve has the rest of the device). Both use the same Haar U (Q of a seeded
    Gaussian, phases of diag(R) folded back; rebuilt for each problem from the same seed).
      easy: V = orth(diag(randn(n)) + 1e-4 randn(n)) (coherent), sigma_1..sigma_{n-1} geometric
            1 -> 0.1, sigma_n = 1e-7;
      hard: Haar V, sigma geometric 1 -> 1e-10.
    Yields (kind, A on the device, sigma sorted descending)."""
    import torch
    for kind in kinds:
        gen = torch.Generator(device=device).manual_seed(int(seed))
        G = torch.randn((m, n), generator=gen, device=device, dtype=torch.float64)
        U, R = torch.linalg.qr(G)
        del G
        d = torch.diagonal(R)
        U *= torch.where(d.abs() > 0, torch.sign(d), torch.ones_like(d))[None, :]
        del R, d
        rng = np.random.default_rng(seed + (1 if kind == "easy" else 2))
        if kind == "easy":
            M = np.diag(rng.standard_normal(n)) + 1e-4 * rng.standard_normal((n, n))
            V, _ = np.linalg.qr(M)
            sigma = np.concatenate([np.geomspace(1.0, 0.1, n - 1), [1e-7]])
        else:
            V = haar_orthonormal(rng, n, n)
            sigma = np.geomspace(1.0, 1e-10, n)
        Vt = torch.from_numpy(np.ascontiguousarray((V * sigma[None, :]).T)).to(device)   # diag(sigma) V^T
        A = torch.empty((m, n), dtype=torch.float64, device=device)
        step = 1 << 17
        for r0 in range(0, m, step):
            torch.matmul(U[r0:r0 + step], Vt, out=A[r0:r0 + step])
        del Vt, U
        torch.cuda.empty_cache()
        yield kind, A, np.sort(sigma)[::-1]
        del A


def planted_on_device(seed: int, m: int, sigma: np.ndarray, device="cuda", complex_: bool = False):
    """A = U diag(sigma) V^H built on a GPU with torch (for sizes where a host QR of the m x n
    Gaussian takes minutes, e.g. 1e6 x 1000). U: Q of a seeded Gaussian (Philox stream of
    torch.Generator(device).manual_seed(seed)) with the phases of diag(R) folded back; V: Haar
    from numpy on the host. Returns (A on the device, sigma sorted descending, V as numpy)."""
    import torch
    sigma = np.asarray(sigma, dtype=np.float64)
    n = sigma.size
    rng = np.random.default_rng(seed)
    V = haar_orthonormal(rng, n, n, complex_)
    gen = torch.Generator(device=device).manual_seed(int(seed))
    dt = torch.complex128 if complex_ else torch.float64
    G = torch.randn((m, n), generator=gen, device=device, dtype=dt)
    Q, R = torch.linalg.qr(G)
    del G
    d = torch.diagonal(R)
    ph = torch.where(d.abs() > 0, d / d.abs(), torch.ones_like(d))
    Q *= ph[None, :]
    del R
    Vd = torch.from_numpy(np.ascontiguousarray(V)).to(device)
    Q *= torch.from_numpy(sigma).to(device=device, dtype=Q.real.dtype)[None, :].to(dt)
    A = Q @ Vd.conj().T
    del Q
    order = np.argsort(-sigma, kind="stable")
    return A.contiguous(), sigma[order], V[:, order]


def planted_large_device(seed: int = SEED_BASE + 4, m: int = 1_000_000, n: int = 1000, k: int = 10, device="cuda"):
    """The 1e6 x 1000 planted workload (sigma_1..990 logspace(0,-4), sigma_991..1000 logspace(-9,-10))
    generated on the device."""
    sigma = np.concatenate([np.logspace(0, -4, n - k), np.logspace(-9, -10, k)])
    return planted_on_device(seed, m, sigma, device=device)
