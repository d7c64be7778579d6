"""Plain CPU RLOBPCG in float64 / complex128: the oracle the GPU library is checked against.

TEST INFRASTRUCTURE ONLY: tests/, __graft_entry__.smoke() and bench.py's CPU baseline may import
it; the GPU library shares no code with it and never calls it.

What it computes: the k smallest singular values of a tall A and their right singular vectors,
by the method of Epperly, Park & Nakatsukasa, "Fast, high-accuracy, randomized nullspace
computations for tall matrices" (arXiv 2602.16797): a SparseStack sketch SA (Sec. 2.2) whose SVD
gives the preconditioner P = V~ Sigma~^{-1} (Sec. 2.1) and the sketch-and-solve start block
V~(:, n-b+1:n) (Sec. 3.1); then block LOBPCG on A^H A (Sec. 2.1, 2.3): each iteration forms the
preconditioned residual direction W = P P^* (A^H A V - V Theta^2), makes it orthonormal and
orthogonal to the current block V and momentum block X (two block Gram-Schmidt passes, then a
Householder Orth), and replaces V by the b right singular vectors of A T, T = [V X W], that belong
to its b smallest singular values (Rayleigh-Ritz by energy minimisation: the SVD of A T instead
of an eigenproblem of T^H A^H A T, which would square the small singular values). The momentum
block is the part of the new trial space orthogonal to the new V (Sec. 2.1, the x-defining
equation). Stopping follows Sec. 2.1 (the sketched tolerance on the residual, with the
stagnation checks). Only numpy / LAPACK primitives are used (matmul, SVD, Householder QR); each
quantity is formed the plain way its definition states, with no blocking, fusion or
reordering, so that it can be checked against the paper by eye. Arithmetic is float64
(complex128 for complex A); the optional FP32 sketch rounds A to float32 and sums in float32, as
the mixed-precision form of the method does, and everything after the sketch SVD is float64. The
'f32_refine' sketch precision (an addition of this library, not in the paper) keeps SA in float64,
factors it in float32 and corrects the factor once by a float64 Cholesky QR (refined_factor).

Readings taken where the paper is silent, ambiguous or inconsistent:
  * SparseStack randomness (Sec. 2.2 says "uniformly random"): entry (i, j) -- source row i, piece
    j -- uses h = SplitMix64 output number i*zeta + j of the stream seeded with `seed`
    (Steele, Lea & Flood, OOPSLA 2014); the position inside piece j is floor((h >> 32) len_j / 2^32)
    and the sign is -1 when bit 0 of h is set. S is real (+-zeta^{-1/2}) also for complex A.
  * "equally sized pieces" when zeta does not divide d: piece j = rows [floor(j d/zeta),
    floor((j+1) d/zeta)).
  * SA is accumulated per destination row in ascending source row i and scaled once by
    zeta^{-1/2} at the end.
  * Orth(M) (Alg. 2) is the Q of a thin Householder QR with diag(R) made real non-negative.
  * The sketch-and-solve start V_0 = V~(:, n-b+1:n) is orthonormalised (Orth) before the initial
    Rayleigh-Ritz step, which assumes orthonormal columns (matters only for the FP32 sketch).
  * Iteration 0 has no X (Alg. 2 initialises X_0 = []): T = [V W], C_s is the last b columns of C
    and Q = Orth(C(1:b, 1:b)^H), i.e. "last b" / "first ncol-b" columns in every iteration.
  * Stopping (Sec. 2.1): with stagnation checks on, the test runs when i mod 5 == 0 (Alg. 1) and
    requires max_j ||R(:,j)|| <= Sigma~(1,1)^2 tau AND both stagnation checks for every column;
    the second check divides by the current theta, as the stagnation-check equation does (Alg. 1's
    listing divides by the previous one). History that does not exist yet (r_{i-4}, theta_{i-9},
    and theta_0, which Alg. 1 sets to infinity) is +inf, so comparisons with it are false and the
    earliest stop is i = 10. Without stagnation checks the tolerance alone is tested every
    iteration (Alg. 2).
  * tau defaults to 2 sqrt(n) eps with eps = 2^-52 (MATLAB eps); max_iter to 200 for b = 1
    (Alg. 1) and 100 otherwise (Alg. 2).

Pins (tests/test_oracle_*.py, all CPU): published SplitMix64 vectors; exact properties of S
(one +-1 per piece, unit column norms, uniform positions); SA against a brute-force dense S on
integer data; sketch SVD against R^H R = (SA)^H (SA); the randomized-preconditioning and
sketch-and-solve Facts (Sec. 3.1) with the measured distortion; planted singular triplets and
exact nullspaces; dense-SVD agreement on small matrices; ||A v_j|| = sigma_j and orthonormal V;
the geometric rate of Theorem 1; the stopping rule on hand-worked histories; and planted
mistakes that those checks catch. Loewner-type inputs have sigma_min at noise level, so there
only backward error and orthonormality are pinned (parity unpinned in sigma and V).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64", "piece_bounds", "sparse_stack", "sketch_dense_matrix", "sketch", "sketch_svd",
    "orth", "rayleigh_ritz", "gram_pass", "householder_r", "stop_check", "rlobpcg", "refined_factor", "svqb",
    "projection_set",
    "default_tau", "EPS",
]

EPS = 2.0 ** -52           # MATLAB eps, the eps_mach of the sketched stopping rule (Sec. 2.1)
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB


# ---------------------------------------------------------------------------------------------
# Embedding generation (Sec. 2.2, SparseStack)
# ---------------------------------------------------------------------------------------------

def splitmix64(seed: int, counter) -> np.ndarray:
    """Output number `counter` (0-based) of SplitMix64 seeded with `seed`.

    SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA
    2014): the state after c+1 steps is seed + (c+1) * 0x9E3779B97F4A7C15 (mod 2^64), and the
    output is that state passed through the finaliser z ^= z>>30; z *= 0xBF58476D1CE4E5B9;
    z ^= z>>27; z *= 0x94D049BB133111EB; z ^= z>>31.
    """
    with np.errstate(over="ignore"):
        c = np.asarray(counter, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (c + np.uint64(1)) * np.uint64(GOLDEN_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def piece_bounds(d: int, zeta: int) -> np.ndarray:
    """Row boundaries of the zeta pieces of a SparseStack column: piece j is
    [floor(j d / zeta), floor((j+1) d / zeta))."""
    return np.array([(j * d) // zeta for j in range(zeta + 1)], dtype=np.int64)


def sparse_stack(m: int, d: int, zeta: int, seed: int):
    """Nonzero pattern of the d x m SparseStack S = zeta^{-1/2} [s_1 ... s_m] (Sec. 2.2).

    Column s_i is cut into zeta pieces; each piece holds one entry +-1 at a uniformly random
    position. Returns (dest, sign): dest[i, j] is the row of S holding the nonzero of piece j of
    column i, and sign[i, j] in {+1.0, -1.0} its sign (before the zeta^{-1/2} scaling).
    """
    if d < zeta:
        raise ValueError("SparseStack needs d >= zeta")
    bounds = piece_bounds(d, zeta)
    i = np.arange(m, dtype=np.uint64)[:, None]
    j = np.arange(zeta, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        h = splitmix64(seed, i * np.uint64(zeta) + j)
    lens = (bounds[1:] - bounds[:-1]).astype(np.uint64)
    pos = ((h >> np.uint64(32)) * lens[None, :]) >> np.uint64(32)
    dest = bounds[:-1][None, :] + pos.astype(np.int64)
    sign = np.where((h & np.uint64(1)) == np.uint64(1), -1.0, 1.0)
    return dest, sign


def sketch_dense_matrix(m: int, d: int, zeta: int, seed: int) -> np.ndarray:
    """The d x m SparseStack as a dense float64 matrix (small sizes only; used by the pins)."""
    dest, sign = sparse_stack(m, d, zeta, seed)
    S = np.zeros((d, m))
    for i in range(m):
        for j in range(zeta):
            S[dest[i, j], i] = sign[i, j]
    return S / np.sqrt(zeta)


def _work_dtype(A, precision: str):
    cplx = np.iscomplexobj(A)
    if precision == "f32":
        return np.complex64 if cplx else np.float32
    if precision == "f64":
        return np.complex128 if cplx else np.float64
    raise ValueError(f"unknown sketch precision {precision!r}")


def sketch(A: np.ndarray, d: int, zeta: int, seed: int, precision: str = "f64") -> np.ndarray:
    """SA, the d x n sketch of A (Alg. 2, first two lines).

    Each destination row accumulates +-a_i over its source rows i in ascending order (one
    destination row is fed by one piece only, so the pieces never interleave), then the whole
    sum is scaled once by zeta^{-1/2}. precision='f32' rounds A to float32 and sums in float32.
    """
    m, n = A.shape
    dest, sign = sparse_stack(m, d, zeta, seed)
    work = _work_dtype(A, precision)
    real = np.float32 if precision == "f32" else np.float64
    Aw = np.asarray(A).astype(work)
    acc = np.zeros((d, n), dtype=work)
    for j in range(zeta):
        # ufunc.at applies the updates one index after another, i.e. in ascending i
        np.add.at(acc, dest[:, j], sign[:, j, None].astype(real) * Aw)
    scale = real(1.0 / np.sqrt(float(zeta)))
    return acc * scale


def refined_factor(SA: np.ndarray) -> np.ndarray:
    """R factor of the FP64 sketch SA from an FP32 Householder QR corrected once in FP64 (the
    sketch precision 'f32_refine', an addition of this library; the paper factors in FP64).

    R_32 = R of QR(SA rounded to float32), computed in float32 (LAPACK geqrf); M = R_32^{-1} in
    float64; Y = SA M; H = Y^H Y; s = n u max_i Re H_ii (u = 2^-53); R_c = the upper Cholesky
    factor of H + s I (H + s I = R_c^H R_c); R = R_c R_32. In exact arithmetic, and without the
    shift, R^H R = SA^H SA: R is a QR factor of SA.
    """
    n = SA.shape[1]
    low = np.complex64 if np.iscomplexobj(SA) else np.float32
    R32 = np.linalg.qr(SA.astype(low), mode="r").astype(SA.dtype)
    M = np.linalg.solve(R32, np.eye(n, dtype=SA.dtype))
    Y = SA @ M
    H = Y.conj().T @ Y
    shift = n * 2.0 ** -53 * float(np.max(np.real(np.diagonal(H))))
    Rc = np.linalg.cholesky(H + shift * np.eye(n)).conj().T
    return Rc @ R32


def sketch_svd(SA: np.ndarray):
    """[~, Sigma~, V~] = SVD(SA) (the SVD of the sketch in Alg. 2): Sigma~ descending, V~ (n x n)
    with the right singular vectors as columns. LAPACK gesdd in the precision of SA."""
    _, s, Vh = np.linalg.svd(SA, full_matrices=False)
    return s, Vh.conj().T


# ---------------------------------------------------------------------------------------------
# Pieces of the LOBPCG iteration (Sec. 2.1 and 2.3)
# ---------------------------------------------------------------------------------------------

def orth(M: np.ndarray) -> np.ndarray:
    """Orth(M) (Alg. 2): Q of a thin Householder QR of M, phases of diag(R) moved into Q so that
    diag(R) is real and non-negative."""
    Q, R = np.linalg.qr(M)
    dg = np.diagonal(R)
    ph = np.ones_like(dg)
    nz = np.abs(dg) > 0
    ph[nz] = dg[nz] / np.abs(dg[nz])
    return Q * ph[None, :]


def svqb(W: np.ndarray, tau: float = EPS) -> np.ndarray:
    """SVQB orthonormalisation of the columns of W (Stathopoulos & Wu, "A block orthogonalization
    procedure with constant synchronization requirements", SISC 2002), the faster alternative to
    Orth that Sec. 2.1 names: S = W^H W, D = diag(S)^{-1/2} (zero columns keep D = 0), the
    eigendecomposition D S D = Z Theta Z^H, every eigenvalue below tau max(Theta) raised to it,
    and W D Z Theta^{-1/2}. It spans the columns of W (for full-rank W) with orthonormal columns
    to about u kappa(W D)^2; Theta ascending (LAPACK heevd)."""
    S = W.conj().T @ W
    dg = np.real(np.diagonal(S)).copy()
    D = np.zeros_like(dg)
    D[dg > 0] = 1.0 / np.sqrt(dg[dg > 0])
    M = (S * D[:, None]) * D[None, :]
    theta, Z = np.linalg.eigh(M)
    top = float(np.max(theta)) if theta.size else 0.0
    theta = np.maximum(theta, tau * top) if top > 0 else np.ones_like(theta)
    return ((W * D[None, :]) @ Z) / np.sqrt(theta)[None, :]


def projection_set(V: np.ndarray, X: np.ndarray, act: np.ndarray) -> np.ndarray:
    """The columns W is made orthogonal to (Alg. 2): all of V -- with locking, the converged
    columns too, which keeps the trial space orthogonal to them (Sec. 2.3) -- and X."""
    return np.concatenate([V, X], axis=1)


def rayleigh_ritz(AT: np.ndarray):
    """[~, Theta, C] = SVD(A_T) (Alg. 2, Rayleigh-Ritz by energy minimisation, Sec. 2.1): Theta
    descending, C square with the right singular vectors of A_T as columns."""
    _, theta, Ch = np.linalg.svd(AT, full_matrices=False)
    return theta, Ch.conj().T


def gram_pass(A: np.ndarray, W: np.ndarray):
    """The two products with A one iteration needs: A W and A^H (A W) (Alg. 2)."""
    AW = A @ W
    return AW, A.conj().T @ AW


def householder_r(M: np.ndarray) -> np.ndarray:
    """R of a Householder QR of M (LAPACK geqrf) with rows scaled so diag(R) is real >= 0."""
    R = np.linalg.qr(M, mode="r")
    dg = np.diagonal(R)
    ph = np.ones_like(dg)
    nz = np.abs(dg) > 0
    ph[nz] = dg[nz] / np.abs(dg[nz])
    return R * ph.conj()[:, None]


def default_tau(n: int) -> float:
    """tau = 2 n^{1/2} eps_mach, the conservative tolerance recommended in Sec. 2.1."""
    return 2.0 * np.sqrt(n) * EPS


def stop_check(i: int, res_hist, theta_hist, sigma11: float, tau: float, use_stagnation: bool):
    """Stopping decision after iteration i (Sec. 2.1, Alg. 1 and Alg. 2).

    res_hist[t] holds the b residual column norms ||R_t(:, j)|| for t = 0 .. i+1 and
    theta_hist[t] the b current singular value estimates (theta_hist[0] = +inf, Alg. 1).
    Returns (tol_check, stag_check_1, stag_check_2); the method stops when the tolerance check
    holds and, if stagnation checks are on, both stagnation checks hold too.
    """
    def r(t):
        return np.asarray(res_hist[t], dtype=np.float64) if t >= 0 else np.inf

    def th(t):
        return np.asarray(theta_hist[t], dtype=np.float64) if t >= 0 else np.inf

    tol = bool(np.max(r(i + 1)) <= sigma11 ** 2 * tau)
    if not use_stagnation:
        return tol, True, True
    with np.errstate(divide="ignore", invalid="ignore"):
        s1 = bool(np.all(1.1 * r(i + 1) >= r(i - 4)))
        lhs = 1.1 * (th(i - 4) - th(i + 1)) / th(i + 1)
        rhs = (th(i - 9) - th(i - 4)) / th(i - 4)
        s2 = bool(np.all(lhs >= rhs))
    return tol, s1, s2


def rlobpcg(A: np.ndarray, k: int, b: int | None = None, d: int | None = None, zeta: int = 8,
            seed: int = 0, tau: float | None = None, max_iter: int | None = None,
            check_every: int | None = None, use_stagnation: bool = True,
            sketch_precision: str = "f64", fixed_iters: int | None = None,
            keep_iterates: bool = False, orth_mode: str = "householder", locking: bool = False,
            precond: str = "sketch") -> dict:
    """Block RLOBPCG (Alg. 2) for the k smallest singular triplets of a tall A (m x n).

    b is the block size (default k), d the sketch rows (default 4n), zeta the SparseStack
    sparsity. fixed_iters runs exactly that many iterations with no stopping test.
    orth_mode: "householder" (Orth of Alg. 2 after the two block Gram-Schmidt passes) or "svqb"
    (SVQB in its place, the alternative Sec. 2.1 names). locking: deflate converged columns
    (Sec. 2.3): a column whose residual meets the tolerance sigma11^2 tau is locked -- kept in V
    with its value frozen, while X and W lose its column, W is made orthogonal to all of V, and
    Rayleigh-Ritz runs on the active columns only, so the trial space stays orthogonal to the
    converged vectors; the solve also ends when every column is locked.
    precond: the P of W = P (P^* R): "sketch" (P = V~ Sigma~^{-1}, Alg. 2), "diag"
    (P = diag(||A(:, i)||^{-1}), the diagonally preconditioned LOBPCG of Sec. 1.1) or "none"
    (P = I, LOBPCG without a preconditioner, Sec. 1.1); every variant starts from the same
    sketch-and-solve block and stops by the same rule (Sec. 1.1 starts all methods from v0).
    Returns a dict with sigma (k, ascending), V (n x k), U = A V diag(sigma)^{-1} (m x k),
    resid (k residual column norms), iters, stop_reason, sigma11 (= Sigma~(1,1)) and the
    per-iteration history of the b estimates and residual norms.
    """
    A = np.asarray(A)
    m, n = A.shape
    b = k if b is None else b
    if not (1 <= k <= b and 3 * b <= n and n <= m):
        raise ValueError("need 1 <= k <= b, 3b <= n <= m")
    d = 4 * n if d is None else d
    tau = default_tau(n) if tau is None else tau
    if max_iter is None:
        max_iter = 200 if b == 1 else 100
    if check_every is None:
        check_every = 5 if use_stagnation else 1
    cplx = np.iscomplexobj(A)
    wt = np.complex128 if cplx else np.float64
    A = A.astype(wt, copy=False)
    AH = A.conj().T

    # Sketch and factorise (the first steps of Alg. 2): P = V~ Sigma~^{-1}. The refined form
    # keeps SA in FP64 and takes V~, Sigma~ from its refined QR factor (SVD(SA) = SVD(R)).
    if sketch_precision == "f32_refine":
        SA = sketch(A, d, zeta, seed, "f64")
        s, Vt = sketch_svd(refined_factor(SA))
    else:
        SA = sketch(A, d, zeta, seed, sketch_precision)
        s, Vt = sketch_svd(SA)
    s = s.astype(np.float64)
    Vt = Vt.astype(wt)
    sigma11 = float(s[0])
    if precond == "sketch":
        P = Vt / s[None, :]
    elif precond == "diag":
        P = np.diag(1.0 / np.linalg.norm(A, axis=0)).astype(wt)
    elif precond == "none":
        P = np.eye(n, dtype=wt)
    else:
        raise ValueError(f"unknown precond {precond!r}")

    # Sketch-and-solve start and the initial Rayleigh-Ritz step (Alg. 2)
    V = orth(Vt[:, n - b:])
    AV = A @ V
    theta, C = rayleigh_ritz(AV)
    V = V @ C
    AV = AV @ C
    Res = AH @ AV - V * (theta ** 2)[None, :]
    theta0 = theta.copy()
    X = np.zeros((n, 0), dtype=wt)
    AX = np.zeros((m, 0), dtype=wt)

    if orth_mode not in ("householder", "svqb"):
        raise ValueError(f"unknown orth_mode {orth_mode!r}")
    normalise = orth if orth_mode == "householder" else svqb
    rnorm = np.linalg.norm(Res, axis=0)
    res_hist = [rnorm.copy()]
    theta_hist = [np.full(b, np.inf)]
    theta_s = theta.copy()
    locked = np.zeros(b, dtype=bool)
    act = np.arange(b)                  # active columns (all of them without locking)
    matvecs = b
    it_hist = []
    stop_reason = "max_iter"
    n_iter = fixed_iters if fixed_iters is not None else max_iter
    i = -1
    for i in range(n_iter):
        a = act.size
        # Search direction (Alg. 2): W = P (P^* R_i), for the active columns
        W = P @ (P.conj().T @ Res[:, act])
        # BCGS2 against [V X] (all of V: locked columns too), then Orth (or SVQB)
        VX = projection_set(V, X, act)
        W = W - VX @ (VX.conj().T @ W)
        W = normalise(W - VX @ (VX.conj().T @ W))
        # Trial space and its image: only W is multiplied by A
        T = np.concatenate([V[:, act], X, W], axis=1)
        AT = np.concatenate([AV[:, act], AX, A @ W], axis=1)
        matvecs += a
        # Rayleigh-Ritz by SVD of A_T
        theta, C = rayleigh_ritz(AT)
        ncol = T.shape[1]
        Cs = C[:, ncol - a:]
        theta_s[act] = theta[ncol - a:]
        V[:, act] = T @ Cs
        AV[:, act] = AT @ Cs
        # Residual matrix R_{i+1} = A^* A_V - V Theta^2 (direct product, as in Alg. 2)
        Res[:, act] = AH @ AV[:, act] - V[:, act] * (theta_s[act] ** 2)[None, :]
        rnorm[act] = np.linalg.norm(Res[:, act], axis=0)
        res_hist.append(rnorm.copy())
        theta_hist.append(theta_s.copy())
        if keep_iterates:
            it_hist.append(V.copy())
        if fixed_iters is None and i % check_every == 0:
            tol, s1, s2 = stop_check(i, res_hist, theta_hist, sigma11, tau, use_stagnation)
            if tol and s1 and s2:
                stop_reason = "converged"
                break
        # Momentum basis X (eq. x-defining): Q = Orth(C(1:a, 1:ncol-a)^*); column p belongs to
        # the p-th active column
        Q = orth(C[:a, : ncol - a].conj().T)
        CQ = C[:, : ncol - a] @ Q
        X = T @ CQ
        AX = AT @ CQ
        if locking:
            newly = rnorm[act] <= sigma11 ** 2 * tau
            if newly.any():
                locked[act[newly]] = True
                X = X[:, ~newly]
                AX = AX[:, ~newly]
                act = act[~newly]
                if act.size == 0:       # every column locked: the solve ends
                    stop_reason = "converged"
                    break

    if fixed_iters is not None:
        stop_reason = "fixed_iters"
    # Outputs (the end of Alg. 2), returned in ascending order of sigma
    # (theta_s is descending without locking; sorting its reverse keeps the reversed order for ties)
    order = (b - 1 - np.argsort(theta_s[::-1], kind="stable"))[:k]
    sig = theta_s[order]
    Vk = V[:, order]
    with np.errstate(divide="ignore", invalid="ignore"):
        U = AV[:, order] / sig[None, :]
    return {
        "sigma": sig, "V": Vk, "U": U, "resid": rnorm[order],
        "iters": i + 1, "stop_reason": stop_reason, "sigma11": sigma11, "sketch_sigma": s,
        "theta0": theta0,
        "res_hist": np.array(res_hist), "theta_hist": np.array(theta_hist), "iterates": it_hist,
        "matvecs": matvecs, "locked": locked.copy(),
    }
