"""Python binding of the C ABI in include/rlobpcg.h (argument marshalling only).

Every entry point keeps the C name. Device buffers are passed as integer addresses (e.g.
``tensor.data_ptr()`` of a CUDA torch tensor) and streams as ``cudaStream_t`` handles
(``torch.cuda.current_stream().cuda_stream``). There is no CPU fallback: if the compiled library
is missing, loading fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_int, c_int64, c_uint64, c_double, c_size_t, c_void_p, c_char_p = (
    ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_char_p)

RLOBPCG_OK = 0
RLOBPCG_NOT_CONVERGED = 1
RLOBPCG_ERR_INVALID_ARG = -1
RLOBPCG_ERR_OOM = -2
RLOBPCG_ERR_CUDA = -3
RLOBPCG_ERR_NONFINITE = -4
RLOBPCG_ERR_TIMEOUT = -5
RLOBPCG_ERR_UNSUPPORTED = -6
RLOBPCG_ERR_CANCELLED = -7
RLOBPCG_F64 = 0
RLOBPCG_C128 = 1
RLOBPCG_SKETCH_F64 = 0
RLOBPCG_SKETCH_F32 = 1
RLOBPCG_SKETCH_F32_REFINE = 2
RLOBPCG_PRECOND_SKETCH = 0
RLOBPCG_PRECOND_DIAG = 1
RLOBPCG_PRECOND_NONE = 2
RLOBPCG_ORTH_HOUSEHOLDER = 0
RLOBPCG_ORTH_SVQB = 1
RLOBPCG_STOP_CONVERGED = 0
RLOBPCG_STOP_MAX_ITER = 1
RLOBPCG_STOP_FIXED = 2
RLOBPCG_SERVE_STREAMS = 0
RLOBPCG_SERVE_BATCHED = 1


class rlobpcg_opts(ctypes.Structure):
    _fields_ = [("seed", c_uint64), ("d", c_int), ("zeta", c_int), ("block", c_int), ("max_iter", c_int),
                ("check_every", c_int), ("use_stagnation", c_int), ("sketch_prec", c_int), ("fixed_iters", c_int),
                ("residual_refresh_every", c_int), ("exact_sketch_svd", c_int), ("gram_split", c_int),
                ("tau", c_double), ("orth_mode", c_int), ("locking", c_int), ("precond", c_int)]


class rlobpcg_info(ctypes.Structure):
    _fields_ = [("iters", c_int), ("matvecs", c_int), ("stop_reason", c_int), ("block", c_int),
                ("sigma11", c_double), ("ms_sketch", c_double), ("ms_factor", c_double), ("ms_iterate", c_double),
                ("ms_total", c_double), ("ms_gram", c_double), ("gram_passes", c_int), ("kernel_launches", c_int),
                ("jacobi_sweeps", c_int), ("ms_gram_ab", c_double), ("ms_gram_atb", c_double), ("ms_split_a", c_double),
                ("rr_sweeps", c_int), ("rr_calls", c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class rlobpcg_engine_stats(ctypes.Structure):
    _fields_ = [("replays", c_int64), ("joins", c_int64), ("retires", c_int64), ("rebuilds", c_int64),
                ("gpu_ms", c_double), ("host_ms", c_double), ("active_mean", c_double)]


class RlobpcgError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__(f"{fn} failed: {rlobpcg_status_string(code)} ({code}); {rlobpcg_last_error()}")


_SIGS = {
    "rlobpcg_default_opts": (c_int, [ctypes.POINTER(rlobpcg_opts)]),
    "rlobpcg_plan": (c_int, [ctypes.POINTER(c_void_p), c_int64, c_int64, c_int, c_int, ctypes.POINTER(rlobpcg_opts),
                             c_void_p]),
    "rlobpcg_solve": (c_int, [c_void_p, c_void_p, c_int64, c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                              ctypes.POINTER(rlobpcg_info)]),
    "rlobpcg_solve_async": (c_int, [c_void_p, c_void_p, c_int64, c_double, c_void_p, c_void_p, c_void_p, c_void_p,
                                    ctypes.POINTER(rlobpcg_info)]),
    "rlobpcg_solve_wait": (c_int, [c_void_p]),
    "rlobpcg_plan_destroy": (c_int, [c_void_p]),
    "rlobpcg_status_string": (c_char_p, [c_int]),
    "rlobpcg_last_error": (c_char_p, []),
    "rlobpcg_sketch": (c_int, [c_void_p, c_int64, c_int64, c_int64, c_int, c_int, c_int, c_uint64, c_int, c_void_p,
                               c_void_p]),
    "rlobpcg_factor": (c_int, [c_void_p, c_int64, c_int64, c_int, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                               c_void_p, c_size_t, c_void_p]),
    "rlobpcg_factor_workspace_size": (c_size_t, [c_int64, c_int64, c_int, c_int]),
    "rlobpcg_gram": (c_int, [c_void_p, c_int64, c_int64, c_int64, c_int, c_void_p, c_int, c_int64, c_void_p, c_int64,
                             c_void_p, c_int64, c_void_p, c_size_t, c_void_p]),
    "rlobpcg_gram_workspace_size": (c_size_t, [c_int64, c_int64, c_int, c_int]),
    "rlobpcg_gram_noalloc": (c_int, [c_void_p, c_int64, c_int64, c_int64, c_int, c_void_p, c_int, c_int64, c_void_p,
                                     c_int64, c_void_p, c_int64, c_void_p]),
    "rlobpcg_gram_split_prepare_size": (c_size_t, [c_int64, c_int64]),
    "rlobpcg_gram_split_prepare": (c_int, [c_void_p, c_int64, c_int64, c_int64, c_void_p, c_size_t, c_void_p]),
    "rlobpcg_gram_split_workspace_size": (c_size_t, [c_int64, c_int64, c_int]),
    "rlobpcg_gram_split": (c_int, [c_void_p, c_int64, c_int64, c_void_p, c_int, c_int64, c_void_p, c_int64, c_void_p,
                                   c_int64, c_void_p, c_size_t, c_void_p]),
    "rlobpcg_gram_split_c128_workspace_size": (c_size_t, [c_int64, c_int64, c_int]),
    "rlobpcg_gram_split_c128": (c_int, [c_void_p, c_int64, c_int64, c_void_p, c_int, c_int64, c_void_p, c_int64,
                                        c_void_p, c_int64, c_void_p, c_size_t, c_void_p]),
    "rlobpcg_tsqr": (c_int, [c_void_p, c_int64, c_int, c_int64, c_int, c_void_p, c_void_p, c_size_t, c_void_p]),
    "rlobpcg_tsqr_workspace_size": (c_size_t, [c_int64, c_int, c_int]),
    "rlobpcg_plan_device_bytes": (c_size_t, [c_void_p]),
    "rlobpcg_history": (c_int, [c_void_p, c_void_p, c_void_p, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "rlobpcg_plan_workspace_size": (c_size_t, [c_int64, c_int64, c_int, c_int, ctypes.POINTER(rlobpcg_opts)]),
    "rlobpcg_server_create": (c_int, [ctypes.POINTER(c_void_p), c_size_t, c_int, c_int]),
    "rlobpcg_server_create_ex": (c_int, [ctypes.POINTER(c_void_p), c_size_t, c_int, c_int, c_int]),
    "rlobpcg_server_engine_stats": (c_int, [c_void_p, ctypes.POINTER(rlobpcg_engine_stats)]),
    "rlobpcg_server_set_batch_limit": (c_int, [c_void_p, c_int64]),
    "rlobpcg_server_submit": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int, c_int,
                                      ctypes.POINTER(rlobpcg_opts), ctypes.POINTER(c_int64)]),
    "rlobpcg_server_poll": (c_int, [c_void_p, c_int64]),
    "rlobpcg_server_wait": (c_int, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, ctypes.POINTER(rlobpcg_info),
                                    ctypes.POINTER(c_double)]),
    "rlobpcg_server_stats": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_double),
                                     ctypes.POINTER(c_double), ctypes.POINTER(c_double), ctypes.POINTER(c_size_t),
                                     ctypes.POINTER(c_int)]),
    "rlobpcg_server_destroy": (c_int, [c_void_p]),
    "rlobpcg_check_bounded_wait": (c_int, [c_int, c_int, c_void_p]),
    "rlobpcg_solve_batch": (c_int, [c_int, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                    ctypes.POINTER(c_int64), ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                    ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                    ctypes.POINTER(rlobpcg_info), ctypes.POINTER(c_int), c_void_p]),
    "rlobpcg_batch_tile": (c_int, [c_int64, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_void_p]),
    "rlobpcg_batch_set_tile": (c_int, [c_int64, c_int, c_int, c_int]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load librlobpcg.so (the in-tree build). Raises if it is missing, unless asked to build."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
                               "or paper_2602_16797_gb300.build.build() (needs nvcc)")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols() -> list[str]:
    return list(_SIGS)


def _check(fn, rc, ok=(RLOBPCG_OK,)):
    if rc not in ok:
        raise RlobpcgError(fn, rc)
    return rc


# ---- thin wrappers, one per C entry point ------------------------------------------------------

def rlobpcg_status_string(code: int) -> str:
    return load().rlobpcg_status_string(code).decode()


def rlobpcg_last_error() -> str:
    return load().rlobpcg_last_error().decode()


def rlobpcg_default_opts() -> rlobpcg_opts:
    o = rlobpcg_opts()
    _check("rlobpcg_default_opts", load().rlobpcg_default_opts(ctypes.byref(o)))
    return o


def rlobpcg_plan(m: int, n: int, k: int, dtype: int, opts: rlobpcg_opts | None = None, stream: int = 0) -> int:
    h = c_void_p()
    rc = load().rlobpcg_plan(ctypes.byref(h), m, n, k, dtype, ctypes.byref(opts) if opts is not None else None, stream)
    _check("rlobpcg_plan", rc)
    return h.value


def rlobpcg_solve(plan: int, A: int, lda: int, tol: float, sigma: int, V: int, U: int | None = None,
                  resid: int | None = None, info: rlobpcg_info | None = None) -> int:
    rc = load().rlobpcg_solve(plan, A, lda, tol, sigma, V, U, resid, ctypes.byref(info) if info is not None else None)
    return _check("rlobpcg_solve", rc, ok=(RLOBPCG_OK, RLOBPCG_NOT_CONVERGED))


def rlobpcg_solve_async(plan: int, A: int, lda: int, tol: float, sigma: int, V: int, U: int | None = None,
                        resid: int | None = None, info: rlobpcg_info | None = None) -> None:
    """Start the solve on a library thread; the buffers (and info) must outlive rlobpcg_solve_wait."""
    rc = load().rlobpcg_solve_async(plan, A, lda, tol, sigma, V, U, resid,
                                    ctypes.byref(info) if info is not None else None)
    _check("rlobpcg_solve_async", rc)


def rlobpcg_solve_wait(plan: int) -> int:
    return _check("rlobpcg_solve_wait", load().rlobpcg_solve_wait(plan), ok=(RLOBPCG_OK, RLOBPCG_NOT_CONVERGED))


def rlobpcg_plan_destroy(plan: int) -> None:
    _check("rlobpcg_plan_destroy", load().rlobpcg_plan_destroy(plan))


def rlobpcg_sketch(A: int, m: int, n: int, lda: int, dtype: int, d: int, zeta: int, seed: int, sketch_prec: int,
                   SA: int, stream: int = 0) -> None:
    _check("rlobpcg_sketch", load().rlobpcg_sketch(A, m, n, lda, dtype, d, zeta, seed, sketch_prec, SA, stream))


def rlobpcg_factor_workspace_size(d: int, n: int, dtype: int, sketch_prec: int) -> int:
    return load().rlobpcg_factor_workspace_size(d, n, dtype, sketch_prec)


def rlobpcg_factor(SA: int, d: int, n: int, dtype: int, sketch_prec: int, R: int | None, sigma: int, Vt: int,
                   Rinv: int | None, work: int, work_bytes: int, stream: int = 0) -> None:
    _check("rlobpcg_factor", load().rlobpcg_factor(SA, d, n, dtype, sketch_prec, R, sigma, Vt, Rinv, work, work_bytes,
                                                   stream))


def rlobpcg_gram_workspace_size(m: int, n: int, b: int, dtype: int) -> int:
    return load().rlobpcg_gram_workspace_size(m, n, b, dtype)


def rlobpcg_gram(A: int, m: int, n: int, lda: int, dtype: int, W: int, b: int, ldw: int, AW: int, ldaw: int, G: int,
                 ldg: int, work: int, work_bytes: int, stream: int = 0) -> None:
    _check("rlobpcg_gram", load().rlobpcg_gram(A, m, n, lda, dtype, W, b, ldw, AW, ldaw, G, ldg, work, work_bytes,
                                               stream))


def rlobpcg_gram_noalloc(A: int, m: int, n: int, lda: int, dtype: int, W: int, b: int, ldw: int, AW: int,
                         ldaw: int, G: int, ldg: int, stream: int = 0) -> None:
    """rlobpcg_gram without a workspace argument (scratch is the library's fixed device buffer)."""
    _check("rlobpcg_gram_noalloc", load().rlobpcg_gram_noalloc(A, m, n, lda, dtype, W, b, ldw, AW, ldaw, G, ldg,
                                                               stream))


def rlobpcg_gram_split_prepare_size(m: int, n: int) -> int:
    return load().rlobpcg_gram_split_prepare_size(m, n)


def rlobpcg_gram_split_prepare(A: int, m: int, n: int, lda: int, prep: int, prep_bytes: int, stream: int = 0) -> None:
    _check("rlobpcg_gram_split_prepare", load().rlobpcg_gram_split_prepare(A, m, n, lda, prep, prep_bytes, stream))


def rlobpcg_gram_split_workspace_size(m: int, n: int, b: int) -> int:
    return load().rlobpcg_gram_split_workspace_size(m, n, b)


def rlobpcg_gram_split(prep: int, m: int, n: int, W: int, b: int, ldw: int, AW: int, ldaw: int, G: int, ldg: int,
                       work: int, work_bytes: int, stream: int = 0) -> None:
    _check("rlobpcg_gram_split", load().rlobpcg_gram_split(prep, m, n, W, b, ldw, AW, ldaw, G, ldg, work, work_bytes,
                                                           stream))


def rlobpcg_gram_split_c128_workspace_size(m: int, n: int, b: int) -> int:
    return load().rlobpcg_gram_split_c128_workspace_size(m, n, b)


def rlobpcg_gram_split_c128(prep: int, m: int, n: int, W: int, b: int, ldw: int, AW: int, ldaw: int, G: int,
                            ldg: int, work: int, work_bytes: int, stream: int = 0) -> None:
    _check("rlobpcg_gram_split_c128", load().rlobpcg_gram_split_c128(prep, m, n, W, b, ldw, AW, ldaw, G, ldg, work,
                                                                      work_bytes, stream))


def rlobpcg_tsqr_workspace_size(m: int, c: int, dtype: int) -> int:
    return load().rlobpcg_tsqr_workspace_size(m, c, dtype)


def rlobpcg_tsqr(X: int, m: int, c: int, ldx: int, dtype: int, R: int, work: int, work_bytes: int,
                 stream: int = 0) -> None:
    _check("rlobpcg_tsqr", load().rlobpcg_tsqr(X, m, c, ldx, dtype, R, work, work_bytes, stream))


# ---- convenience for torch tensors (still only marshalling) -----------------------------------

def _torch_dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float64:
        return RLOBPCG_F64
    if t.dtype == torch.complex128:
        return RLOBPCG_C128
    raise TypeError("A must be float64 or complex128")


def solve(A, k: int, *, opts: rlobpcg_opts | None = None, tol: float = -1.0, want_u: bool = False,
          stream: int | None = None):
    """Smallest k singular triplets of A (torch tensor, CUDA or CPU-pinned; float64/complex128).

    Returns (sigma [k] float64, V [n, k], U [m, k] or None, resid [k] -- all on the GPU -- and the
    info dict).
    """
    import torch
    m, n = A.shape
    dtype = _torch_dtype_code(A)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    plan = rlobpcg_plan(m, n, k, dtype, opts, stream)
    try:
        dev = A.device if A.is_cuda else torch.device("cuda")
        sigma = torch.empty(k, dtype=torch.float64, device=dev)
        resid = torch.empty(k, dtype=torch.float64, device=dev)
        V = torch.empty((n, k), dtype=A.dtype, device=dev)
        U = torch.empty((m, k), dtype=A.dtype, device=dev) if want_u else None
        info = rlobpcg_info()
        rc = rlobpcg_solve(plan, A.data_ptr(), A.stride(0), tol, sigma.data_ptr(), V.data_ptr(),
                           U.data_ptr() if U is not None else None, resid.data_ptr(), info)
        out = info.as_dict()
        out["status"] = rc
        return sigma, V, U, resid, out
    finally:
        rlobpcg_plan_destroy(plan)


def rlobpcg_history(plan: int):
    """(theta, resnorm) of the plan's last solve as numpy arrays [iterations + 1, b]."""
    import numpy as np
    rows, b = c_int(), c_int()
    _check("rlobpcg_history", load().rlobpcg_history(plan, None, None, 0, ctypes.byref(rows), ctypes.byref(b)))
    th = np.zeros((rows.value, b.value))
    rs = np.zeros((rows.value, b.value))
    _check("rlobpcg_history", load().rlobpcg_history(plan, th.ctypes.data, rs.ctypes.data, rows.value,
                                                     ctypes.byref(rows), ctypes.byref(b)))
    return th, rs


def rlobpcg_plan_device_bytes(plan: int) -> int:
    return load().rlobpcg_plan_device_bytes(plan)


def rlobpcg_plan_workspace_size(m: int, n: int, k: int, dtype: int, opts: rlobpcg_opts | None = None) -> int:
    return load().rlobpcg_plan_workspace_size(m, n, k, dtype, ctypes.byref(opts) if opts is not None else None)


def rlobpcg_server_create(budget_bytes: int, max_active: int, device: int = 0, mode: int | None = None) -> int:
    h = c_void_p()
    if mode is None:
        _check("rlobpcg_server_create", load().rlobpcg_server_create(ctypes.byref(h), budget_bytes, max_active, device))
    else:
        _check("rlobpcg_server_create_ex",
               load().rlobpcg_server_create_ex(ctypes.byref(h), budget_bytes, max_active, device, mode))
    return h.value


def rlobpcg_server_submit(server: int, A: int, m: int, n: int, lda: int, k: int, dtype: int,
                          opts: rlobpcg_opts | None = None) -> int:
    t = c_int64()
    _check("rlobpcg_server_submit", load().rlobpcg_server_submit(server, A, m, n, lda, k, dtype,
                                                                 ctypes.byref(opts) if opts is not None else None,
                                                                 ctypes.byref(t)))
    return t.value


def rlobpcg_server_poll(server: int, ticket: int) -> int:
    return load().rlobpcg_server_poll(server, ticket)


def rlobpcg_server_wait(server: int, ticket: int, sigma: int | None, V: int | None, resid: int | None,
                        info: rlobpcg_info | None = None):
    lat = c_double()
    rc = load().rlobpcg_server_wait(server, ticket, sigma, V, resid, ctypes.byref(info) if info is not None else None,
                                    ctypes.byref(lat))
    _check("rlobpcg_server_wait", rc, ok=(RLOBPCG_OK, RLOBPCG_NOT_CONVERGED))
    return rc, lat.value


def rlobpcg_server_stats(server: int) -> dict:
    c, p50, p99, sps, pk, pr = c_int64(), c_double(), c_double(), c_double(), c_size_t(), c_int()
    _check("rlobpcg_server_stats", load().rlobpcg_server_stats(server, ctypes.byref(c), ctypes.byref(p50),
                                                               ctypes.byref(p99), ctypes.byref(sps), ctypes.byref(pk),
                                                               ctypes.byref(pr)))
    return {"completed": c.value, "p50_ms": p50.value, "p99_ms": p99.value, "solves_per_s": sps.value,
            "peak_bytes": pk.value, "peak_running": pr.value}


def rlobpcg_server_destroy(server: int) -> None:
    _check("rlobpcg_server_destroy", load().rlobpcg_server_destroy(server))


def rlobpcg_check_bounded_wait(kind: int, spins: int, stream: int | None = None) -> int:
    """Status of the bounded-wait health check (RLOBPCG_ERR_TIMEOUT when the path works)."""
    return load().rlobpcg_check_bounded_wait(kind, spins, stream)


def rlobpcg_solve_batch(plans, A, lda, sigma, V, U, resid, stream: int | None = None):
    """Batched solves (pointers as ints; U / resid entries may be None). Returns (rc, infos,
    statuses)."""
    n = len(plans)
    arr = lambda xs: (c_void_p * n)(*[x if x else None for x in xs])
    infos = (rlobpcg_info * n)()
    st = (c_int * n)()
    rc = load().rlobpcg_solve_batch(n, arr(plans), arr(A), (c_int64 * n)(*lda), arr(sigma), arr(V),
                                    arr(U) if U is not None else None, arr(resid) if resid is not None else None,
                                    infos, st, stream)
    return rc, list(infos), list(st)


def rlobpcg_batch_tile(n: int, b: int, stream: int | None = None):
    """(trows, rt) of the batched kernels for the (n, b) class (autotuned on first use)."""
    t, r = c_int(), c_int()
    _check("rlobpcg_batch_tile", load().rlobpcg_batch_tile(n, b, ctypes.byref(t), ctypes.byref(r), stream))
    return t.value, r.value


def rlobpcg_batch_set_tile(n: int, b: int, trows: int, rt: int) -> None:
    _check("rlobpcg_batch_set_tile", load().rlobpcg_batch_set_tile(n, b, trows, rt))


def rlobpcg_server_engine_stats(server: int) -> dict:
    st = rlobpcg_engine_stats()
    _check("rlobpcg_server_engine_stats", load().rlobpcg_server_engine_stats(server, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in rlobpcg_engine_stats._fields_}


def rlobpcg_server_set_batch_limit(server: int, max_mnb: int) -> None:
    _check("rlobpcg_server_set_batch_limit", load().rlobpcg_server_set_batch_limit(server, max_mnb))
