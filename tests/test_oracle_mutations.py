"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins catch each one.

A pin that a wrong oracle still passes pins nothing; each case below replaces one building block
of the oracle with a subtly wrong version and expects one of the pins of test_oracle_pins.py to
fail.
"""
import sys

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins

MOD = sys.modules["oracle.rlobpcg"]


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(MOD, name, fn)
    monkeypatch.setattr(oracle, name, fn)


def _expect_failure(check):
    with pytest.raises(AssertionError):
        check()


def test_wrong_splitmix_constant_is_caught(monkeypatch):
    orig = MOD.splitmix64

    def bad(seed, counter):
        return orig(seed, counter) ^ np.uint64(1 << 17)
    _patch(monkeypatch, "splitmix64", bad)
    _expect_failure(pins.test_splitmix64_published_vectors)


def test_off_by_one_piece_bounds_is_caught(monkeypatch):
    def bad(d, zeta):
        return np.array([(j * d + zeta - 1) // zeta for j in range(zeta + 1)], dtype=np.int64)
    _patch(monkeypatch, "piece_bounds", bad)
    _expect_failure(lambda: pins.test_sparse_stack_structure(300, 37, 4))


def test_wrong_sketch_scaling_is_caught(monkeypatch):
    orig = MOD.sketch

    def bad(A, d, zeta, seed, precision="f64"):
        return orig(A, d, zeta, seed, precision) * zeta      # zeta^{+1/2} instead of zeta^{-1/2}
    _patch(monkeypatch, "sketch", bad)
    _expect_failure(lambda: pins.test_randomized_preconditioning_fact(False))


def test_transposed_sketch_vectors_are_caught(monkeypatch):
    def bad(SA):
        _, s, Vh = np.linalg.svd(SA, full_matrices=False)
        return s, Vh                                         # rows instead of columns
    _patch(monkeypatch, "sketch_svd", bad)
    _expect_failure(lambda: pins.test_randomized_preconditioning_fact(False))


def test_largest_instead_of_smallest_ritz_is_caught(monkeypatch):
    def bad(AT):
        _, th, Ch = np.linalg.svd(AT, full_matrices=False)
        return th[::-1], Ch.conj().T[:, ::-1]                # ascending: keeps the largest
    _patch(monkeypatch, "rayleigh_ritz", bad)
    _expect_failure(pins.test_planted_small_workload)


def test_missing_normalisation_in_orth_is_caught(monkeypatch):
    def bad(M):
        return M                                             # no orthonormalisation at all
    _patch(monkeypatch, "orth", bad)
    _expect_failure(lambda: pins.test_block_planted_cluster(False))


def test_missing_conjugation_is_caught(monkeypatch):
    def bad(AT):
        _, th, Ch = np.linalg.svd(AT, full_matrices=False)
        return th, Ch.T                                      # transpose without conjugate
    _patch(monkeypatch, "rayleigh_ritz", bad)
    _expect_failure(lambda: pins.test_block_planted_cluster(True))


def test_wrong_stagnation_index_is_caught(monkeypatch):
    orig = MOD.stop_check

    def bad(i, res_hist, theta_hist, sigma11, tau, use_stagnation):
        return orig(i - 1, res_hist, theta_hist, sigma11, tau, use_stagnation)
    _patch(monkeypatch, "stop_check", bad)
    _expect_failure(pins.test_stop_rule_hand_worked)


def test_gram_pass_without_conjugate_is_caught(monkeypatch):
    def bad(A, W):
        AW = A @ W
        return AW, A.T @ AW                                  # A^T instead of A^H
    _patch(monkeypatch, "gram_pass", bad)
    _expect_failure(lambda: pins.test_gram_pass_exact_on_integers(True))


def test_gram_pass_dropping_a_row_is_caught(monkeypatch):
    def bad(A, W):
        AW = A @ W
        return AW, A[1:].conj().T @ AW[1:]                   # first row missing from the sum
    _patch(monkeypatch, "gram_pass", bad)
    _expect_failure(lambda: pins.test_gram_pass_exact_on_integers(False))
    _expect_failure(pins.test_gram_pass_within_rounding_of_exact_rationals)


def test_refinement_dropped_is_caught(monkeypatch):
    def bad(SA):
        low = np.complex64 if np.iscomplexobj(SA) else np.float32
        return np.linalg.qr(SA.astype(low), mode="r").astype(SA.dtype)   # the FP32 factor alone
    _patch(monkeypatch, "refined_factor", bad)
    _expect_failure(lambda: pins.test_refined_factor_is_a_qr_factor_of_the_sketch(False, 1e10))
    _expect_failure(lambda: pins.test_refined_factor_satisfies_the_preconditioning_fact(False))


def test_refinement_without_conjugate_is_caught(monkeypatch):
    orig = MOD.refined_factor

    def bad(SA):
        return orig(SA).conj()                                              # a transposed-only Gram
    _patch(monkeypatch, "refined_factor", bad)
    _expect_failure(lambda: pins.test_refined_factor_is_a_qr_factor_of_the_sketch(True, 1e13))


def test_locking_without_deflation_is_caught(monkeypatch):
    def bad(V, X, act):
        return np.concatenate([V[:, act], X], axis=1)      # locked columns left out of the projection
    _patch(monkeypatch, "projection_set", bad)
    _expect_failure(lambda: pins.test_locking_deflates_converged_columns("householder"))


def test_svqb_without_the_eigen_scaling_is_caught(monkeypatch):
    def bad(W, tau=oracle.EPS):
        S = W.conj().T @ W
        D = 1.0 / np.sqrt(np.real(np.diagonal(S)))
        return W * D[None, :]                             # column scaling only
    _patch(monkeypatch, "svqb", bad)
    _expect_failure(lambda: pins.test_svqb_orthonormalises_and_keeps_the_span(False))


def test_no_preconditioner_that_is_diagonal_is_caught(monkeypatch):
    orig = oracle.rlobpcg

    def bad(*a, **kw):
        if kw.get("precond") == "none":
            kw["precond"] = "diag"
        return orig(*a, **kw)
    monkeypatch.setattr(oracle, "rlobpcg", bad)
    _expect_failure(pins.test_no_preconditioner_is_rotation_covariant)


def test_diagonal_preconditioner_that_is_none_is_caught(monkeypatch):
    orig = oracle.rlobpcg

    def bad(*a, **kw):
        if kw.get("precond") == "diag":
            kw["precond"] = "none"
        return orig(*a, **kw)
    monkeypatch.setattr(oracle, "rlobpcg", bad)
    _expect_failure(pins.test_diagonal_preconditioner_is_exact_for_orthogonal_columns)
