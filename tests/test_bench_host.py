"""Host-side helpers of bench.py that feed the roofline and CPU-baseline objects (no GPU needed).

The Gram pass must move A once and write A W once (its algorithmic bytes); the split-bf16 form
also runs a fixed number of digit-pair products on the tensor cores. The roofline takes the
slower of the two roofs as the bound and reports the other beside it. DRAM traffic is scaled
from the committed ncu summary only when that summary was taken on the current kernel source.
The CPU baseline scales a row sample of the oracle: the parts that stream A by m / sample_m, the
SVD of the d x n sketch not at all.
"""
import hashlib
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("m,n,b,cplx", [(100000, 500, 5, False), (1, 1, 1, False), (200000, 300, 3, True),
                                         (1000000, 1000, 10, False)])
def test_pass_algorithmic_bytes_are_one_read_of_A_and_one_write_of_AW(m, n, b, cplx):
    esz = 16 if cplx else 8
    assert bench.pass_algorithmic_bytes(m, n, b, cplx) == esz * m * n + esz * m * b


def test_pass_tensor_flops_count_both_products_over_all_digit_pairs():
    m, n, b = 1000000, 1000, 10
    assert bench.pass_tensor_flops(m, n, b) == 2 * bench.DIGIT_PAIRS * 2 * m * n * b


def test_roofline_takes_the_slower_roof_as_the_bound():
    peaks = {"hbm_gbs": 6779.0, "bf16_tflops_sustained": 1710.4}
    m, n = 1000000, 1000
    # b = 20: tensor work 3.44e12 flop (2.01 ms) against 8.16 GB (1.20 ms): tensor-bound
    r = bench.gram_roofline(m, n, 20, False, True, 3.0e-3, peaks, 1.26, "derived")
    assert r["bound"] == "tensor" and r["other"]["bound"] == "hbm"
    assert r["frac"] == pytest.approx(bench.pass_tensor_flops(m, n, 20) / 3.0e-3 / 1e12 / 1710.4)
    assert r["other"]["frac"] == pytest.approx(bench.pass_algorithmic_bytes(m, n, 20, False) / 3.0e-3 / 1e9 / 6779.0)
    # b = 1: 0.26e12 flop (0.15 ms) against 8.01 GB (1.18 ms): HBM-bound
    r = bench.gram_roofline(m, n, 1, False, True, 2.0e-3, peaks, 1.26, "derived")
    assert r["bound"] == "hbm" and r["other"]["bound"] == "tensor"
    assert r["roof_ms"] == pytest.approx(bench.pass_algorithmic_bytes(m, n, 1, False) / 6779.0e9 * 1e3)
    # FP64 path: FP64 flops against the derived FP64 peak
    r = bench.gram_roofline(200000, 300, 3, True, False, 3.0e-3, peaks, 1.259, "derived")
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(16 * 200000 * 300 * 3 / 3.0e-3 / 1e12 / 1.259)
    # complex split path: the real pass on the real view (m x 2n, block 2b), 16-byte elements
    r = bench.gram_roofline(200000, 300, 3, True, True, 0.4e-3, peaks, 1.259, "derived")
    tc = r if r["bound"] == "tensor" else r["other"]
    hb = r if r["bound"] == "hbm" else r["other"]
    assert tc["flops_per_pass"] == bench.pass_tensor_flops(200000, 600, 6) == 4 * bench.pass_tensor_flops(200000, 300, 3)
    assert hb["bytes_per_pass"] == 16 * 200000 * 300 + 16 * 200000 * 3


def _fake_tree(tmp_path, src_text, summary_sha, per=8.2):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2602_16797_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "gram_tc.cu").write_text(src_text)
    (tmp_path / "profiles" / "gram_split_ncu_summary.md").write_text(
        "# summary\n\n"
        f"gram_tc.cu sha256[:16]: {summary_sha}\n"
        f"dram bytes per element of A per pass: {per}\n")


def test_traffic_scales_the_summary_when_it_matches_the_source(tmp_path, monkeypatch):
    src = "// kernel source\n"
    sha = hashlib.sha256(src.encode()).hexdigest()[:16]
    _fake_tree(tmp_path, src, sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.pass_traffic(100000, 500) == pytest.approx(8.2 * 100000 * 500)


def test_traffic_is_null_once_the_kernel_changed(tmp_path, monkeypatch):
    _fake_tree(tmp_path, "// kernel source, edited\n", "0123456789abcdef")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.pass_traffic(100000, 500) is None


def test_full_size_estimate_scales_only_what_streams_A():
    w = {"m": 1000000}
    ph = {"sample_m": 100000, "t_svd": 2.0, "t_once_stream": 0.5, "t_iter": 0.1}
    assert bench.oracle_full_solve_seconds(w, ph, 40) == pytest.approx(0.5 * 10 + 2.0 + 40 * 0.1 * 10)


def test_single_thread_oracle_sample_runs_in_a_fresh_interpreter():
    one = bench.oracle_rate_one_thread("small_4000x50", 5, timeout=240)
    assert one is not None and one[0] > 0 and one[1] > 0
    assert bench.oracle_rate_one_thread("no_such_workload", 5, timeout=120) is None


def test_sigma_error_is_relative_and_floored_for_a_nullspace():
    # planted values well above the floor: plain relative error
    assert bench.sigma_err([1.0e-10 * (1 + 1e-6)], np.array([1.0e-10]), 1.0) == pytest.approx(1e-6)
    # an exact nullspace (sigma_true = 0): the error in units of Sigma~(1,1) 2^-52, finite
    e = bench.sigma_err([3.0 * 2.0 ** -52], np.array([0.0]), 1.0)
    assert e == pytest.approx(3.0)
