"""Host-side helpers of bench.py that feed the roofline object (no GPU needed).

The split Gram kernels must move the byte digits of A (one byte per digit, eight digits per
element of the row- and column-padded matrix) plus A W and its bf16 digits; the DRAM traffic
reported beside it is scaled from the committed ncu summary only when that summary was taken on
the current kernel source.
"""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("m,n,b", [(100000, 500, 5), (1, 1, 1), (129, 17, 9), (1000000, 1000, 10)])
def test_split_algorithmic_bytes_count_the_padded_byte_digits(m, n, b):
    a = bench.split_algorithmic_bytes(m, n, b)
    mp, npad16, npad128 = -(-m // 128) * 128, -(-n // 16) * 16, -(-n // 128) * 128
    assert a["ab_digits"] == 8 * mp * npad16            # row tiles x 16-column blocks
    assert a["atb_digits"] == 8 * mp * npad128          # column tiles x row chunks
    N = 8 * (8 if b <= 8 else 16)
    y = mp * N * 2                                       # bf16 digits of A W per padded row
    assert a["ab"] == a["ab_digits"] + 8 * m * b + y
    assert a["atb"] == a["atb_digits"] + (npad128 // 128) * y


def _fake_tree(tmp_path, src_text, summary_sha, ab=1.04, atb=1.02):
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_2602_16797_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "gram_tc.cu").write_text(src_text)
    (tmp_path / "profiles" / "gram_split_ncu_summary.md").write_text(
        "# summary\n\n"
        f"gram_tc.cu sha256[:16]: {summary_sha}\n"
        f"dram bytes per digit byte (ab): {ab}\n"
        f"dram bytes per digit byte (atb): {atb}\n")


def test_traffic_scales_the_summary_when_it_matches_the_source(tmp_path, monkeypatch):
    src = "// kernel source\n"
    sha = hashlib.sha256(src.encode()).hexdigest()[:16]
    _fake_tree(tmp_path, src, sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    tr = bench.split_traffic_per_launch(100000, 500, 5)
    alg = bench.split_algorithmic_bytes(100000, 500, 5)
    assert tr == pytest.approx({"ab": 1.04 * alg["ab_digits"], "atb": 1.02 * alg["atb_digits"]})


def test_traffic_is_null_once_the_kernel_changed(tmp_path, monkeypatch):
    _fake_tree(tmp_path, "// kernel source, edited\n", "0123456789abcdef")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.split_traffic_per_launch(100000, 500, 5) is None


def test_single_thread_oracle_sample_runs_in_a_fresh_interpreter():
    one = bench.oracle_rate_one_thread("small_4000x50", timeout=240)
    assert one is not None and one[0] > 0 and one[1] > 0
    assert bench.oracle_rate_one_thread("no_such_workload", timeout=120) is None
