"""Parity bars shared by the GPU solve tests.

A backward-stable method cannot beat u sigma_1 / sigma_min in relative sigma error nor
u / gap_abs in angle (Sec. 4 of arXiv 2602.16797), so the literal bars (1e-10 relative in sigma,
1e-8 in subspace angle) are applied wherever those floors allow and the floors (with a constant
c = 10 sqrt(n)) elsewhere:
  sigma:  |sigma_gpu - sigma_oracle| <= max(1e-10 sigma_oracle, c u Sigma~(1,1))
  angle:  sin angle(V_gpu, V_oracle) <= max(1e-8, c u / gap_abs^(k)),
          gap_abs^(k) = (sigma_{n-k} - sigma_{n-k+1}) / sigma_1
  truth:  |sigma_gpu - sigma_true| <= max(1e-10 sigma_true, 4 |sigma_oracle - sigma_true|, c u Sigma~(1,1))
"""
import numpy as np

U = 2.0 ** -53


def sub_sin(V1, V2):
    Q1, _ = np.linalg.qr(V1)
    Q2, _ = np.linalg.qr(V2)
    return float(np.linalg.norm(Q1 - Q2 @ (Q2.conj().T @ Q1), 2))


def c_of(n):
    return 10.0 * np.sqrt(n)


def check_sigma(sig_gpu, sig_ora, sigma11, n):
    bar = np.maximum(1e-10 * np.abs(sig_ora), c_of(n) * U * sigma11)
    diff = np.abs(np.asarray(sig_gpu) - np.asarray(sig_ora))
    assert np.all(diff <= bar), (diff, bar)


def check_truth(sig_gpu, sig_ora, sig_true, sigma11, n):
    e_g = np.abs(np.asarray(sig_gpu) - sig_true)
    e_o = np.abs(np.asarray(sig_ora) - sig_true)
    bar = np.maximum.reduce([1e-10 * sig_true, 4 * e_o, np.full_like(e_g, c_of(n) * U * sigma11)])
    assert np.all(e_g <= bar), (e_g, bar)


def check_angle(V_gpu, V_ora, gap_abs, n):
    bar = max(1e-8, c_of(n) * U / gap_abs)
    s = sub_sin(V_gpu, V_ora)
    assert s <= bar, (s, bar)
    return s
