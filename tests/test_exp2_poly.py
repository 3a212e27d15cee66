"""The FMA-pipe exp2 of the distance-pass epilogue (CPU only).

* its coefficients in csrc/kkm_gram_tc.cu are the FP32 roundings of the
  minimax fit that paper_2410_05902_gb300/exp2_poly.py computes;
* the kernel's evaluation, emulated step by step in FP32, stays within
  2.5e-7 relative error of 2^x on the range the epilogue feeds it, about the
  accuracy of the MUFU's ex2.approx it stands in for;
* the clamp at -127 gives a non-negative value no larger than 2^-126.
"""
import os
import re

import numpy as np
import pytest

from paper_2410_05902_gb300 import exp2_poly as ep

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CU = os.path.join(ROOT, "paper_2410_05902_gb300", "csrc", "kkm_gram_tc.cu")


def kernel_coefficients():
    src = open(CU).read()
    body = src[src.index("exp2_fma2"):]
    vals = {}
    for name, v in re.findall(r"\b(C[0-5]) = ([0-9.eE+-]+)f", body[:2000]):
        vals.setdefault(name, float(v))
    return np.array([vals[f"C{i}"] for i in range(6)], dtype=np.float32)


def test_kernel_constants_are_the_minimax_fit():
    pytest.importorskip("scipy")
    c64, err = ep.minimax()
    assert err < 1e-7
    np.testing.assert_array_equal(kernel_coefficients(), c64.astype(np.float32))


def test_fp32_evaluation_error():
    c = kernel_coefficients()
    x = np.concatenate([np.linspace(-125.0, 1.0, 1_000_001), -np.logspace(-8, 0, 2001), [0.0, -0.5, 0.5]])
    x = x.astype(np.float32)
    y = ep.exp2_fp32(x, c).astype(np.float64)
    ref = np.exp2(x.astype(np.float64))
    rel = np.abs(y - ref) / ref
    assert rel.max() <= 2.5e-7
    assert abs(float(ep.exp2_fp32(np.float32(0.0), c)) - 1.0) <= 2e-7


def test_clamp_below():
    c = kernel_coefficients()
    for x in (-127.0, -150.0, -1e4, -np.inf):
        v = float(ep.exp2_fp32(np.float32(x), c))
        assert 0.0 <= v <= 2.0 ** -126
