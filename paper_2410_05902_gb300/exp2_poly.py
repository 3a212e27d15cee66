"""Coefficients of the FMA-pipe exp2 used by the distance-pass epilogue.

2^x = 2^j * 2^f with j = round(x) and f = x - j in [-1/2, 1/2] (Cody-Waite
range reduction). 2^f is a polynomial whose coefficients minimise the largest
relative error on [-1/2, 1/2] (a minimax fit, posed as a linear programme over
a dense grid and solved with scipy). The kernel evaluates it by Horner's rule
in FP32 FMAs and adds j to the exponent bits. Running this module prints the
FP32 coefficients that csrc/kkm_gram_tc.cu embeds; tests/test_exp2_poly.py
checks the two agree and bounds the error of the FP32 evaluation.
"""
from __future__ import annotations

import numpy as np

DEGREE = 5


def minimax(degree: int = DEGREE, points: int = 4001) -> tuple[np.ndarray, float]:
    """(c_0..c_degree in FP64, max relative error on the grid) for 2^f on [-1/2, 1/2]."""
    from scipy.optimize import linprog
    f = np.linspace(-0.5, 0.5, points)
    y = np.exp2(f)
    V = np.vander(f, degree + 1, increasing=True) / y[:, None]   # relative residual rows
    n = degree + 1
    # minimise e subject to -e <= V c - 1 <= e
    c_obj = np.zeros(n + 1)
    c_obj[-1] = 1.0
    A = np.block([[V, -np.ones((points, 1))], [-V, -np.ones((points, 1))]])
    b = np.concatenate([np.ones(points), -np.ones(points)])
    res = linprog(c_obj, A_ub=A, b_ub=b, bounds=[(None, None)] * n + [(0, None)], method="highs")
    if not res.success:
        raise RuntimeError(res.message)
    return res.x[:n], float(res.x[-1])


def fp32_coefficients(degree: int = DEGREE) -> np.ndarray:
    return minimax(degree)[0].astype(np.float32)


def _fma32(a, b, c):
    """FP32 fused multiply-add: the product of two FP32 values is exact in FP64."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def exp2_fp32(x, coeffs) -> np.ndarray:
    """The kernel's evaluation, step by step in FP32 (x is clamped to >= -127)."""
    x = np.maximum(np.asarray(x, np.float32), np.float32(-127.0))
    magic = np.float32(12582912.0)                      # 1.5 * 2^23: adding it rounds to an integer
    t = (x + magic).astype(np.float32)
    j = (t - magic).astype(np.float32)
    f = (x - j).astype(np.float32)
    c = np.asarray(coeffs, np.float32)
    p = np.full_like(f, c[-1])
    for ci in c[-2::-1]:
        p = _fma32(p, f, np.full_like(f, ci))
    e = (t.view(np.int32).astype(np.int64) << 23) & 0xFFFFFFFF      # j << 23 (two's complement)
    bits = (p.view(np.int32).astype(np.int64) + e) & 0xFFFFFFFF
    return bits.astype(np.uint32).view(np.float32)


if __name__ == "__main__":
    c, err = minimax()
    print(f"max relative error (FP64 evaluation): {err:.3e}")
    for i, v in enumerate(c.astype(np.float32)):
        print(f"c{i} = {float(v)!r}f  ({np.float32(v).view(np.uint32):#010x})")
