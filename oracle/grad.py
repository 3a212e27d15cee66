"""FP64 oracle of the batch objective with fixed assignments, and its gradient
(test infrastructure only).

The objective is the mini-batch objective of Sec. 3 (f_A(C), a mean of
feature-space distances) evaluated at given assignments:

    L(Q, s) = (1/m) sum_x Delta(x, C_{a(x)}),
    Delta(x, C) = K(x,x) - 2 sum_t w_t K(x, y_t) + sum_{t,u} w_t w_u K(y_t, y_u),

with the assignments a(x), the support rows y_t of every center and their
weights w_t held fixed. The bandwidth is parameterised by s = log sigma:
the Gaussian kernel exp(-||x-y||^2 / kappa) has kappa = 2 sigma^2 = 2 e^{2s},
the Laplacian exp(-||x-y|| / sigma) has sigma = e^s. Both kernels have
K(x,x) = 1, so the first term carries no gradient. The support rows are
constants even where they coincide with query rows, so the query gradient
flows only through the cross term:

    dDelta/dx = -2 sum_t w_t dK(x, y_t)/dx
        Gaussian:   dK/dx = -(2/kappa) K (x - y)
        Laplacian:  dK/dx = -(K/sigma) (x - y)/||x - y||   (0 where x = y)
    dDelta/ds = -2 sum_t w_t dK(x, y_t)/ds + sum_{t,u} w_t w_u dK(y_t, y_u)/ds
        Gaussian:   dK/ds = K * D^2 * 2/kappa      (dkappa/ds = 2 kappa)
        Laplacian:  dK/ds = K * D / sigma           (dsigma/ds = sigma)

Everything is computed from these definitions with direct differences
x - y in FP64; nothing here comes from the CUDA path. The gradient is
pinned in the tests by central finite differences of ``objective``.
"""
from __future__ import annotations

import numpy as np

from .kernels import GAUSSIAN, LAPLACIAN

__all__ = ["bandwidth_param", "objective", "objective_grad", "pair_terms"]


def bandwidth_param(kind: int, s: float) -> float:
    """The kernel parameter at s = log sigma: kappa = 2 e^{2s} or sigma = e^s."""
    if kind == GAUSSIAN:
        return 2.0 * np.exp(2.0 * s)
    if kind == LAPLACIAN:
        return float(np.exp(s))
    raise ValueError("the bandwidth objective is defined for the Gaussian and Laplacian kernels")


def pair_terms(A, B, kind: int, s: float):
    """For every pair of rows (a, b): K, dK/ds and the coefficient g with
    dK/da = -g * K * (a - b), all FP64, shape (len(A), len(B))."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    diff = A[:, None, :] - B[None, :, :]
    d2 = np.einsum("ijk,ijk->ij", diff, diff)
    p = bandwidth_param(kind, s)
    if kind == GAUSSIAN:
        K = np.exp(-d2 / p)
        dks = K * d2 * (2.0 / p)
        g = np.full_like(d2, 2.0 / p)
    else:
        D = np.sqrt(d2)
        K = np.exp(-D / p)
        dks = K * D / p
        with np.errstate(divide="ignore"):
            g = np.where(D > 0.0, 1.0 / (p * np.where(D > 0.0, D, 1.0)), 0.0)
    return K, dks, g


def _center_terms(Y, w, kind, s):
    K, dks, _ = pair_terms(Y, Y, kind, s)
    return float(w @ K @ w), float(w @ dks @ w)


def objective(Q, assign, centers, kind: int, s: float):
    """(L, Delta per row). ``centers[j] = (Y_j, w_j)``: support rows and weights."""
    Q = np.asarray(Q, dtype=np.float64)
    assign = np.asarray(assign)
    delta = np.empty(len(Q), dtype=np.float64)
    for j, (Y, w) in enumerate(centers):
        rows = np.nonzero(assign == j)[0]
        if len(rows) == 0:
            continue
        Y = np.asarray(Y, dtype=np.float64)
        w = np.asarray(w, dtype=np.float64)
        n2, _ = _center_terms(Y, w, kind, s)
        K, _, _ = pair_terms(Q[rows], Y, kind, s)
        delta[rows] = 1.0 - 2.0 * (K @ w) + n2
    return float(delta.mean()), delta


def objective_grad(Q, assign, centers, kind: int, s: float):
    """(L, dL/dQ, dL/ds) by the formulas in the module docstring."""
    Q = np.asarray(Q, dtype=np.float64)
    assign = np.asarray(assign)
    m = len(Q)
    delta = np.empty(m, dtype=np.float64)
    dQ = np.zeros_like(Q)
    ds = 0.0
    for j, (Y, w) in enumerate(centers):
        rows = np.nonzero(assign == j)[0]
        if len(rows) == 0:
            continue
        Y = np.asarray(Y, dtype=np.float64)
        w = np.asarray(w, dtype=np.float64)
        n2, dn2 = _center_terms(Y, w, kind, s)
        K, dks, g = pair_terms(Q[rows], Y, kind, s)
        delta[rows] = 1.0 - 2.0 * (K @ w) + n2
        # dDelta/dx = -2 sum_t w_t (-g K (x - y_t)) = 2 sum_t c_t (x - y_t), c = w g K
        c = K * g * w[None, :]
        dQ[rows] = 2.0 * (Q[rows] * c.sum(axis=1)[:, None] - c @ Y) / m
        ds += float((-2.0 * (dks @ w) + dn2).sum()) / m
    return float(delta.mean()), dQ, ds
