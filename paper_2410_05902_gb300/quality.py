"""Clustering quality and the full-batch baseline the paper compares against.

``full_batch`` runs full-batch kernel k-means (kernel Lloyd: every iteration
assigns all n points, then every center becomes the mean of its points in
feature space) on the library's own kernels. It is the windowed run with the
batch equal to X in order (b = n), the constant rate eta = 1 and tau = 1:
with alpha = 1 a center's older blocks carry weight 0, and tau = 1 keeps
only the newest block, the cluster mean. A cluster that gets no points keeps
its center (alpha = 0). Limited to n <= 8192, the library's batch bound.

``adjusted_rand`` and ``normalized_mutual_info`` are the usual external
indices against the latent labels of the synthetic generators (ARI of Hubert
and Arabie 1985; NMI with the arithmetic-mean normaliser).
"""
from __future__ import annotations

import time

import numpy as np


def _contingency(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    m = np.zeros((ai.max() + 1, bi.max() + 1), dtype=np.int64)
    np.add.at(m, (ai, bi), 1)
    return m


def adjusted_rand(labels_true, labels_pred) -> float:
    """Adjusted Rand index: (index - expected) / (max - expected) over pairs."""
    m = _contingency(labels_true, labels_pred)
    n = m.sum()
    comb2 = lambda v: v * (v - 1) / 2.0
    idx = comb2(m).sum()
    a = comb2(m.sum(axis=1)).sum()
    b = comb2(m.sum(axis=0)).sum()
    expected = a * b / comb2(n) if n > 1 else 0.0
    top = 0.5 * (a + b)
    if top == expected:
        return 1.0
    return float((idx - expected) / (top - expected))


def normalized_mutual_info(labels_true, labels_pred) -> float:
    """I(U; V) / ((H(U) + H(V)) / 2), natural logarithms."""
    m = _contingency(labels_true, labels_pred).astype(np.float64)
    n = m.sum()
    pu = m.sum(axis=1) / n
    pv = m.sum(axis=0) / n
    nz = m > 0
    pij = m[nz] / n
    mi = float((pij * np.log(pij / (pu[:, None] * pv[None, :])[nz])).sum())
    hu = float(-(pu[pu > 0] * np.log(pu[pu > 0])).sum())
    hv = float(-(pv[pv > 0] * np.log(pv[pv > 0])).sum())
    if hu + hv == 0.0:
        return 1.0
    return max(0.0, mi / (0.5 * (hu + hv)))


def full_batch(X, k: int, kernel: str, param: float, init_idx, iters: int, precision: str = "fp32",
               coef0: float = 0.0, degree: int = 2, stop_when_stable: bool = True):
    """Full-batch kernel k-means on the GPU (see the module docstring).

    Returns (assignments of the last iteration, f_X after it, iterations run,
    seconds on the device). With stop_when_stable the loop ends once an
    iteration leaves every assignment unchanged (Lloyd's fixed point).
    """
    import torch
    from .kkm import KKM
    n = X.shape[0]
    if n > 8192:
        raise ValueError("full_batch needs n <= 8192 (one batch holds all of X)")
    run = KKM(X, k, n, kernel=kernel, param=param, coef0=coef0, degree=degree, tau=1, lr="const", eta=1.0,
              precision=precision, init_idx=init_idx)
    idx = torch.arange(n, dtype=torch.int32, device=X.device)
    a = torch.empty(n, dtype=torch.int32, device=X.device)
    prev = None
    done = 0
    run.sync()
    t0 = time.perf_counter()
    for _ in range(iters):
        run.step(idx, None, a)
        done += 1
        if stop_when_stable:
            cur = a.clone()
            if prev is not None and torch.equal(cur, prev):
                break
            prev = cur
    run.sync()
    seconds = time.perf_counter() - t0
    assign = run.assign(X)[0].cpu().numpy()
    fx = run.objective()
    run.close()
    return assign, fx, done, seconds
