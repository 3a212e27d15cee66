"""Clustering quality and the full-batch baseline the paper compares against.

``full_batch`` runs full-batch kernel k-means (kernel Lloyd: every iteration
assigns all n points, then every center becomes the mean of its points in
feature space) through the library's kkm_lloyd_* entry points: the n x n
Gram pass of X against X sorted by center, on the same distance kernels as
the mini-batch run. A cluster that gets no points keeps its center.

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
               coef0: float = 0.0, degree: int = 2, stop_when_stable: bool = True, chunk_rows: int = 0,
               trace: list | None = None):
    """Full-batch kernel k-means on the GPU (see the module docstring).

    Returns (assignments at the final centers, f_X at them, iterations run,
    seconds of the loop on the host clock). With stop_when_stable the loop
    ends after the first iteration that changes no assignment (Lloyd's fixed
    point). With a list as ``trace``, appends (iterations, seconds since the
    loop started, f_X) after the initial assignment and after every iteration.
    """
    import torch
    from .kkm import Lloyd
    run = Lloyd(X, k, np.asarray(init_idx, np.int64), kernel=kernel, param=param, coef0=coef0, degree=degree,
                precision=precision, chunk_rows=chunk_rows)
    done = 0
    t0 = time.perf_counter()
    fx, _, _ = run.read()
    if trace is not None:
        trace.append((0, 0.0, fx))
    for _ in range(iters):
        run.iterate(1)
        fx, changed, done = run.read()
        if trace is not None:
            trace.append((done, time.perf_counter() - t0, fx))
        if stop_when_stable and changed == 0:
            break
    seconds = time.perf_counter() - t0
    assign = run.assignments()[0].cpu().numpy()
    torch.cuda.synchronize()
    run.close()
    return assign, fx, done, seconds
