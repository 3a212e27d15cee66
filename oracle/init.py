"""Kernel k-means++ seeding in the oracle (test infrastructure only).

Secs. 1 and 5 initialise the centers with k-means++ (Arthur and Vassilvitskii,
2007), run in feature space, so every initial center is a single data point.
The paper does not spell the procedure out. This is the standard D^2 sampling:

1. The first center is uniform over X.
2. Each later center is x with probability proportional to
   D(x)^2 = min over chosen c of Delta(x, c), where
   Delta(x, c) = K(x,x) - 2 K(x,c) + K(c,c).

The uniform variates are u_t = (h_t >> 11) * 2^-53. Here h_t is output t of
SplitMix64 seeded with ``seed`` (see rng.py). A draw picks the first x whose
running sum of D^2 exceeds u * total.
"""
from __future__ import annotations

import numpy as np

from .kernels import Kernel, kernel_diag, kernel_matrix
from .rng import index_below, splitmix64


def uniform01(seed: int, counter: int) -> float:
    return (splitmix64(seed, counter) >> 11) * (1.0 / (1 << 53))


def kmeanspp(X, k: int, kernel: Kernel, seed: int) -> np.ndarray:
    """k data indices chosen by D^2 sampling in feature space."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = X.shape[0]
    if not 1 <= k <= n:
        raise ValueError("need 1 <= k <= n")
    chosen = [index_below(splitmix64(seed, 0), n)]
    kxx = kernel_diag(X, kernel)

    def delta_to(c):
        kcc = kernel_diag(X[c], kernel)[0]
        return np.maximum(kxx - 2.0 * kernel_matrix(X, X[c], kernel)[:, 0] + kcc, 0.0)

    d2 = delta_to(chosen[0])
    for t in range(1, k):
        total = float(np.sum(d2))
        if total <= 0.0:
            # every point coincides with a chosen one: fall back to uniform picks
            c = index_below(splitmix64(seed, t), n)
        else:
            target = uniform01(seed, t) * total
            c = int(np.searchsorted(np.cumsum(d2), target, side="right"))
            c = min(c, n - 1)
        chosen.append(c)
        d2 = np.minimum(d2, delta_to(c))
    return np.array(chosen, dtype=np.int64)
