"""Counter-based batch sampler of the oracle (test infrastructure only).

Algorithms 1 and 2 sample b elements uniformly at random, with repetitions.
Both the oracle and the CUDA library draw them from SplitMix64, implemented
separately on each side from its published definition (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014):

    state_c = seed + (c + 1) * 0x9E3779B97F4A7C15         (mod 2^64)
    z = state_c
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9             (mod 2^64)
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB             (mod 2^64)
    out_c = z ^ (z >> 31)

The c-th output (0-based) of the sequential generator seeded with ``seed`` is
therefore a pure function of (seed, c). A 64-bit output h becomes an index in
[0, n) by Lemire's multiply-high reduction, floor(h * n / 2^64).

Iteration i (1-based) of a run with batch size b uses counters
(i - 1) * b ... (i - 1) * b + b - 1, in slot order.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, counter: int) -> int:
    """Output number ``counter`` (0-based) of SplitMix64 seeded with ``seed``."""
    z = (seed + (counter + 1) * GOLDEN_GAMMA) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def index_below(h: int, n: int) -> int:
    """Lemire's multiply-high map of a 64-bit value onto [0, n)."""
    return (h * n) >> 64


def batch_indices(seed: int, iteration: int, b: int, n: int) -> np.ndarray:
    """Batch of iteration ``iteration`` (1-based): b indices in [0, n), with repetition."""
    if iteration < 1:
        raise ValueError("iterations are numbered from 1")
    base = (iteration - 1) * b
    return np.array([index_below(splitmix64(seed, base + s), n) for s in range(b)],
                    dtype=np.int64)
