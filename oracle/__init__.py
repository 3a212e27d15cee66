"""FP64 CPU oracle of mini-batch kernel k-means: TEST INFRASTRUCTURE ONLY.

Only ``tests/``, the smoke check in ``__graft_entry__`` and the CPU-baseline
leg of ``bench.py`` may import, call, link or run anything in this package.
The CUDA library and its Python binding never do. The oracle and the CUDA path
share no code. The only common dependency is the seeded input generator
module, which holds none of the method's arithmetic.

Contents:
  kernels.py  kernel functions by definition (FP64; C helper gram.c)
  kkm.py      Algorithm 2 / Algorithm 1 step by step, windows rebuilt from
              the full history every iteration, no recurrences
  rng.py      SplitMix64 counter sampler for batch indices
  init.py     kernel k-means++ seeding (D^2 sampling in feature space)
  grad.py     batch objective at fixed assignments and its gradient with
              respect to the query rows and s = log sigma

Every function is pinned by the ``-m "not gpu"`` tests in
tests/test_oracle_*.py against closed forms, special cases that reduce to
textbook algorithms, invariants the paper proves, or brute force.
"""
from .kernels import GAUSSIAN, LAPLACIAN, LINEAR, POLY, Kernel, kernel_diag, kernel_matrix, kernel_wsum
from .kkm import (CenterRep, MiniBatchKernelKMeans, StepRecord, combination_norm2,
                  distance_to_combination, state_distances)
from .rng import batch_indices, index_below, splitmix64
from .init import kmeanspp
from . import grad

__all__ = [
    "GAUSSIAN", "LAPLACIAN", "LINEAR", "POLY", "Kernel", "kernel_diag", "kernel_matrix",
    "kernel_wsum", "CenterRep", "combination_norm2", "distance_to_combination", "state_distances", "MiniBatchKernelKMeans", "StepRecord", "batch_indices",
    "index_below", "splitmix64", "kmeanspp", "grad",
]
