"""The full-batch baseline (kernel Lloyd on the library's kernels) against the
oracle's kernel Lloyd: Algorithm 1 with the identity batch and alpha = 1, whose
equality with textbook Lloyd for the linear kernel the oracle pins."""
import numpy as np
import pytest

import oracle
from paper_2410_05902_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel", ["gaussian", "linear"])
def test_full_batch_matches_oracle_lloyd(kernel):
    torch = torch_cuda()
    from paper_2410_05902_gb300.quality import full_batch
    X, labels = inputs.isotropic_mixture(1200, 8, 6, seed=4)
    sigma = inputs.median_sigma(X, seed=1)
    param = 2 * sigma * sigma if kernel == "gaussian" else 1.0
    kind = oracle.GAUSSIAN if kernel == "gaussian" else oracle.LINEAR
    init = inputs.init_indices(len(X), 6, seed=5)
    iters = 6
    assign, fx, done, _ = full_batch(torch.from_numpy(X).cuda(), 6, kernel, param, init, iters,
                                     stop_when_stable=False)
    ora = oracle.MiniBatchKernelKMeans(X.astype(np.float64), 6, oracle.Kernel(kind, param), len(X), init,
                                       tau=None, lr="const", eta=1.0)
    for _ in range(iters):
        ora.step(np.arange(len(X)))
    ref = ora.distances(X.astype(np.float64))
    scale = float(np.max(np.abs(ref)))
    order = np.sort(ref, axis=1)
    bad = np.nonzero(assign != ref.argmin(axis=1))[0]
    assert np.all(order[bad, 1] - order[bad, 0] <= 1e-5 * scale)
    assert fx == pytest.approx(ora.objective(), rel=1e-5)
    assert done == iters
