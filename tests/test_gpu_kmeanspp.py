"""GPU kernel k-means++ (kkm_kmeanspp) against the oracle's D^2 sampling
(oracle/init.py): both draw from the same SplitMix64 stream and evaluate D^2
in FP64, so the chosen indices must be identical."""
import numpy as np
import pytest

import oracle
from paper_2410_05902_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kernel,n,d,k,seed", [
    ("gaussian", 2000, 16, 10, 1),
    ("laplacian", 3000, 8, 12, 2),
    ("linear", 1500, 5, 7, 3),
    ("poly", 800, 4, 6, 4),
    ("gaussian", 20000, 64, 30, 5),
    ("gaussian", 5, 3, 5, 6),          # k = n: every point is chosen once
])
def test_kmeanspp_matches_oracle(kernel, n, d, k, seed):
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KERNELS, kmeanspp
    X, _ = inputs.isotropic_mixture(n, d, max(2, k // 2), seed=100 + seed)
    sigma = inputs.median_sigma(X, seed=1)
    param = {"gaussian": 2 * sigma * sigma, "laplacian": sigma}.get(kernel, 1.0)
    kind = {"gaussian": oracle.GAUSSIAN, "laplacian": oracle.LAPLACIAN, "linear": oracle.LINEAR,
            "poly": oracle.POLY}[kernel]
    ref = oracle.kmeanspp(X.astype(np.float64), k, oracle.Kernel(kind, param, 1.0, 2), seed=seed)
    got = kmeanspp(torch.from_numpy(X).cuda(), k, kernel, param, coef0=1.0, degree=2, seed=seed)
    np.testing.assert_array_equal(got, ref)


def test_kmeanspp_duplicate_points_fall_back_to_uniform():
    """All points equal: D^2 is 0 after the first draw, so later draws are uniform."""
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import kmeanspp
    X = np.ones((50, 4), np.float32)
    ref = oracle.kmeanspp(X.astype(np.float64), 5, oracle.Kernel(oracle.GAUSSIAN, 1.0), seed=9)
    got = kmeanspp(torch.from_numpy(X).cuda(), 5, "gaussian", 1.0, seed=9)
    np.testing.assert_array_equal(got, ref)


def test_run_seeded_with_kmeanspp():
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KKM
    X, _ = inputs.isotropic_mixture(1000, 8, 5, seed=7)
    sigma = inputs.median_sigma(X, seed=1)
    run = KKM(torch.from_numpy(X).cuda(), 5, 64, param=2 * sigma * sigma, tau=30, init_idx="kmeans++", seed=11)
    st = run.get_state()
    ref = oracle.kmeanspp(X.astype(np.float64), 5, oracle.Kernel(oracle.GAUSSIAN, 2 * sigma * sigma), seed=11)
    np.testing.assert_array_equal(st["row_idx"], ref)
    run.close()
