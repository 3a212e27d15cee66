"""Pins of the FP64 gradient oracle (oracle/grad.py), CPU only.

* central finite differences of the objective in FP64 (the step the
  differentiation workload names, 1e-3, and a finer one) for every query
  coordinate and for s = log sigma, Gaussian and Laplacian kernels;
* the forward value at argmin assignments equals the batch objective of the
  Algorithm 2 oracle at the same centers (distances computed by the C helper,
  a separate code path);
* a query that coincides with a support row gives a finite gradient.
"""
import numpy as np
import pytest

import oracle
from oracle import grad as og
from paper_2410_05902_gb300 import inputs


def _problem(seed, m=7, d=3, k=3, sizes=(4, 1, 6)):
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(m, d))
    centers = []
    for j in range(k):
        Y = rng.normal(size=(sizes[j], d)) + j
        w = rng.uniform(0.1, 1.0, size=sizes[j])
        w = w / w.sum() * rng.uniform(0.5, 1.0)    # truncated centers: weights sum to <= 1
        centers.append((Y, w))
    assign = rng.integers(0, k, size=m)
    assign[:k] = np.arange(k)                      # every center has a row
    return Q, assign, centers


def _fd(f, x0, h):
    return (f(x0 + h) - f(x0 - h)) / (2.0 * h)


@pytest.mark.parametrize("kind", [oracle.GAUSSIAN, oracle.LAPLACIAN])
@pytest.mark.parametrize("h,tol", [(1e-3, 2e-5), (1e-5, 1e-8)])
def test_gradient_matches_central_differences(kind, h, tol):
    Q, assign, centers = _problem(11)
    s = 0.3
    L, dQ, ds = og.objective_grad(Q, assign, centers, kind, s)
    assert L == pytest.approx(og.objective(Q, assign, centers, kind, s)[0], rel=1e-15)
    scale = max(np.max(np.abs(dQ)), abs(ds))
    for i in range(Q.shape[0]):
        for c in range(Q.shape[1]):
            def f(v, i=i, c=c):
                Qp = Q.copy()
                Qp[i, c] = v
                return og.objective(Qp, assign, centers, kind, s)[0]
            assert abs(_fd(f, Q[i, c], h) - dQ[i, c]) <= tol * scale
    fs = _fd(lambda v: og.objective(Q, assign, centers, kind, v)[0], s, h)
    assert abs(fs - ds) <= tol * scale


def test_bandwidth_parameterisation():
    assert og.bandwidth_param(oracle.GAUSSIAN, 0.0) == 2.0
    assert og.bandwidth_param(oracle.GAUSSIAN, np.log(3.0)) == pytest.approx(18.0, rel=1e-15)
    assert og.bandwidth_param(oracle.LAPLACIAN, np.log(3.0)) == pytest.approx(3.0, rel=1e-15)
    with pytest.raises(ValueError):
        og.bandwidth_param(oracle.LINEAR, 0.0)


@pytest.mark.parametrize("kind", [oracle.GAUSSIAN, oracle.LAPLACIAN])
def test_forward_equals_algorithm2_batch_objective(kind):
    X, _ = inputs.isotropic_mixture(300, 4, 3, seed=5)
    X = X.astype(np.float64)
    s = float(np.log(inputs.median_sigma(X, seed=1)))
    kern = oracle.Kernel(kind, og.bandwidth_param(kind, s))
    init = inputs.init_indices(len(X), 3, seed=2)
    ora = oracle.MiniBatchKernelKMeans(X, 3, kern, 40, init, tau=30)
    for B in inputs.batch_stream(len(X), 40, 6, seed=4):
        ora.step(B)
    Q = X[inputs.batch_stream(len(X), 40, 1, seed=9)[0]]
    dist = ora.distances(Q)
    a = np.argmin(dist, axis=1)
    centers = [(X[c.idx], c.w) for c in (ora.center(j) for j in range(3))]
    L, delta = og.objective(Q, a, centers, kind, s)
    np.testing.assert_allclose(delta, dist[np.arange(len(Q)), a], rtol=1e-12, atol=1e-12)
    assert L == pytest.approx(float(np.mean(np.min(dist, axis=1))), rel=1e-12)


@pytest.mark.parametrize("kind", [oracle.GAUSSIAN, oracle.LAPLACIAN])
def test_coincident_query_gives_finite_gradient(kind):
    Q, assign, centers = _problem(3)
    Q[0] = centers[assign[0]][0][0]
    _, dQ, ds = og.objective_grad(Q, assign, centers, kind, 0.1)
    assert np.all(np.isfinite(dQ)) and np.isfinite(ds)
