"""The full-batch baseline (kernel Lloyd, kkm_lloyd_*) against the oracle.

Kernel Lloyd is Algorithm 1 with the identity batch and alpha = 1; the
oracle pins its equality with textbook Lloyd for the linear kernel. Three
levels of checks:
- the whole trajectory against the oracle's own kernel Lloyd (small n);
- teacher-forced, every iteration: the oracle computes Delta(x, C_j) for the
  centers that the GPU run's previous assignment defines (means of the
  assigned points in feature space, Eq. (1) with weights 1/n_j), so one
  near-tie cannot make the two runs part; every precision form, Gaussian and
  Laplacian kernels, with several Gram-pass chunks and a ragged last chunk;
- at the 70000 x 784 image workload's size, sampled rows: the oracle's cross
  term <phi(x), C_j> for 16 rows against all 70000 support rows.
"""
import numpy as np
import pytest

import oracle
from paper_2410_05902_gb300 import inputs

from gpu_helpers import CN_RTOL, DIST_TOL, OBJ_TOL_FORM, KIND, torch_cuda

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


def _state_from(assign, k, prev):
    """Centers as weighted rows: the means of the assigned rows; a center
    without rows keeps its previous rows and weights."""
    cols = []
    for j in range(k):
        rows = np.nonzero(assign == j)[0]
        cols.append((rows, np.full(len(rows), 1.0 / len(rows))) if len(rows) else prev[j])
    state = {"row_idx": np.concatenate([c[0] for c in cols]).astype(np.int64),
             "row_w": np.concatenate([c[1] for c in cols]),
             "rows_per_center": np.array([len(c[0]) for c in cols], np.int64)}
    return state, cols


def _compare(D, a, fx, cn, D_ora, cn_ora, form, what):
    scale = float(np.max(np.abs(D_ora)))
    err = float(np.max(np.abs(D - D_ora))) / scale
    assert err <= DIST_TOL[form], f"{what}: normwise distance error {err:.3e}"
    order = np.sort(D_ora, axis=1)
    bad = np.nonzero(a != D_ora.argmin(axis=1))[0]
    assert np.all(order[bad, 1] - order[bad, 0] <= 2 * DIST_TOL[form] * scale), f"{what}: assignments"
    f_ora = float(np.mean(D_ora.min(axis=1)))
    assert abs(fx - f_ora) <= OBJ_TOL_FORM[form] * abs(f_ora), f"{what}: f_X {fx} vs {f_ora}"
    np.testing.assert_allclose(cn, cn_ora, rtol=CN_RTOL[form], atol=CN_RTOL[form], err_msg=what)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32", "bf16"])
@pytest.mark.parametrize("kernel", ["gaussian", "laplacian"])
def test_lloyd_teacher_forced_every_iteration(precision, kernel):
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import Lloyd
    n, d, k = 3000, 24, 8
    X, _ = inputs.isotropic_mixture(n, d, k, seed=21)
    sigma = inputs.median_sigma(X, seed=1)
    param = 2 * sigma * sigma if kernel == "gaussian" else sigma
    kern = oracle.Kernel(KIND[kernel], param)
    X64 = X.astype(np.float64)
    init = inputs.init_indices(n, k, seed=6)
    run = Lloyd(torch.from_numpy(X).cuda(), k, init, kernel=kernel, param=param, precision=precision,
                chunk_rows=1024)
    _, chunks, rows = run.info()
    assert (chunks, rows) == (3, 1024)          # 1024 + 1024 + a ragged 952
    cols = [(np.array([i]), np.array([1.0])) for i in init]
    state = {"row_idx": np.asarray(init, np.int64), "row_w": np.ones(k), "rows_per_center": np.ones(k, np.int64)}
    prev_fx = None
    for it in range(5):
        fx, changed, done = run.read()
        assert done == it
        D = run.distances().cpu().numpy().astype(np.float64)
        a = run.assignments()[0].cpu().numpy()
        cn = run.center_norms()
        D_ora, cn_ora = oracle.state_distances(X64, X64, state, kern)
        _compare(D, a, fx, cn, D_ora, cn_ora, precision, f"{precision} {kernel} iteration {it}")
        if it == 0:
            assert changed == n
        if prev_fx is not None and precision in ("fp32", "bf16x3"):
            assert fx <= prev_fx * (1 + 1e-6)       # Lloyd never increases f_X
        prev_fx = fx
        state, cols = _state_from(a, k, cols)
        run.iterate(1)
    run.close()


def test_lloyd_stops_at_its_fixed_point():
    torch = torch_cuda()
    from paper_2410_05902_gb300.quality import full_batch
    X, labels = inputs.isotropic_mixture(2000, 16, 5, seed=31)
    sigma = inputs.median_sigma(X, seed=1)
    init = inputs.init_indices(len(X), 5, seed=2)
    trace = []
    assign, fx, done, _ = full_batch(torch.from_numpy(X).cuda(), 5, "gaussian", 2 * sigma * sigma, init, 100,
                                     precision="fp32", trace=trace)
    assert done < 100
    assert len(trace) == done + 1
    fxs = [t[2] for t in trace]
    assert all(b <= a * (1 + 1e-6) for a, b in zip(fxs, fxs[1:]))
    assert fx == fxs[-1]


@pytest.mark.parametrize("precision", ["bf16x3", "bf16"])
def test_lloyd_image_workload_sampled_rows(precision):
    """70000 x 784, k = 10: one Gram pass of 70000 x 70000 per iteration."""
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import Lloyd
    X, _ = inputs.image_like(70000, seed=3)
    n, k = X.shape[0], 10
    sigma = inputs.median_sigma(X, seed=1)
    param = 2 * sigma * sigma
    kern = oracle.Kernel(oracle.GAUSSIAN, param)
    init = inputs.init_indices(n, k, seed=4)
    run = Lloyd(torch.from_numpy(X).cuda(), k, init, kernel="gaussian", param=param, precision=precision)
    fx0, _, _ = run.read()                      # f_X at the initial points
    a0 = run.assignments()[0].cpu().numpy()
    run.iterate(1)
    fx1, _, _ = run.read()
    D = run.distances().cpu().numpy().astype(np.float64)
    cn = run.center_norms()
    rng = np.random.default_rng(9)
    sample = rng.choice(n, size=16, replace=False)
    Xs = X[sample].astype(np.float64)
    X64 = X.astype(np.float64)
    # <phi(x), C_j> from the GPU's distances and norms (K(x, x) = 1), against the
    # oracle's for C_j = the mean of the rows a0 assigns to j
    cross_gpu = 0.5 * (1.0 + cn[None, :] - D[sample])
    cross_ora = np.empty((16, k))
    for j in range(k):
        rows = np.nonzero(a0 == j)[0]
        assert len(rows) > 0
        cross_ora[:, j] = oracle.kernel_wsum(Xs, X64[rows], np.full(len(rows), 1.0 / len(rows)), kern)
    err = float(np.max(np.abs(cross_gpu - cross_ora))) / float(np.max(np.abs(cross_ora)))
    assert err <= DIST_TOL[precision], f"cross-term error {err:.3e}"
    # f_X is the mean of the row minima, and a Lloyd iteration does not increase it
    assert abs(fx1 - float(np.mean(np.min(D, axis=1)))) <= 1e-5 * abs(fx1)
    assert fx1 <= fx0 * (1 + 1e-4)
    run.iterate(1)
    fx2, _, _ = run.read()
    assert fx2 <= fx1 * (1 + 1e-4)
    run.close()
