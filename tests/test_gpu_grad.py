"""Parity of the objective at fixed assignments and its adjoint (kkm_objective_fwd /
kkm_objective_bwd, through the C-ABI and the autograd binding) with the FP64
oracle of oracle/grad.py, whose gradient is pinned by finite differences.

The centers are whatever the GPU run holds after some iterations; the oracle
evaluates the same centers (support indices and FP64 weights from
kkm_get_state, rows from X) in FP64.
"""
import numpy as np
import pytest

import oracle
from oracle import grad as og
from paper_2410_05902_gb300 import inputs

from gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu

KIND = {"gaussian": oracle.GAUSSIAN, "laplacian": oracle.LAPLACIAN}
# FP32 pair sums over a few hundred support rows: 1e-5 on the objective,
# 1e-4 normwise on the query gradient and on d/ds (relative to the size of
# its two terms, which cancel in part).
LOSS_TOL, GRAD_TOL = 1e-5, 1e-4


def _centers(state, X):
    out, o = [], 0
    for r in state["rows_per_center"]:
        idx = np.asarray(state["row_idx"][o:o + r], np.int64)
        out.append((X[idx].astype(np.float64), np.asarray(state["row_w"][o:o + r], np.float64)))
        o += r
    return out


def _run(X, k, b, tau, kernel, precision, iters, seed=3):
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KKM
    sigma = inputs.median_sigma(X, seed=1)
    param = 2 * sigma * sigma if kernel == "gaussian" else sigma
    Xd = torch.from_numpy(X).cuda()
    run = KKM(Xd, k, b, kernel=kernel, param=param, tau=tau, precision=precision,
              init_idx=inputs.init_indices(len(X), k, seed=seed))
    for B in inputs.batch_stream(len(X), b, iters, seed=seed + 1):
        run.step(torch.from_numpy(B.astype(np.int32)).cuda())
    run.sync()
    return run, Xd, float(np.log(sigma))


def _ds_scale(Q, assign, centers, kind, s):
    """Size of the two terms of dL/ds (the cross term and the center-norm term)."""
    tot = 0.0
    for j, (Y, w) in enumerate(centers):
        rows = np.nonzero(assign == j)[0]
        if len(rows) == 0:
            continue
        _, dks, _ = og.pair_terms(Q[rows], Y, kind, s)
        _, dkc, _ = og.pair_terms(Y, Y, kind, s)
        tot += 2.0 * float(np.abs(dks @ w).sum()) + len(rows) * float(abs(w @ dkc @ w))
    return tot / len(Q)


def _check(run, Xd, X, kernel, s, batch, assign):
    torch = torch_cuda()
    kind = KIND[kernel]
    Q = Xd[torch.from_numpy(batch.astype(np.int64)).cuda()].contiguous()
    a = torch.from_numpy(assign.astype(np.int32)).cuda()
    centers = _centers(run.get_state(), X)
    Q64 = X[batch].astype(np.float64)
    L, dQ, ds = og.objective_grad(Q64, assign, centers, kind, s)
    loss, delta = run.objective_fwd(Q, a, s, want_delta=True)
    g = torch.ones(1, dtype=torch.float64, device="cuda")
    gq, gs = run.objective_bwd(Q, a, s, g)
    run.sync()
    _, delta_ref = og.objective(Q64, assign, centers, kind, s)
    assert abs(float(loss.cpu()[0]) - L) <= LOSS_TOL * abs(L)
    assert np.max(np.abs(delta.cpu().numpy() - delta_ref)) <= LOSS_TOL * max(1.0, np.max(np.abs(delta_ref)))
    gq = gq.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gq - dQ)) <= GRAD_TOL * np.max(np.abs(dQ))
    assert abs(float(gs.cpu()[0]) - ds) <= GRAD_TOL * _ds_scale(Q64, assign, centers, kind, s)
    return Q, a, L, dQ, ds


@pytest.mark.parametrize("kernel", ["gaussian", "laplacian"])
@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_objective_and_adjoint_small(kernel, precision):
    X, _ = inputs.isotropic_mixture(800, 16, 6, seed=2)
    run, Xd, s = _run(X, 6, 128, 60, kernel, precision, 8)
    batch = inputs.batch_stream(len(X), 200, 1, seed=42)[0]
    rng = np.random.default_rng(7)
    for assign in (rng.integers(0, 6, size=200),                       # arbitrary fixed assignments
                   run.assign(Xd[batch.astype(np.int64)])[0].cpu().numpy()):   # the argmin ones
        _check(run, Xd, X, kernel, s + 0.2, batch, np.asarray(assign))
    run.close()


def test_objective_wide_rows_and_long_windows():
    """d = 150 (several feature chunks in the pair and row kernels, ragged last
    chunk), windows of more than 256 rows (several slabs of the row kernel), a
    ragged batch of 333 rows, and arbitrary assignments that leave a center
    without rows."""
    X, _ = inputs.isotropic_mixture(3000, 150, 3, seed=6)
    run, Xd, s = _run(X, 3, 300, 400, "gaussian", "fp32", 6)
    assert max(run.get_state()["rows_per_center"]) > 256
    batch = inputs.batch_stream(len(X), 333, 1, seed=9)[0]
    rng = np.random.default_rng(5)
    for assign in (rng.integers(0, 2, size=333),
                   run.assign(Xd[batch.astype(np.int64)])[0].cpu().numpy()):
        _check(run, Xd, X, "gaussian", s, batch, np.asarray(assign))
    run.close()


def test_autograd_matches_the_adjoint():
    torch = torch_cuda()
    from paper_2410_05902_gb300.autograd import objective
    X, _ = inputs.isotropic_mixture(600, 8, 4, seed=4)
    run, Xd, s = _run(X, 4, 96, 40, "gaussian", "fp32", 5)
    batch = inputs.batch_stream(len(X), 64, 1, seed=5)[0]
    Q = Xd[torch.from_numpy(batch.astype(np.int64)).cuda()].clone().requires_grad_(True)
    a = run.assign(Q.detach())[0]
    ls = torch.tensor(s, dtype=torch.float64, device="cuda", requires_grad=True)
    L = objective(run, Q, ls, a)
    (3.0 * L).backward()
    g3 = torch.full((1,), 3.0, dtype=torch.float64, device="cuda")
    gq, gs = run.objective_bwd(Q.detach(), a, s, g3)
    run.sync()
    assert torch.equal(Q.grad, gq)
    assert float(ls.grad) == float(gs.cpu()[0])
    ref, _ = run.objective_fwd(Q.detach(), a, s)
    assert float(L.detach()) == float(ref.cpu()[0])


def test_differentiation_workload_full_size():
    """n=2e5, d=64, 50 components, k=50, b=2048, tau=200, Gaussian: 50 warm-up
    iterations, then the objective and its adjoint at the argmin assignments
    against the FP64 oracle, plus oracle central differences (step 1e-3) on 64
    random query coordinates and on log sigma."""
    w = inputs.WORKLOADS["differentiation"]
    X, _ = w.make()
    run, Xd, s = _run(X, w.k, w.b, w.tau, "gaussian", "fp32", 50)
    batch = inputs.batch_stream(w.n, w.b, 1, seed=77)[0]
    assign = run.assign(Xd[batch.astype(np.int64)])[0].cpu().numpy()
    Q, a, L, dQ, ds = _check(run, Xd, X, "gaussian", s, batch, assign)
    centers = _centers(run.get_state(), X)
    Q64 = X[batch].astype(np.float64)
    rng = np.random.default_rng(11)
    h = 1e-3
    scale = np.max(np.abs(dQ))
    for _ in range(64):
        i, c = int(rng.integers(0, w.b)), int(rng.integers(0, w.d))
        # only row i's Delta depends on Q[i, c]: L = (1/m) sum_x Delta_x
        qp, qm = Q64[i:i + 1].copy(), Q64[i:i + 1].copy()
        qp[0, c] += h
        qm[0, c] -= h
        ai = assign[i:i + 1]
        fd = (og.objective(qp, ai, centers, oracle.GAUSSIAN, s)[0]
              - og.objective(qm, ai, centers, oracle.GAUSSIAN, s)[0]) / (2 * h * w.b)
        assert abs(fd - dQ[i, c]) <= 1e-3 * scale
    fs = (og.objective(Q64, assign, centers, oracle.GAUSSIAN, s + h)[0]
          - og.objective(Q64, assign, centers, oracle.GAUSSIAN, s - h)[0]) / (2 * h)
    assert abs(fs - ds) <= 1e-3 * _ds_scale(Q64, assign, centers, oracle.GAUSSIAN, s)
    run.close()
