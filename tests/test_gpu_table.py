"""The table form of Algorithm 1 (KKM_ALGO_TABLE, Appendix A) against the
untruncated FP64 oracle (Algorithm 1 with centers rebuilt from the full
history). Both sides take the same batches; the GPU is forced to the
oracle's assignments, so the trajectories stay together, and every step's
batch distances (which read the table and ||C||^2 before the update) and
f_B are compared; f_X over the whole dataset closes the run."""
import numpy as np
import pytest

import oracle
from paper_2410_05902_gb300 import inputs

from gpu_helpers import DIST_TOL, OBJ_TOL_FORM, Pair, dist_rel_err, near_tie_ok, torch_cuda

pytestmark = pytest.mark.gpu


def _run(X, k, b, iters, precision="fp32", kernel="gaussian", lr="beta", eta=None, seed=31, coef0=0.0,
         dist_tile=0):
    p = Pair(X, k=k, b=b, tau=0, precision=precision, kernel=kernel, lr=lr, eta=eta, algo="table",
             coef0=coef0, dist_tile=dist_tile)
    tol = DIST_TOL[precision]
    worst = 0.0
    for B in inputs.batch_stream(len(X), b, iters, seed=seed):
        rec = p.ora.step(B)
        d, a, f = p.gpu_step(B, forced=rec.assign)
        err = dist_rel_err(d, rec.dist)
        worst = max(worst, err)
        assert err <= tol, f"iteration {rec.iteration}: {err:.3e}"
        assert near_tie_ok(a, rec, p.abs_tol(rec))[0]
        assert abs(f - rec.batch_objective) <= OBJ_TOL_FORM[precision] * abs(rec.batch_objective) + 1e-12
    fx = p.gpu.objective()
    ref = p.ora.objective()
    assert abs(fx - ref) <= 10 * OBJ_TOL_FORM[precision] * abs(ref) + 1e-12
    return p, worst


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32", "bf16"])
def test_table_form_matches_algorithm1(precision):
    X, _ = inputs.isotropic_mixture(1500, 16, 6, seed=3)
    p, _ = _run(X, 6, 128, 12, precision)
    p.close()


@pytest.mark.parametrize("kernel,extra", [("laplacian", {}), ("linear", {}), ("poly", {"coef0": 1.0})])
def test_table_form_other_kernels(kernel, extra):
    X, _ = inputs.isotropic_mixture(800, 6, 4, seed=5)
    X = X / 4.0
    p, _ = _run(X, 4, 64, 8, "fp32", kernel=kernel, **extra)
    p.close()


def test_table_form_sklearn_rate_and_duplicates():
    X, _ = inputs.isotropic_mixture(60, 4, 3, seed=6)    # b = 50 draws from 60 points repeat
    p, _ = _run(X, 3, 50, 10, "fp32", lr="sklearn")
    p.close()


def test_table_form_wide_rows_and_tiles():
    X, _ = inputs.image_like(3000, seed=7, d=784, classes=8)
    for tile in (64, 256):
        p, _ = _run(X, 8, 512, 4, "bf16x3", dist_tile=tile, seed=40 + tile)
        p.close()


def test_table_form_rejects_window_calls():
    torch = torch_cuda()
    from paper_2410_05902_gb300.kkm import KKM, KKMError
    X, _ = inputs.isotropic_mixture(300, 4, 3, seed=8)
    run = KKM(torch.from_numpy(X).cuda(), 3, 32, tau=0, algo="table", param=1.0)
    with pytest.raises(KKMError, match="ENOTSUP"):
        run.get_state()
    with pytest.raises(KKMError, match="ENOTSUP"):
        run.assign(torch.from_numpy(X[:10]).cuda())
    run.close()
