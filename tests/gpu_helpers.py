"""Shared helpers of the GPU parity tests (oracle vs the CUDA path through the C-ABI)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2410_05902_gb300 import inputs

# Distance tolerances, normwise over the b x k matrix:
#     max |d_gpu - d| / max |d|.
# Delta = K(x,x) - 2<phi(x),C> + ||C||^2 is a difference of O(gamma^2) terms, so
# its absolute error floor is gamma^2 times the unit roundoff whatever its size.
# An elementwise relative bound would fail on legitimately small distances in
# any finite precision. FP32 and the split-BF16 form are held to 1e-5 and BF16
# to 2e-3. The objective is held to 1e-4 relative. Assignments must match
# except on rows whose FP64 oracle gap d_(2) - d_(1) lies within the form's
# absolute error bound, tol * max |d|.
# TF32 operands carry 11 significant bits to BF16's 8, so its bound is BF16's / 8.
DIST_TOL = {"fp32": 1e-5, "bf16x3": 1e-5, "bf16": 2e-3, "tf32": 2.5e-4}
OBJ_TOL = 1e-4
# BF16 operands carry 8 significant bits: its f_B error is of the order of its
# distance error, so it is held to that here (the benchmark reports whether the
# BF16 form reaches the 1e-4 objective bar on its workload).
OBJ_TOL_FORM = {"fp32": OBJ_TOL, "bf16x3": OBJ_TOL, "bf16": 2e-3, "tf32": 2.5e-4}
# center norms after one teacher-forced step (the Gram error enters the recurrence's sums)
CN_RTOL = {"fp32": 1e-6, "bf16x3": 1e-6, "bf16": 5e-3, "tf32": 1e-3}
KIND = {"gaussian": oracle.GAUSSIAN, "laplacian": oracle.LAPLACIAN, "linear": oracle.LINEAR,
        "poly": oracle.POLY}


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def dist_rel_err(d_gpu, d_ref) -> float:
    d_gpu = np.asarray(d_gpu, dtype=np.float64)
    return float(np.max(np.abs(d_gpu - d_ref)) / max(float(np.max(np.abs(d_ref))), 1e-300))


def near_tie_ok(assign_gpu, rec, tol_abs) -> tuple[bool, int]:
    """All assignment mismatches are certified near-ties of the oracle."""
    bad = np.nonzero(np.asarray(assign_gpu) != rec_argmin(rec))[0]
    ok = bool(np.all(rec.gap[bad] <= tol_abs))
    return ok, len(bad)


def rec_argmin(rec):
    return np.argmin(rec.dist, axis=1)


class Pair:
    """An oracle run and a GPU run on the same data, kernel and initial centers."""

    def __init__(self, X, k, b, kernel="gaussian", param=None, tau=200, precision="fp32",
                 init=None, lr="beta", eta=None, max_iters=0, coef0=0.0, degree=2, seed=0, dist_tile=0,
                 algo="windows"):
        torch = torch_cuda()
        from paper_2410_05902_gb300.kkm import KKM
        self.torch = torch
        self.X = np.ascontiguousarray(X, dtype=np.float32)
        n = len(self.X)
        if param is None:
            sigma = inputs.median_sigma(self.X, seed=1)
            param = 2 * sigma * sigma if kernel == "gaussian" else sigma
        self.param = float(param)
        self.k, self.b, self.precision = k, b, precision
        self.init = inputs.init_indices(n, k, seed=3) if init is None else np.asarray(init, np.int64)
        self.kern = oracle.Kernel(KIND[kernel], self.param, coef0, degree)
        self.ora = oracle.MiniBatchKernelKMeans(self.X.astype(np.float64), k, self.kern, b, self.init,
                                                tau=(tau if tau > 0 else None), lr=lr, eta=eta)
        self.Xd = torch.from_numpy(self.X).cuda()
        self.gpu = KKM(self.Xd, k, b, kernel=kernel, param=self.param, coef0=coef0, degree=degree,
                       tau=tau, lr=lr, eta=eta or 0.0, precision=precision, seed=seed,
                       init_idx=self.init, max_iters=max_iters, dist_tile=dist_tile, algo=algo)
        self.dist = torch.empty((b, k), dtype=torch.float32, device="cuda")
        self.assign = torch.empty(b, dtype=torch.int32, device="cuda")
        self.obj = torch.empty(1, dtype=torch.float64, device="cuda")

    def gpu_step(self, batch, forced=None):
        torch = self.torch
        bi = torch.from_numpy(np.asarray(batch, np.int32)).cuda()
        fa = None if forced is None else torch.from_numpy(np.asarray(forced, np.int32)).cuda()
        self.gpu.step(bi, fa, self.assign, self.dist, self.obj)
        torch.cuda.synchronize()
        return self.dist.cpu().numpy(), self.assign.cpu().numpy(), float(self.obj.cpu()[0])

    def abs_tol(self, rec):
        return DIST_TOL[self.precision] * float(np.max(np.abs(rec.dist)))

    def close(self):
        self.gpu.close()


def compare_states(gpu_state, ora_state, w_rtol=1e-12, cn_rtol=1e-6):
    """Window layout identical, weights to FP64 rounding, norms to the form's accuracy."""
    for key in ("rows_per_center", "row_idx", "blocks_per_center", "block_iter", "block_count"):
        np.testing.assert_array_equal(np.asarray(gpu_state[key], np.int64),
                                      np.asarray(ora_state[key], np.int64), err_msg=key)
    np.testing.assert_array_equal(gpu_state["c1_kept"].astype(bool), ora_state["c1_kept"])
    np.testing.assert_allclose(gpu_state["row_w"], ora_state["row_w"], rtol=w_rtol, atol=1e-300)
    np.testing.assert_allclose(gpu_state["cnorm"], ora_state["cnorm"], rtol=cn_rtol, atol=cn_rtol)
    if "cum_counts" in gpu_state and "cum_counts" in ora_state:
        np.testing.assert_array_equal(gpu_state["cum_counts"], ora_state["cum_counts"])
    assert gpu_state["iteration"] == ora_state["iteration"]
