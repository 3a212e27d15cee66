"""torch.autograd binding of the batch objective at fixed assignments.

``objective(run, Q, log_sigma, assign)`` returns
L = (1/m) sum_x Delta(x, C_{assign(x)}) for the centers ``run`` currently
holds (support rows and weights fixed), with the bandwidth parameterised by
s = log sigma (Gaussian kappa = 2 e^{2s}, Laplacian sigma = e^s). Gradients
flow to ``Q`` (float32, m x d, CUDA) and ``log_sigma`` (a 0-dim or 1-element
float64 CUDA tensor). Forward and backward are the library's
kkm_objective_fwd / kkm_objective_bwd kernels; the backward recomputes the
kernel values instead of storing them. The assignments are not
differentiable.
"""
from __future__ import annotations

import torch

from .kkm import KKM


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Q, log_sigma, run, assign):
        if not (Q.is_cuda and Q.dtype == torch.float32 and Q.dim() == 2 and Q.stride(1) == 1):
            raise TypeError("Q must be a row-contiguous 2-D float32 CUDA tensor")
        if assign.dtype != torch.int32 or not assign.is_contiguous():
            raise TypeError("assign must be a contiguous int32 tensor")
        s = float(log_sigma.detach().reshape(-1)[0].item())
        loss, _ = run.objective_fwd(Q, assign, s)
        ctx.save_for_backward(Q, assign)
        ctx.run = run
        ctx.s = s
        ctx.ls_shape = log_sigma.shape
        return loss.reshape(())

    @staticmethod
    def backward(ctx, grad_out):
        Q, assign = ctx.saved_tensors
        g = grad_out.detach().to(torch.float64).reshape(1).contiguous()
        gq, gs = ctx.run.objective_bwd(Q, assign, ctx.s, g)
        return gq, gs.reshape(ctx.ls_shape), None, None


def objective(run: KKM, Q: torch.Tensor, log_sigma: torch.Tensor, assign: torch.Tensor) -> torch.Tensor:
    """Differentiable batch objective (see the module docstring)."""
    return _Objective.apply(Q, log_sigma, run, assign)
