"""torch.autograd.Function over the adjoint gradient of qaoa_gradient (argument marshalling only).

`qaoa_expectation_fn(gamma, beta, state)` returns <C> as a 0-d float64 tensor whose backward
yields d<C>/d gamma and d<C>/d beta.  The forward call already runs the GPU forward levels and the
adjoint sweep (the sweep needs the final state, and keeping it costs nothing extra), so backward
only scales the stored derivatives by the incoming gradient.
"""
from __future__ import annotations

import torch

from .binding import QAOAState, qaoa_gradient


class QAOAExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, gamma: torch.Tensor, beta: torch.Tensor, state: QAOAState, work: torch.Tensor):
        c, dg, db = qaoa_gradient(state.handle, gamma.detach().cpu().double().numpy(),
                                  beta.detach().cpu().double().numpy(), work.data_ptr(),
                                  work.numel() * work.element_size())
        ctx.save_for_backward(torch.from_numpy(dg).to(gamma.dtype), torch.from_numpy(db).to(beta.dtype))
        return torch.tensor(c, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        dg, db = ctx.saved_tensors
        g = grad_out.to(dg.dtype)
        return g * dg, g * db, None, None


def qaoa_expectation_fn(gamma: torch.Tensor, beta: torch.Tensor, state: QAOAState, work: torch.Tensor | None = None):
    """<C>(gamma, beta) of `state`'s graph as a differentiable function of the angles.  `work` is a
    device buffer of state.nbytes bytes for the adjoint sweep (allocated here when omitted)."""
    if work is None:
        work = torch.empty(state.nbytes, dtype=torch.uint8, device=state.buffer.device)
    return QAOAExpectation.apply(gamma, beta, state, work)
