"""``torch.autograd.Function`` over (p0_1..K, c): forward = pat_forward,
backward = pat_vjp (the discrete adjoint of Sec. 3 with an arbitrary adjoint
source dL/dy).

The forward keeps wavefield checkpoints (every s steps, the plan's
ckpt_every) in a workspace owned by the autograd node; the backward recomputes
each segment from its checkpoint and runs the adjoint through it, so long time
series fit in HBM.  Gradients with respect to c cover the domain cells only
(c in the PML is fixed).
"""
from __future__ import annotations

import torch

from . import _binding as B
from .solver import Plan


class KSpaceForward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p0: torch.Tensor, c: torch.Tensor, plan: Plan):
        p0c = p0.detach().contiguous()
        cc = c.detach().contiguous()
        ws = torch.empty(plan.workspace_bytes(B.PAT_WS_GRADIENT), dtype=torch.uint8, device=plan.device)
        y = plan.forward(cc, p0c, keep_checkpoints=True, ws=ws)
        # the workspace (checkpoints) is saved like the inputs: autograd releases it after the
        # backward pass, or keeps it for another one when the graph is retained
        ctx.save_for_backward(p0c, cc, ws)
        ctx.plan = plan
        return y

    @staticmethod
    def backward(ctx, ybar: torch.Tensor):
        p0, c, ws = ctx.saved_tensors
        gp, gc = ctx.plan.vjp(c, p0, ybar.contiguous().to(torch.float32), ws=ws)
        return (gp if ctx.needs_input_grad[0] else None, gc if ctx.needs_input_grad[1] else None, None)


def pat_forward(p0: torch.Tensor, c: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable sensor traces y[K][nt][m] = f(p0, c)."""
    return KSpaceForward.apply(p0, c, plan)


def data_misfit(y: torch.Tensor, y_meas: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """J = sum_k w_k / 2 ||y_k - y_meas_k||^2 (Eq. Minimised_functional, data term), FP64 sum.

    A loss for the differentiable path above, in torch operations on traces that the library
    computed (its gradient dJ/dy = w_k (y_k - y_meas_k) becomes the adjoint source of pat_vjp).
    The library evaluates the same J itself, with the gradient, in pat_adjoint_grad
    (Plan.adjoint_grad); the reconstruction uses that one.
    """
    d = (y - y_meas).double()
    return 0.5 * (w.double()[:, None, None] * d * d).sum()
