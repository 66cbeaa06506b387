"""torch.autograd binding of the discrete adjoint.

``CGFlow.apply(z0, D, plan, n_steps, checkpoint_every)`` returns z(T) from the
CUDA stepper; its backward calls the discrete adjoint kernels with
sqrt(T)-checkpointed recomputation (cg_adjoint_run), giving dL/dz0 and dL/dD
for each diffusive field's D (anisotropy ratio fixed; skipped when D does
not require a gradient).  ``D`` must hold the diffusivities the plan was
built with; it is an input only so that autograd can route its gradient.
"""
from __future__ import annotations

import torch


class CGFlow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z0, D, plan, n_steps, checkpoint_every=0):
        z0c = z0.detach().contiguous()
        zT = plan.run(z0c, int(n_steps))
        ctx.save_for_backward(z0c)
        ctx.plan = plan
        ctx.n_steps = int(n_steps)
        ctx.every = int(checkpoint_every)
        ctx.d_shape = D.shape
        return zT

    @staticmethod
    def backward(ctx, grad_zT):
        (z0,) = ctx.saved_tensors
        want_dD = ctx.needs_input_grad[1]
        lam0, dLdD = ctx.plan.adjoint(z0, grad_zT.detach().contiguous(), ctx.n_steps, ctx.every,
                                      with_dD=want_dD)
        return lam0, dLdD.reshape(ctx.d_shape) if want_dD else None, None, None, None


def flow(z0: torch.Tensor, D: torch.Tensor, plan, n_steps: int, checkpoint_every: int = 0) -> torch.Tensor:
    """Differentiable n-step flow map of the stepper (see CGFlow)."""
    return CGFlow.apply(z0, D, plan, n_steps, checkpoint_every)
