"""torch.autograd binding of the discrete adjoint.

``CGFlow.apply(z0, D, plan, n_steps, checkpoint_every)`` returns z(T) from the
CUDA stepper for the diffusivities ``D`` (one per diffusive field: u and v
for FitzHugh-Nagumo, u for the other models; each field keeps the plan's
ratio Dyy/Dxx).  The forward keeps every c-th state of the run
(cg_adjoint_forward, c = checkpoint_every, default ceil(sqrt(T))), and its
backward sweeps back from those checkpoints with the discrete adjoint
kernels (cg_adjoint_reverse: each segment recomputed with its stage inputs
kept, then reversed), giving dL/dz0 and dL/dD (skipped when D does not
require a gradient); the values are bit for bit those of cg_adjoint_run,
without its forward sweep.  A pending backward holds ceil(T/c) states.  When ``D`` equals the plan's
own diffusivities the plan itself runs; otherwise a plan with the same
grid, model, scheme, ghosts and launch shape but these diffusivities is
built (and kept for reuse with that D).
"""
from __future__ import annotations

import dataclasses
from collections import OrderedDict

import torch

from . import api

_MAX_CACHED = 4


def _diffusive_fields(model: int) -> int:
    return 2 if model == api.FHN else 1


def _plan_D(plan) -> list:
    """The plan's Dxx of each diffusive field."""
    p = plan.problems[0]
    Dxx = list(api._DEFAULT_D.get(p.model, ()) if p.D is None else p.D)
    return [float(Dxx[i]) if i < len(Dxx) else 0.0 for i in range(_diffusive_fields(p.model))]


def plan_for_D(plan, D: torch.Tensor):
    """``plan`` if D holds its diffusivities, else a plan for D (cached on
    ``plan``, the few most recent values)."""
    if len(plan.problems) != 1:
        raise ValueError("the differentiable flow needs a single-instance plan")
    p = plan.problems[0]
    nd = _diffusive_fields(p.model)
    vals = [float(x) for x in D.detach().reshape(-1).cpu().tolist()]
    if len(vals) != nd:
        raise ValueError("D has %d entries; this model has %d diffusive field(s)" % (len(vals), nd))
    base = _plan_D(plan)
    if vals == base:
        return plan
    cache = plan.__dict__.setdefault("_d_plans", OrderedDict())
    key = tuple(vals)
    if key in cache:
        cache.move_to_end(key)
        return cache[key]
    Dxx = list(api._DEFAULT_D.get(p.model, ()) if p.D is None else p.D)
    Dyy = list(Dxx if p.Dyy is None else p.Dyy)
    new_xx, new_yy = list(Dxx), list(Dyy)
    for i, d in enumerate(vals):
        ratio = Dyy[i] / Dxx[i] if i < len(Dxx) and Dxx[i] != 0.0 else 1.0
        while len(new_xx) <= i:
            new_xx.append(0.0)
            new_yy.append(0.0)
        new_xx[i], new_yy[i] = d, d * ratio
    q = dataclasses.replace(p, D=tuple(new_xx), Dyy=tuple(new_yy), _keep=[])
    cache[key] = api.Plan(q, tuning=plan.tuning)
    # evicted plans are not closed here: a pending backward may still hold
    # one (its autograd context keeps a reference); they close when freed
    while len(cache) > _MAX_CACHED:
        cache.popitem(last=False)
    return cache[key]


class CGFlow(torch.autograd.Function):
    @staticmethod
    def forward(ctx, z0, D, plan, n_steps, checkpoint_every=0):
        run_plan = plan_for_D(plan, D)
        z0c = z0.detach().contiguous()
        zT, ctx.ckpt = run_plan.forward_checkpointed(z0c, int(n_steps), int(checkpoint_every))
        ctx.d_shape = D.shape
        return zT

    @staticmethod
    def backward(ctx, grad_zT):
        want_dD = ctx.needs_input_grad[1]
        lam0, dLdD = ctx.ckpt.adjoint(grad_zT.detach().contiguous(), with_dD=want_dD)
        return lam0, dLdD.reshape(ctx.d_shape) if want_dD else None, None, None, None


def flow(z0: torch.Tensor, D: torch.Tensor, plan, n_steps: int, checkpoint_every: int = 0) -> torch.Tensor:
    """Differentiable n-step flow map of the stepper (see CGFlow)."""
    return CGFlow.apply(z0, D, plan, n_steps, checkpoint_every)
