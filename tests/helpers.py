"""Shared helpers of the test suite: build the same problem for the CUDA path
(through the C ABI) and for the CPU oracle, and compare results."""
from __future__ import annotations

import numpy as np

import oracle as O

_MODEL = {0: O.FHN, 1: O.BOCF, 2: O.KARMA, 3: O.DIFFUSION}


def oracle_problem(p):
    """Oracle record for a paper_1309_1720_gb300.Problem."""
    from paper_1309_1720_gb300 import api
    c = p.to_c()
    return O.problem(_MODEL[p.model], nx=p.nx, ny=p.ny, dx=c.dx, dy=c.dy,
                     Dxx=[c.Dxx[i] for i in range(4)], Dyy=[c.Dyy[i] for i in range(4)],
                     stencil=p.stencil, alpha_d=p.alpha_d, bc=p.bc, scheme=p.scheme, dt=p.dt,
                     params=None if p.params is None else list(p.params),
                     variant=O.TANH_AS_HK if (p.flags & api.FLAG_TANH_AS_HK) else O.AS_WRITTEN)


def oracle_run(p, z0: np.ndarray, n_steps: int) -> np.ndarray:
    return O.step(oracle_problem(p), z0, n_steps)


def gpu_run(p, z0: np.ndarray, n_steps: int, tuning=None, inplace: bool = False) -> np.ndarray:
    import torch
    from paper_1309_1720_gb300 import Plan
    plan = Plan(p, tuning=tuning)
    z = torch.from_numpy(np.ascontiguousarray(z0)).cuda()
    if inplace:
        plan.run(z, n_steps, out=z)
        out = z
    else:
        out = plan.run(z, n_steps)
    plan.status()
    res = out.cpu().numpy()
    plan.close()
    return res


def field_rel_err(g: np.ndarray, o: np.ndarray) -> float:
    """Max over fields of max|g - o| / max|o| (the parity metric)."""
    errs = []
    for f in range(o.shape[0]):
        den = np.max(np.abs(o[f]))
        errs.append(np.max(np.abs(g[f] - o[f])) / (den if den > 0 else 1.0))
    return float(max(errs))
