"""Tangent-linear kernels against the oracle's tangent-linear model and
against central finite differences of the CUDA stepper itself."""
import numpy as np
import pytest

from helpers import field_rel_err, oracle_problem
from paper_1309_1720_gb300 import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


def _prob(model, n, stencil, scheme):
    from paper_1309_1720_gb300 import Problem, FHN
    if model == FHN:
        return Problem(model=FHN, nx=n, ny=n - 7, dx=0.04, stencil=stencil, scheme=scheme, dt=2e-4)
    from paper_1309_1720_gb300 import BOCF
    return Problem(model=BOCF, nx=n, ny=n - 7, dx=0.03, D=(1.171e-3,), Dyy=(1.171e-3 / 4,), stencil=stencil,
                   scheme=scheme, dt=0.05)


def _z0(model, p):
    from paper_1309_1720_gb300 import FHN
    if model == FHN:
        return I.fhn_broken_wave(p.nx, p.ny, width=6)
    return I.bocf_spiral_cores(p.nx, p.ny, n_cores=2)


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_tlm_matches_oracle(cuda_ok, model, stencil, scheme):
    import torch
    from paper_1309_1720_gb300 import Plan
    p = _prob(model, 70, stencil, scheme)
    z0 = _z0(model, p)
    T, steps = 3, 25
    dz0 = np.stack([I.unit_direction(z0.shape, 40 + i) for i in range(T)])
    plan = Plan(p)
    zT, dzT = plan.tlm(torch.from_numpy(z0).cuda(), torch.from_numpy(dz0).cuda(), steps)
    plan.status()
    zT, dzT = zT.cpu().numpy(), dzT.cpu().numpy()
    op = oracle_problem(p)
    for i in range(T):
        oz, odz = O.tlm(op, z0, dz0[i], steps)
        assert field_rel_err(dzT[i], odz) <= 1e-12, i
    assert field_rel_err(zT, O.step(op, z0, steps)) <= 1e-12
    # the primal of the TLM run equals a plain run bitwise
    assert np.array_equal(zT, plan.run(torch.from_numpy(z0).cuda(), steps).cpu().numpy())


def test_tlm_fd_full_size(cuda_ok):
    """512^2 RK4 5-point: 64 unit tangents in one run; two of them against
    central differences of the CUDA stepper (eps = 1e-6) to 1e-8."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, RK4
    n, steps = 512, 50
    p = Problem(model=FHN, nx=n, ny=n, dx=0.04, scheme=RK4, dt=2.5e-4)
    z0 = I.fhn_broken_wave(n, n, seed=0)
    T = 64
    dz0 = np.stack([I.unit_direction(z0.shape, 2, offset=i * z0.size) for i in range(T)])
    plan = Plan(p)
    zd = torch.from_numpy(z0).cuda()
    _, dzT = plan.tlm(zd, torch.from_numpy(dz0).cuda(), steps)
    plan.status()
    # Central differences of a 524288-dimensional state: each run carries
    # ~1e-15 of rounding per cell, so at eps = 1e-6 the difference quotient
    # has a noise floor of ~1e-15/2e-6 * sqrt(N) ~ 4e-7 in the relative
    # 2-norm; at eps = 1e-4 the floor is ~4e-9 and the O(eps^2) truncation is
    # far smaller, so that is where the 1e-8 bound is checked.
    for eps, tol in ((1e-6, 2e-6), (1e-4, 1e-8)):
        for i in (0, 63):
            d = torch.from_numpy(dz0[i]).cuda()
            fd = (plan.run(zd + eps * d, steps) - plan.run(zd - eps * d, steps)) / (2 * eps)
            err = torch.linalg.norm(dzT[i] - fd) / torch.linalg.norm(fd)
            assert float(err) <= tol, (eps, i, float(err))
