"""The adjoint split at the end of the forward run (cg_adjoint_forward keeps
the checkpoints, cg_adjoint_reverse sweeps back from them): zT bit for bit
that of a plain run, lam0 and dL/dD bit for bit those of cg_adjoint_run
from the same z0 (which the oracle pins in test_adjoint_gpu.py), several
reverse calls on one set of checkpoints, and the rejection of buffers and
counts that the plan did not checkpoint."""
import numpy as np
import pytest

from paper_1309_1720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _prob(model, nx, ny, stencil, scheme):
    from paper_1309_1720_gb300 import Problem, FHN, BOCF, KARMA
    if model == FHN:
        return Problem(model=FHN, nx=nx, ny=ny, dx=0.04, stencil=stencil, scheme=scheme, dt=2e-4)
    if model == KARMA:
        return Problem(model=KARMA, nx=nx, ny=ny, dx=I.KARMA_DX, stencil=stencil, scheme=scheme, dt=0.05)
    return Problem(model=BOCF, nx=nx, ny=ny, dx=0.03, D=(1.171e-3,), Dyy=(1.171e-3 / 4,), stencil=stencil,
                   scheme=scheme, dt=0.05)


def _z0(p):
    from paper_1309_1720_gb300 import FHN, BOCF
    if p.model == FHN:
        return I.fhn_broken_wave(p.nx, p.ny, width=6)
    if p.model == BOCF:
        return I.bocf_spiral_cores(p.nx, p.ny, n_cores=2)
    u = 0.5 + 0.5 * I.uniform_pm1(3, p.nx * p.ny)
    v = 0.5 + 0.5 * I.uniform_pm1(4, p.nx * p.ny)
    return np.stack([u, v]).reshape(2, p.ny, p.nx)


@pytest.mark.parametrize("model,stencil,scheme", [(0, 0, 2), (0, 1, 0), (1, 1, 2), (1, 0, 1), (2, 0, 2)])
@pytest.mark.parametrize("steps,every", [(17, 0), (17, 1), (17, 5), (17, 17), (1, 0), (0, 0), (13, 40)])
def test_split_equals_adjoint_run(cuda_ok, model, stencil, scheme, steps, every):
    import torch
    from paper_1309_1720_gb300 import Plan
    p = _prob(model, 67, 45, stencil, scheme)
    z0 = torch.from_numpy(_z0(p)).cuda()
    plan = Plan(p)
    zT, ck = plan.forward_checkpointed(z0, steps, every)
    assert torch.equal(zT, plan.run(z0, steps))
    for seed in (77, 78):
        lamT = torch.from_numpy(I.unit_direction(tuple(z0.shape), seed)).cuda()
        lam0, dLdD = ck.adjoint(lamT)
        ref0, refD = plan.adjoint(z0, lamT, steps, checkpoint_every=every)
        plan.status()
        assert torch.equal(lam0, ref0)
        assert torch.equal(dLdD, refD)
        lam0s, none = ck.adjoint(lamT, with_dD=False)
        assert none is None and torch.equal(lam0s, ref0)


@pytest.mark.parametrize("tuning", [None, {"cells_x": 1, "threads": 512, "rows": 8, "schedule": 1}])
def test_split_at_larger_grid(cuda_ok, tuning):
    """The 512^2 two-field RK4 gradient, with the default launch shape and
    with the tile queue for the plain run: still bit for bit."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, RK4
    p = Problem(model=FHN, nx=512, ny=512, dx=0.04, scheme=RK4, dt=2.5e-4)
    plan = Plan(p, tuning=tuning)
    z0 = torch.from_numpy(I.fhn_broken_wave(512, 512, seed=0)).cuda()
    steps = 100
    zT, ck = plan.forward_checkpointed(z0, steps)
    assert torch.equal(zT, plan.run(z0, steps))
    lamT = torch.zeros_like(zT)
    lamT[0] = 2.0 * zT[0]
    lam0, dLdD = ck.adjoint(lamT)
    ref0, refD = plan.adjoint(z0, lamT, steps)
    plan.status()
    assert torch.equal(lam0, ref0) and torch.equal(dLdD, refD)


def test_reverse_rejects_what_was_not_checkpointed(cuda_ok):
    import ctypes
    import torch
    from paper_1309_1720_gb300 import Plan, CGError, _lib
    p = _prob(0, 40, 33, 0, 2)
    plan = Plan(p)
    z0 = torch.from_numpy(_z0(p)).cuda()
    zT, ck = plan.forward_checkpointed(z0, 12, 4)
    lamT = torch.ones_like(zT)
    lam0 = torch.empty_like(zT)
    ws = plan._adjoint_workspace(12, 4)
    L = _lib.lib()

    def rev(buf, n, every):
        return L.cg_adjoint_reverse(plan._h, buf.data_ptr(), lamT.data_ptr(), lam0.data_ptr(), None, n, every,
                                    ws.data_ptr(), None)

    assert rev(ck.buf, 12, 4) == 0
    assert rev(ck.buf, 13, 4) == 1                       # another step count
    assert rev(ck.buf, 12, 3) == 1                       # another checkpoint interval
    assert rev(torch.zeros_like(ck.buf), 12, 4) == 1     # a buffer never filled
    other = Plan(p)
    assert L.cg_adjoint_reverse(other._h, ck.buf.data_ptr(), lamT.data_ptr(), lam0.data_ptr(), None, 12, 4,
                                ws.data_ptr(), None) == 1  # another plan
    # every = 0 resolves to ceil(sqrt(n)): the same checkpoints as every = 4 for n = 12
    assert rev(ck.buf, 12, 0) == 0
    # lam0 inside the checkpoint buffer is rejected before any work
    assert L.cg_adjoint_reverse(plan._h, ck.buf.data_ptr(), lamT.data_ptr(), ck.buf.data_ptr(), None, 12, 4,
                                ws.data_ptr(), None) == 1
    # z0 / zT inside the checkpoint buffer are rejected before any work
    with pytest.raises(CGError):
        L2 = ck.buf.view(torch.uint8)
        _lib.check(L.cg_adjoint_forward(plan._h, z0.data_ptr(), L2.data_ptr(), 12, 4, ck.buf.data_ptr(),
                                        plan.workspace().data_ptr(), None))
    torch.cuda.synchronize()
    plan.status()
    other.close()
