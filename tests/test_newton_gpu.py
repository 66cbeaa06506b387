"""Newton-Krylov step (GMRES with exact Jacobian-vector products), the
deterministic vector kernels, and the torch.autograd binding."""
import ctypes

import numpy as np
import pytest

from helpers import oracle_problem
from paper_1309_1720_gb300 import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


def _dense_jacobian(op, z0, steps):
    """Oracle flow-map Jacobian column by column from its tangent-linear model."""
    n = z0.size
    J = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        _, col = O.tlm(op, z0, e.reshape(z0.shape), steps)
        J[:, k] = col.ravel()
    return J


@pytest.mark.parametrize("model", [0, 3])
def test_gmres_step_small_exact(cuda_ok, model):
    """On a 6 x 5 grid the Krylov space spans the whole state, so one GMRES
    cycle solves the Newton system; its residual, measured with the oracle's
    dense Jacobian and flow map, is at rounding level."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, DIFFUSION, RK4
    if model == FHN:
        p = Problem(model=FHN, nx=6, ny=5, dx=0.5, scheme=RK4, dt=0.01)
        z0 = I.fhn_broken_wave(6, 5, width=2)
    else:
        p = Problem(model=DIFFUSION, nx=6, ny=5, dx=0.5, D=(1.0,), scheme=RK4, dt=0.01)
        z0 = (1.0 + 0.3 * I.uniform_pm1(4, 30)).reshape(1, 5, 6)
    steps = 40
    n = z0.size
    plan = Plan(p)
    dz, hist = plan.newton_step(torch.from_numpy(z0).cuda(), steps, restart=n, max_restarts=1, rtol=1e-13)
    op = oracle_problem(p)
    J = _dense_jacobian(op, z0, steps)
    b = -(O.step(op, z0, steps) - z0).ravel()
    r = (J - np.eye(n)) @ dz.cpu().numpy().ravel() - b
    assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(b)
    assert hist[0] == pytest.approx(np.linalg.norm(b), rel=1e-12)


def test_gmres_residuals_decrease_c5_shape(cuda_ok):
    """512^2 RK4 5-point, period 200 steps, GMRES(30): the Arnoldi residual
    history is non-increasing and the true residual of the returned step
    (recomputed with the tangent kernels) matches the last history entry."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, RK4
    n, T = 512, 200
    p = Problem(model=FHN, nx=n, ny=n, dx=0.04, scheme=RK4, dt=2.5e-4)
    z0 = torch.from_numpy(I.fhn_broken_wave(n, n, seed=0)).cuda()
    plan = Plan(p)
    dz, hist = plan.newton_step(z0, T, restart=30, max_restarts=1, rtol=1e-12)
    assert len(hist) == 31
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(30))
    _, Jdz = plan.tlm(z0, dz[None].contiguous(), T)
    b = -(plan.run(z0, T) - z0)
    true_r = float(torch.linalg.norm(Jdz[0] - dz - b))
    assert abs(true_r - hist[-1]) <= 1e-6 * hist[0]


def test_dot_and_axpby_deterministic(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import _lib
    L = _lib.lib()
    x = torch.from_numpy(I.uniform_pm1(1, 1_000_003)).cuda()
    y = torch.from_numpy(I.uniform_pm1(2, 1_000_003)).cuda()
    ws = torch.empty(256, dtype=torch.float64, device="cuda")
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    assert L.cg_dot(x.data_ptr(), y.data_ptr(), x.numel(), out.data_ptr(), ws.data_ptr(), s) == 0
    assert L.cg_dot(x.data_ptr(), y.data_ptr(), x.numel(), out[1:].data_ptr(), ws.data_ptr(), s) == 0
    torch.cuda.synchronize()
    ref = np.dot(x.cpu().numpy(), y.cpu().numpy())
    assert out[0].item() == out[1].item()
    assert abs(out[0].item() - ref) <= 1e-12 * np.sum(np.abs(x.cpu().numpy() * y.cpu().numpy()))
    yy = y.clone()
    assert L.cg_axpby(ctypes.c_double(0.5), x.data_ptr(), ctypes.c_double(-2.0), yy.data_ptr(), x.numel(), s) == 0
    torch.cuda.synchronize()
    assert torch.allclose(yy, 0.5 * x - 2.0 * y, rtol=0, atol=1e-15)


def test_autograd_flow(cuda_ok):
    """CGFlow.backward = the adjoint kernels: gradients of
    L = sum (u_T - u_tgt)^2 w.r.t. z0 and D_u equal cg_adjoint_run's and
    match central differences."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, RK4
    from paper_1309_1720_gb300.autograd import flow
    n, steps = 96, 120
    base = dict(model=FHN, nx=n, ny=n, dx=0.04, scheme=RK4, dt=2.5e-4)
    plan = Plan(Problem(**base))
    z0 = torch.from_numpy(I.fhn_broken_wave(n, n, seed=0)).cuda().requires_grad_(True)
    D = torch.tensor([1.0, 1.5], dtype=torch.float64, device="cuda", requires_grad=True)
    u_tgt = Plan(Problem(D=(1.05, 1.5), **base)).run(z0.detach(), steps)[0]
    zT = flow(z0, D, plan, steps, checkpoint_every=7)
    loss = torch.sum((zT[0] - u_tgt) ** 2)
    loss.backward()
    lamT = torch.zeros_like(zT)
    lamT[0] = 2 * (zT[0].detach() - u_tgt)
    lam0, dLdD = plan.adjoint(z0.detach(), lamT, steps, checkpoint_every=7)
    assert torch.equal(z0.grad, lam0) and torch.equal(D.grad, dLdD)
    eps = 1e-6

    def L_of(Du):
        q = Plan(Problem(D=(Du, 1.5), **base))
        return float(torch.sum((q.run(z0.detach(), steps)[0] - u_tgt) ** 2))
    fd = (L_of(1 + eps) - L_of(1 - eps)) / (2 * eps)
    assert abs(float(D.grad[0]) - fd) <= 1e-8 * abs(fd)


def test_autograd_flow_follows_D(cuda_ok):
    """The differentiable flow runs with the D it is given: with D unlike the
    plan's, the forward equals a plan built with that D bit for bit, the
    gradients equal that plan's adjoint, and dL/dD matches central
    differences; D back at the plan's values runs the plan itself."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, BOCF, RK4, STENCIL9
    from paper_1309_1720_gb300.autograd import flow, plan_for_D
    n, steps = 64, 80
    base = dict(model=FHN, nx=n, ny=n + 5, dx=0.04, scheme=RK4, dt=2.5e-4)
    plan = Plan(Problem(**base))
    z0 = torch.from_numpy(I.fhn_broken_wave(n, n + 5, seed=3)).cuda()
    u_tgt = Plan(Problem(D=(1.05, 1.5), **base)).run(z0, steps)[0]
    for Dv in ((1.1, 1.4), (1.0, 1.5)):
        D = torch.tensor(Dv, dtype=torch.float64, device="cuda", requires_grad=True)
        z = z0.clone().requires_grad_(True)
        zT = flow(z, D, plan, steps)
        ref_plan = Plan(Problem(D=Dv, **base))
        assert torch.equal(zT, ref_plan.run(z0, steps))
        assert (plan_for_D(plan, D) is plan) == (Dv == (1.0, 1.5))
        loss = torch.sum((zT[0] - u_tgt) ** 2)
        loss.backward()
        lamT = torch.zeros_like(zT)
        lamT[0] = 2 * (zT[0].detach() - u_tgt)
        lam0, dLdD = ref_plan.adjoint(z0, lamT, steps)
        assert torch.equal(z.grad, lam0) and torch.equal(D.grad, dLdD)
        eps = 1e-6

        def L_of(Du):
            q = Plan(Problem(D=(Du, Dv[1]), **base))
            return float(torch.sum((q.run(z0, steps)[0] - u_tgt) ** 2))
        fd = (L_of(Dv[0] + eps) - L_of(Dv[0] - eps)) / (2 * eps)
        assert abs(float(D.grad[0]) - fd) <= 1e-8 * abs(fd)
    # more distinct D values than the plan keeps, all forwards first: every
    # backward still runs on the plan of its own D
    outs = []
    for j in range(6):
        Dj = torch.tensor((1.0 + 0.02 * (j + 1), 1.5), dtype=torch.float64, device="cuda", requires_grad=True)
        zj = z0.clone().requires_grad_(True)
        outs.append((Dj, zj, flow(zj, Dj, plan, 10)))
    for j, (Dj, zj, oj) in enumerate(outs):
        oj[0].sum().backward()
        ref_plan = Plan(Problem(D=(1.0 + 0.02 * (j + 1), 1.5), **base))
        lam = torch.zeros_like(oj)
        lam[0] = 1.0
        l0, dd = ref_plan.adjoint(z0, lam, 10)
        assert torch.equal(zj.grad, l0) and torch.equal(Dj.grad, dd), j
    # anisotropic four-field plan: the ratio Dyy/Dxx of the plan is kept
    bp = dict(model=BOCF, nx=40, ny=33, dx=0.03, stencil=STENCIL9, scheme=RK4, dt=0.05)
    plan_b = Plan(Problem(D=(1.171e-3,), Dyy=(1.171e-3 / 4,), **bp))
    zb = torch.from_numpy(I.bocf_spiral_cores(40, 33, n_cores=2)).cuda()
    Db = torch.tensor([1.3e-3], dtype=torch.float64, device="cuda")
    out = flow(zb, Db, plan_b, 10)
    assert torch.equal(out, Plan(Problem(D=(1.3e-3,), Dyy=(1.3e-3 / 4,), **bp)).run(zb, 10))
    with pytest.raises(ValueError):
        flow(zb, torch.tensor([1e-3, 1e-3], dtype=torch.float64, device="cuda"), plan_b, 10)
