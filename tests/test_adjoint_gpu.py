"""Discrete adjoint kernels: parity with the oracle's adjoint (which stores
every state and applies the literal transposed stencil), the dot-product
identity against the CUDA tangent-linear kernels, central finite
differences, and bitwise reproducibility of dL/dD."""
import numpy as np
import pytest

from helpers import field_rel_err, oracle_problem
from paper_1309_1720_gb300 import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


def _prob(model, nx, ny, stencil, scheme, bc=0):
    from paper_1309_1720_gb300 import Problem, FHN, BOCF, DIFFUSION
    if model == FHN:
        return Problem(model=FHN, nx=nx, ny=ny, dx=0.04, stencil=stencil, scheme=scheme, bc=bc, dt=2e-4)
    if model == DIFFUSION:
        return Problem(model=DIFFUSION, nx=nx, ny=ny, dx=0.1, D=(1.0,), Dyy=(0.6,), stencil=stencil,
                       scheme=scheme, bc=bc, dt=1e-3)
    return Problem(model=BOCF, nx=nx, ny=ny, dx=0.03, D=(1.171e-3,), Dyy=(1.171e-3 / 4,), stencil=stencil,
                   scheme=scheme, bc=bc, dt=0.05)


def _z0(p):
    from paper_1309_1720_gb300 import FHN, BOCF
    if p.model == FHN:
        return I.fhn_broken_wave(p.nx, p.ny, width=6)
    if p.model == BOCF:
        return I.bocf_spiral_cores(p.nx, p.ny, n_cores=2)
    return (1.0 + 0.3 * I.uniform_pm1(9, p.nx * p.ny)).reshape(1, p.ny, p.nx)


@pytest.mark.parametrize("model", [0, 1, 3])
@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("bc", [0, 1])
def test_adjoint_matches_oracle(cuda_ok, model, stencil, scheme, bc):
    import torch
    from paper_1309_1720_gb300 import Plan
    p = _prob(model, 67, 45, stencil, scheme, bc)
    z0 = _z0(p)
    steps = 17
    lamT = I.unit_direction(z0.shape, 77)
    plan = Plan(p)
    for every in (0, 1, 5, 17):
        lam0, dLdD = plan.adjoint(torch.from_numpy(z0).cuda(), torch.from_numpy(lamT).cuda(), steps,
                                  checkpoint_every=every)
        plan.status()
        olam0, odLdD = O.adjoint(oracle_problem(p), z0, lamT, steps)
        assert field_rel_err(lam0.cpu().numpy(), olam0) <= 1e-12, every
        g = dLdD.cpu().numpy()
        assert np.all(np.abs(g - odLdD[:len(g)]) <= 1e-10 * np.maximum(np.abs(odLdD[:len(g)]), 1e-30)), (g, odLdD)


def test_tiny_grids_and_edges(cuda_ok):
    """2 x 2 and 3 x 7 grids, where every cell is a boundary cell."""
    import torch
    from paper_1309_1720_gb300 import Plan
    for (nx, ny) in [(2, 2), (3, 7), (33, 2)]:
        for stencil in (0, 1):
            p = _prob(0, nx, ny, stencil, 2)
            z0 = _z0(p)
            lamT = I.unit_direction(z0.shape, 5)
            lam0, dLdD = Plan(p).adjoint(torch.from_numpy(z0).cuda(), torch.from_numpy(lamT).cuda(), 9)
            olam0, odLdD = O.adjoint(oracle_problem(p), z0, lamT, 9)
            assert field_rel_err(lam0.cpu().numpy(), olam0) <= 1e-12
            # dL/dD_u of the 2 x 2 grid is a near-cancelling sum (1-ulp noise in
            # z0 moves it by 1e-11 relative in the oracle itself), so the
            # gradient's 1e-8 bound applies here
            assert np.allclose(dLdD.cpu().numpy(), odLdD, rtol=1e-8, atol=0)


@pytest.mark.parametrize("model", [0, 1])
def test_dot_product_identity(cuda_ok, model):
    """<J v, w> from the tangent kernels equals <v, J^T w> from the adjoint
    kernels to 1e-13 relative."""
    import torch
    from paper_1309_1720_gb300 import Plan, STENCIL9, RK4
    p = _prob(model, 150, 97, STENCIL9, RK4)
    z0 = _z0(p)
    v = I.unit_direction(z0.shape, 1)
    w = I.unit_direction(z0.shape, 2)
    plan = Plan(p)
    zd = torch.from_numpy(z0).cuda()
    _, Jv = plan.tlm(zd, torch.from_numpy(v)[None].cuda().contiguous(), 40)
    JTw, _ = plan.adjoint(zd, torch.from_numpy(w).cuda(), 40)
    lhs = float(torch.sum(Jv[0] * torch.from_numpy(w).cuda()))
    rhs = float(torch.sum(torch.from_numpy(v).cuda() * JTw))
    scale = float(torch.linalg.norm(Jv)) * 1.0
    assert abs(lhs - rhs) <= 1e-13 * max(scale, abs(lhs))


def test_gradient_fd_and_cpu_reference(cuda_ok):
    """L = sum (u_T - u_tgt)^2 on a 128^2 two-field RK4 run of 200 steps, the
    target from D_u * 1.05: the adjoint gradient w.r.t. z0 (along a random
    direction) and D_u against central differences (eps = 1e-6) and against
    the oracle's stored-trajectory gradient, each to 1e-8 relative."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, RK4
    n, steps = 128, 200
    base = dict(model=FHN, nx=n, ny=n, dx=0.04, scheme=RK4, dt=2.5e-4)
    z0 = I.fhn_broken_wave(n, n, seed=0)
    tgt_plan = Plan(Problem(D=(1.05, 1.5), **base))
    zd = torch.from_numpy(z0).cuda()
    u_tgt = tgt_plan.run(zd, steps)[0].clone()
    plan = Plan(Problem(**base))

    def loss(plan_, z):
        return float(torch.sum((plan_.run(z, steps)[0] - u_tgt) ** 2))

    zT = plan.run(zd, steps)
    lamT = torch.zeros_like(zT)
    lamT[0] = 2 * (zT[0] - u_tgt)
    lam0, dLdD = plan.adjoint(zd, lamT, steps)
    eps = 1e-6
    # along the gradient itself the directional derivative is |grad|, large
    # against the difference quotient's rounding noise (~1e-14 / 2 eps)
    d = lam0 / torch.linalg.norm(lam0)
    fd_z = (loss(plan, zd + eps * d) - loss(plan, zd - eps * d)) / (2 * eps)
    g_z = float(torch.sum(lam0 * d))
    assert abs(g_z - fd_z) <= 1e-8 * abs(fd_z), (g_z, fd_z)
    # along a random unit direction the derivative is ~1e-3 and the same
    # noise floor is ~1e-6 relative
    d = torch.from_numpy(I.unit_direction(z0.shape, 21)).cuda()
    fd_z = (loss(plan, zd + eps * d) - loss(plan, zd - eps * d)) / (2 * eps)
    g_z = float(torch.sum(lam0 * d))
    assert abs(g_z - fd_z) <= 2e-6 * abs(fd_z), (g_z, fd_z)
    fd_D = (loss(Plan(Problem(D=(1 + eps, 1.5), **base)), zd) -
            loss(Plan(Problem(D=(1 - eps, 1.5), **base)), zd)) / (2 * eps)
    assert abs(float(dLdD[0]) - fd_D) <= 1e-8 * abs(fd_D), (float(dLdD[0]), fd_D)
    # CPU reference gradient (all states stored, literal transposes)
    olam0, odLdD = O.adjoint(oracle_problem(plan.problems[0]), z0, lamT.cpu().numpy(), steps)
    assert field_rel_err(lam0.cpu().numpy(), olam0) <= 1e-8
    assert abs(float(dLdD[0]) - odLdD[0]) <= 1e-8 * abs(odLdD[0])


@pytest.mark.parametrize("flags", [1 << 1, 1 << 2])
def test_adjoint_and_tlm_other_sync_modes(cuda_ok, flags):
    """Per-stage launches and neighbour synchronisation give the same
    adjoint and tangents as the default grid barrier, bitwise."""
    import torch
    from paper_1309_1720_gb300 import Plan, RK4, STENCIL9
    p = _prob(0, 150, 97, STENCIL9, RK4)
    z0 = torch.from_numpy(_z0(p)).cuda()
    lamT = torch.from_numpy(I.unit_direction(z0.shape, 3)).cuda()
    dz = lamT[None].contiguous()
    a0, d0 = Plan(p).adjoint(z0, lamT, 21, checkpoint_every=4)
    _, t0 = Plan(p).tlm(z0, dz, 21)
    p.flags = flags
    a1, d1 = Plan(p).adjoint(z0, lamT, 21, checkpoint_every=4)
    _, t1 = Plan(p).tlm(z0, dz, 21)
    assert torch.equal(a0, a1) and torch.equal(t0, t1)
    # dL/dD: one launch per stage adds each stage's warp sums to the dL/dD
    # slots instead of each launch's, and neighbour synchronisation keeps the
    # equal-cell schedule (the grid-barrier adjoint balances its boundary
    # cost), so the same terms are associated differently
    assert torch.allclose(d0, d1, rtol=1e-10, atol=0)


def test_dLdD_bitwise_reproducible(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, RK4, STENCIL9
    p = _prob(0, 300, 200, STENCIL9, RK4)
    z0 = torch.from_numpy(_z0(p)).cuda()
    lamT = torch.from_numpy(I.unit_direction(z0.shape, 3)).cuda()
    plan = Plan(p)
    a0, d0 = plan.adjoint(z0, lamT, 30)
    a1, d1 = plan.adjoint(z0, lamT, 30)
    assert torch.equal(a0, a1) and torch.equal(d0, d1)


@pytest.mark.parametrize("model,stencil", [(0, 1), (1, 1), (3, 0)])
def test_state_only_adjoint_same_lam0(cuda_ok, model, stencil):
    """Without dLdD the adjoint skips the dL/dD accumulation and its
    reduction and returns the same dL/dz0 bit for bit, for every checkpoint
    interval; autograd takes that path when D needs no gradient."""
    import torch
    from paper_1309_1720_gb300 import Plan, RK4, autograd
    p = _prob(model, 70, 45, stencil, RK4)
    z0 = torch.from_numpy(_z0(p)).cuda()
    lamT = torch.from_numpy(I.unit_direction(z0.shape, 5)).cuda()
    plan = Plan(p)
    lam = {}
    for every in (0, 3, 12):
        a0, d0 = plan.adjoint(z0, lamT, 12, checkpoint_every=every)
        a1, d1 = plan.adjoint(z0, lamT, 12, checkpoint_every=every, with_dD=False)
        assert d1 is None and d0.shape[0] >= 1
        assert torch.equal(a0, a1)
        lam[every] = a0
    # the plan's own diffusivities, no gradient wanted
    D = torch.tensor(autograd._plan_D(plan), dtype=torch.float64, device="cuda")
    assert D.shape[0] == d0.shape[0]
    z = z0.clone().requires_grad_(True)
    autograd.flow(z, D, plan, 12).mul(lamT).sum().backward()
    assert torch.equal(z.grad, lam[0])
