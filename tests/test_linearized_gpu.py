"""Linearized tangent-linear runs: one run keeps every stage's local
Jacobian, later runs advance tangents alone with them.  The tangents must
equal those of the ordinary tangent-linear run (which recomputes the primal)
bit for bit, the linearizing run's state must equal a plain run bit for bit,
and the GMRES Newton step and the periodic-orbit solver built on it must give
the same iterates as without it."""
import numpy as np
import pytest

from helpers import field_rel_err, oracle_problem
from paper_1309_1720_gb300 import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


def _prob(model, nx, ny, stencil, scheme, **kw):
    from paper_1309_1720_gb300 import Problem, FHN, BOCF
    if model == FHN:
        return Problem(model=FHN, nx=nx, ny=ny, dx=0.04, stencil=stencil, scheme=scheme, dt=2e-4, **kw)
    if model == BOCF:
        return Problem(model=BOCF, nx=nx, ny=ny, dx=0.03, D=(1.171e-3,), Dyy=(1.171e-3 / 4,), stencil=stencil,
                       scheme=scheme, dt=0.05, **kw)
    return Problem(model=3, nx=nx, ny=ny, dx=0.1, D=(1.0,), Dyy=(0.6,), stencil=stencil, scheme=scheme, dt=1e-3,
                   **kw)


def _z0(model, nx, ny):
    if model == 0:
        return I.fhn_broken_wave(nx, ny, width=max(1, nx // 8))
    if model == 1:
        return I.bocf_spiral_cores(nx, ny, n_cores=2)
    return (1.0 + 0.3 * I.uniform_pm1(9, nx * ny)).reshape(1, ny, nx)


@pytest.mark.parametrize("model", [0, 1, 3])
@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_apply_equals_tlm_bitwise(cuda_ok, model, stencil, scheme):
    import torch
    from paper_1309_1720_gb300 import Plan
    nx, ny, steps, T = 77, 41, 13, 3
    p = _prob(model, nx, ny, stencil, scheme)
    z0 = torch.from_numpy(_z0(model, nx, ny)).cuda()
    dz0 = torch.from_numpy(np.stack([I.unit_direction(tuple(z0.shape), 50 + i) for i in range(T)])).cuda()
    plan = Plan(p)
    zT, dzT = plan.tlm(z0, dz0, steps)
    lin = plan.linearize(z0, steps, max_tangents=T)
    assert torch.equal(lin.zT, zT)
    assert torch.equal(lin.zT, plan.run(z0, steps))
    got = lin.apply(dz0)
    assert torch.equal(got, dzT)
    # the stored Jacobians survive applications and other runs of the plan
    plan.run(z0, 3)
    assert torch.equal(lin.apply(dz0[1:2].contiguous())[0], dzT[1])
    lin.status()
    plan.status()


def test_apply_matches_oracle_and_variants(cuda_ok):
    """A ragged BOCF grid with the tanh-as-H_k variant and periodic ghosts,
    against the oracle's tangent-linear model to 1e-12."""
    import torch
    from paper_1309_1720_gb300 import Plan, BOCF, PERIODIC, RK4, STENCIL9, FLAG_TANH_AS_HK
    nx, ny, steps = 53, 29, 9
    p = _prob(BOCF, nx, ny, STENCIL9, RK4, bc=PERIODIC, flags=FLAG_TANH_AS_HK)
    z0 = _z0(BOCF, nx, ny)
    dz0 = I.unit_direction(z0.shape, 7)
    plan = Plan(p)
    lin = plan.linearize(torch.from_numpy(z0).cuda(), steps)
    got = lin.apply(torch.from_numpy(dz0[None].copy()).cuda())[0].cpu().numpy()
    lin.status()
    oz, odz = O.tlm(oracle_problem(p), z0, dz0, steps)
    assert field_rel_err(got, odz) <= 1e-12
    assert field_rel_err(lin.zT.cpu().numpy(), oz) <= 1e-12


@pytest.mark.parametrize("mode", ["per_stage", "neighbor"])
def test_apply_launch_modes(cuda_ok, mode):
    import torch
    from paper_1309_1720_gb300 import Plan, FHN, RK4, STENCIL9, FLAG_PER_STAGE_LAUNCH, FLAG_NEIGHBOR_SYNC
    flags = {"per_stage": FLAG_PER_STAGE_LAUNCH, "neighbor": FLAG_NEIGHBOR_SYNC}[mode]
    nx, ny, steps = 200, 90, 11
    z0 = torch.from_numpy(_z0(FHN, nx, ny)).cuda()
    dz0 = torch.from_numpy(I.unit_direction(tuple(z0.shape), 3)[None].copy()).cuda()
    ref = Plan(_prob(FHN, nx, ny, STENCIL9, RK4)).tlm(z0, dz0, steps)[1]
    lin = Plan(_prob(FHN, nx, ny, STENCIL9, RK4, flags=flags)).linearize(z0, steps)
    assert torch.equal(lin.apply(dz0), ref)
    lin.status()


def test_apply_in_place_and_zero_steps(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, FHN, HEUN, STENCIL5
    nx, ny = 64, 48
    p = _prob(FHN, nx, ny, STENCIL5, HEUN)
    plan = Plan(p)
    z0 = torch.from_numpy(_z0(FHN, nx, ny)).cuda()
    dz0 = torch.from_numpy(np.stack([I.unit_direction(tuple(z0.shape), 11 + i) for i in range(2)])).cuda()
    ref = plan.tlm(z0, dz0, 6)[1]
    lin = plan.linearize(z0, 6, max_tangents=2)
    d = dz0.clone()
    lin.apply(d, dzT=d)
    assert torch.equal(d, ref)
    lin0 = plan.linearize(z0, 0, max_tangents=2)
    assert torch.equal(lin0.zT, z0)
    assert torch.equal(lin0.apply(dz0), dz0)
    lin.status()


def test_linearized_rejections(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import CGError, Plan, BOCF, FHN, RUSH_LARSEN, EULER, STENCIL5
    z = torch.from_numpy(_z0(BOCF, 32, 32)).cuda()
    with pytest.raises(CGError):
        Plan(_prob(BOCF, 32, 32, STENCIL5, RUSH_LARSEN)).linearize(z, 4)
    with pytest.raises(CGError):
        Plan([_prob(FHN, 32, 32, STENCIL5, EULER)] * 2).linearize(torch.zeros(2, 2, 32, 32, dtype=torch.float64).cuda(), 4)
    zf = torch.from_numpy(_z0(FHN, 32, 32)).cuda()
    lin = Plan(_prob(FHN, 32, 32, STENCIL5, EULER)).linearize(zf, 4)
    d = zf[None].clone()
    with pytest.raises(CGError):                     # Euler tangents cannot run in place
        lin.apply(d, dzT=d)


@pytest.mark.parametrize("model", [0, 3])
def test_newton_step_linearized_bitwise(cuda_ok, model):
    """Small grid (the Krylov space spans the state) and 256^2 GMRES(10):
    the linearized Newton step returns the same dz and residual history."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, DIFFUSION, RK4
    if model == FHN:
        p = Problem(model=FHN, nx=6, ny=5, dx=0.5, scheme=RK4, dt=0.01)
        z0 = I.fhn_broken_wave(6, 5, width=2)
    else:
        p = Problem(model=DIFFUSION, nx=6, ny=5, dx=0.5, D=(1.0,), scheme=RK4, dt=0.01)
        z0 = (1.0 + 0.3 * I.uniform_pm1(4, 30)).reshape(1, 5, 6)
    plan = Plan(p)
    zd = torch.from_numpy(z0).cuda()
    a, ha = plan.newton_step(zd, 40, restart=z0.size, max_restarts=1, rtol=1e-13)
    b, hb = plan.newton_step(zd, 40, restart=z0.size, max_restarts=1, rtol=1e-13, linearized=True)
    assert torch.equal(a, b) and ha == hb
    n = 256
    q = Problem(model=FHN, nx=n, ny=n, dx=0.04, scheme=RK4, dt=2.5e-4)
    zq = torch.from_numpy(I.fhn_broken_wave(n, n, seed=0)).cuda()
    pq = Plan(q)
    a, ha = pq.newton_step(zq, 60, restart=10, max_restarts=2, rtol=1e-12)
    b, hb = pq.newton_step(zq, 60, restart=10, max_restarts=2, rtol=1e-12, linearized=True)
    assert torch.equal(a, b) and ha == hb
    pq.status()


def test_periodic_orbit_linearized_same_iterates(cuda_ok):
    """Two Newton iterations of the travelling-pulse orbit search on a 256 x 2
    periodic ring, with and without stored Jacobians: identical iterates."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, PERIODIC, RK4
    from paper_1309_1720_gb300.newton import periodic_orbit
    nx, ny, dt = 256, 2, 0.05
    base = Problem(model=FHN, nx=nx, ny=ny, dx=0.5, bc=PERIODIC, scheme=RK4, dt=dt)
    z = np.empty((2, ny, nx))
    z[0] = I.FHN_U_REST
    z[1] = I.FHN_V_REST
    z[0, :, 10:20] = 1.0
    z[1, :, 0:10] = 0.6
    z[1, :, -30:] = 0.6
    z1 = Plan(base).run(torch.from_numpy(z).cuda(), 4000)
    T0, n = 230.0, 4600
    za, Ta, ha = periodic_orbit(base, z1, T0, n, max_newton=2, linearized=False)
    zb, Tb, hb = periodic_orbit(base, z1, T0, n, max_newton=2, linearized=True)
    assert torch.equal(za, zb) and Ta == Tb and ha == hb


def test_apply_needs_a_linearized_workspace(cuda_ok):
    """cg_tlm_apply refuses a workspace the plan never linearized, or one
    linearized over another step count."""
    import ctypes
    import torch
    from paper_1309_1720_gb300 import Plan, FHN, RK4, STENCIL5, _lib
    L = _lib.lib()
    plan = Plan(_prob(FHN, 40, 30, STENCIL5, RK4))
    z0 = torch.from_numpy(_z0(FHN, 40, 30)).cuda()
    dz = z0[None].clone()
    sz = ctypes.c_size_t()
    assert L.cg_tlm_linearized_workspace_size(plan.handle, 1, 5, ctypes.byref(sz)) == 0
    ws = torch.zeros(int(sz.value), dtype=torch.uint8, device="cuda")
    out = torch.empty_like(dz)
    assert L.cg_tlm_apply(plan.handle, dz.data_ptr(), out.data_ptr(), 1, 5, ws.data_ptr(), None) == 1
    zT = torch.empty_like(z0)
    assert L.cg_tlm_linearize(plan.handle, z0.data_ptr(), zT.data_ptr(), 5, ws.data_ptr(), None) == 0
    assert L.cg_tlm_apply(plan.handle, dz.data_ptr(), out.data_ptr(), 1, 4, ws.data_ptr(), None) == 1
    assert L.cg_tlm_apply(plan.handle, dz.data_ptr(), out.data_ptr(), 1, 5, ws.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert torch.equal(out, plan.tlm(z0, dz, 5)[1])
