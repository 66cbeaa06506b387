"""Parity of the CUDA path with the oracle for periodic ghosts (Sect. 3), the
Rush-Larsen and implicit-Euler gate integrators of the four-field model
(Sect. 3, Table 2) and its tanh-as-smoothed-step variant (Sect. 6), all
through the C ABI.  Bound: per-field max-norm relative error 1e-12."""
import numpy as np
import pytest

from helpers import field_rel_err, gpu_run, oracle_problem, oracle_run
from paper_1309_1720_gb300 import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _fhn(nx, ny, **kw):
    from paper_1309_1720_gb300 import Problem, FHN
    base = dict(model=FHN, nx=nx, ny=ny, dx=0.04, dt=1e-4)
    base.update(kw)
    return Problem(**base)


def _bocf(nx, ny, **kw):
    from paper_1309_1720_gb300 import Problem, BOCF, STENCIL9, RK4
    base = dict(model=BOCF, nx=nx, ny=ny, dx=0.03, D=(1.171e-3,), Dyy=(1.171e-3 / 4,), stencil=STENCIL9,
                scheme=RK4, dt=0.05)
    base.update(kw)
    return Problem(**base)


# ------------------------------------------------------------ periodic ghosts
@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("shape", [(67, 45), (2, 2), (3, 7), (129, 65), (64, 32)])
def test_periodic_fhn(cuda_ok, stencil, scheme, shape):
    from paper_1309_1720_gb300 import PERIODIC
    nx, ny = shape
    p = _fhn(nx, ny, stencil=stencil, scheme=scheme, bc=PERIODIC)
    z0 = I.fhn_broken_wave(nx, ny, width=max(1, nx // 8))
    assert field_rel_err(gpu_run(p, z0, 100), oracle_run(p, z0, 100)) <= TOL


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 2])
def test_periodic_bocf(cuda_ok, stencil, scheme):
    from paper_1309_1720_gb300 import PERIODIC
    p = _bocf(77, 41, stencil=stencil, scheme=scheme, bc=PERIODIC)
    z0 = I.bocf_spiral_cores(77, 41, n_cores=3)
    assert field_rel_err(gpu_run(p, z0, 40), oracle_run(p, z0, 40)) <= TOL


@pytest.mark.parametrize("tuning", [dict(cells_x=1, threads=128), dict(cells_x=2, threads=256, blocks_per_sm=2),
                                    dict(cells_x=1, rows=3, threads=512, schedule=1),
                                    dict(cells_x=2, rows=5, threads=128, schedule=1)])
@pytest.mark.parametrize("flags", [0, 1 << 1, 1 << 2])
def test_periodic_tunings_and_modes(cuda_ok, tuning, flags):
    """Every launch shape and synchronisation mode (neighbour waits fall
    back to the grid barrier under periodic ghosts)."""
    from paper_1309_1720_gb300 import PERIODIC, RK4, STENCIL9
    p = _fhn(150, 97, stencil=STENCIL9, scheme=RK4, bc=PERIODIC, dt=2e-4, flags=flags)
    z0 = I.fhn_broken_wave(150, 97, width=20)
    assert field_rel_err(gpu_run(p, z0, 60, tuning=tuning), oracle_run(p, z0, 60)) <= TOL


@pytest.mark.parametrize("model", [0, 1])
def test_periodic_translation_bitwise(cuda_ok, model):
    """Every cell of a periodic grid sees the same arithmetic on the GPU
    too: a rolled state steps to the rolled result bit for bit."""
    from paper_1309_1720_gb300 import PERIODIC, RK4, STENCIL9
    n = 96
    if model == 0:
        p = _fhn(n, n, stencil=STENCIL9, scheme=RK4, bc=PERIODIC)
        z0 = I.fhn_broken_wave(n, n, width=12)
    else:
        p = _bocf(n, n, bc=PERIODIC)
        z0 = I.bocf_spiral_cores(n, n, n_cores=2)
    base = gpu_run(p, z0, 30)
    for sy, sx in [(0, 33), (17, 0), (5, 64)]:
        zr = np.ascontiguousarray(np.roll(z0, (sy, sx), axis=(1, 2)))
        assert np.array_equal(gpu_run(p, zr, 30), np.roll(base, (sy, sx), axis=(1, 2)))


@pytest.mark.parametrize("model", [0, 1])
def test_periodic_tlm_and_adjoint(cuda_ok, model):
    import torch
    from paper_1309_1720_gb300 import Plan, PERIODIC
    if model == 0:
        p = _fhn(70, 45, stencil=1, scheme=2, bc=PERIODIC, dt=2e-4)
        z0 = I.fhn_broken_wave(70, 45, width=6)
    else:
        p = _bocf(70, 45, bc=PERIODIC)
        z0 = I.bocf_spiral_cores(70, 45, n_cores=2)
    steps = 15
    op = oracle_problem(p)
    plan = Plan(p)
    dz0 = np.stack([I.unit_direction(z0.shape, 50 + i) for i in range(2)])
    _, dzT = plan.tlm(torch.from_numpy(z0).cuda(), torch.from_numpy(dz0).cuda(), steps)
    for i in range(2):
        assert field_rel_err(dzT[i].cpu().numpy(), O.tlm(op, z0, dz0[i], steps)[1]) <= TOL
    lamT = I.unit_direction(z0.shape, 77)
    lam0, dLdD = plan.adjoint(torch.from_numpy(z0).cuda(), torch.from_numpy(lamT).cuda(), steps)
    plan.status()
    olam0, odLdD = O.adjoint(op, z0, lamT, steps)
    assert field_rel_err(lam0.cpu().numpy(), olam0) <= TOL
    g = dLdD.cpu().numpy()
    assert np.all(np.abs(g - odLdD[:len(g)]) <= 1e-10 * np.abs(odLdD[:len(g)]))


# ------------------------------------------------------------ gate integrators
@pytest.mark.parametrize("scheme", [3, 4])
@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shape", [(77, 41), (3, 7), (130, 66)])
def test_gate_integrators(cuda_ok, scheme, stencil, bc, shape):
    nx, ny = shape
    p = _bocf(nx, ny, stencil=stencil, scheme=scheme, bc=bc, dt=0.05)
    z0 = I.bocf_spiral_cores(nx, ny, n_cores=3)
    assert field_rel_err(gpu_run(p, z0, 100), oracle_run(p, z0, 100)) <= TOL


@pytest.mark.parametrize("scheme", [3, 4])
@pytest.mark.parametrize("tuning", [dict(cells_x=1, threads=128, blocks_per_sm=4, schedule=1, rows=2),
                                    dict(cells_x=2, threads=512), dict(cells_x=1, threads=256)])
@pytest.mark.parametrize("flags", [0, 1 << 1, 1 << 2, 1 << 3])
def test_gate_integrators_tunings_modes_variant(cuda_ok, scheme, tuning, flags):
    """Launch shapes, launch and synchronisation modes, and the tanh variant
    (flag 1 << 3) with the gate integrators; dt = 0.15 ms, three times the
    explicit runs' step."""
    p = _bocf(150, 97, scheme=scheme, dt=0.15, flags=flags)
    z0 = I.bocf_spiral_cores(150, 97, n_cores=4, seed=5)
    assert field_rel_err(gpu_run(p, z0, 40, tuning=tuning), oracle_run(p, z0, 40)) <= TOL


def test_gate_integrators_batch(cuda_ok):
    """A batch of uneven four-field instances with Rush-Larsen equals the
    oracle instance by instance."""
    import torch
    from paper_1309_1720_gb300 import Plan, RUSH_LARSEN
    sizes = [(70, 33), (3, 5), (129, 64), (40, 40)]
    probs = [_bocf(nx, ny, scheme=RUSH_LARSEN, D=(1.171e-3 * (1 + 0.1 * i),), Dyy=(1.171e-3 / 4,))
             for i, (nx, ny) in enumerate(sizes)]
    z0s = [I.bocf_spiral_cores(nx, ny, n_cores=2, seed=i) for i, (nx, ny) in enumerate(sizes)]
    plan = Plan(probs)
    out = plan.run(plan.pack([torch.from_numpy(z).cuda() for z in z0s]), 30)
    plan.status()
    for p, z0, g in zip(probs, z0s, plan.unpack(out)):
        assert field_rel_err(g.cpu().numpy(), oracle_run(p, z0, 30)) <= TOL


def test_gate_integrators_have_no_tangents(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import CGError, Plan, IMPLICIT_EULER
    p = _bocf(40, 30, scheme=IMPLICIT_EULER)
    plan = Plan(p)
    z = torch.from_numpy(I.bocf_spiral_cores(40, 30)).cuda()
    with pytest.raises(CGError):
        plan.tlm(z, z.clone()[None], 3)
    with pytest.raises(CGError):
        plan.adjoint(z, z.clone(), 3)


# ---------------------------------------------------- tanh as smoothed step
@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_tanh_variant(cuda_ok, stencil, scheme):
    from paper_1309_1720_gb300 import FLAG_TANH_AS_HK
    p = _bocf(130, 66, stencil=stencil, scheme=scheme, flags=FLAG_TANH_AS_HK)
    z0 = I.bocf_spiral_cores(130, 66, n_cores=3)
    g = gpu_run(p, z0, 60)
    assert field_rel_err(g, oracle_run(p, z0, 60)) <= TOL
    # and it is a different model
    from paper_1309_1720_gb300 import Problem
    q = _bocf(130, 66, stencil=stencil, scheme=scheme)
    assert field_rel_err(g, oracle_run(q, z0, 60)) > 1e-6


def test_tanh_variant_tlm_and_adjoint(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, FLAG_TANH_AS_HK
    p = _bocf(70, 45, flags=FLAG_TANH_AS_HK)
    z0 = I.bocf_spiral_cores(70, 45, n_cores=2)
    steps = 15
    op = oracle_problem(p)
    plan = Plan(p)
    dz0 = I.unit_direction(z0.shape, 60)[None].copy()
    _, dzT = plan.tlm(torch.from_numpy(z0).cuda(), torch.from_numpy(dz0).cuda(), steps)
    assert field_rel_err(dzT[0].cpu().numpy(), O.tlm(op, z0, dz0[0], steps)[1]) <= TOL
    lamT = I.unit_direction(z0.shape, 78)
    lam0, dLdD = plan.adjoint(torch.from_numpy(z0).cuda(), torch.from_numpy(lamT).cuda(), steps)
    plan.status()
    olam0, odLdD = O.adjoint(op, z0, lamT, steps)
    assert field_rel_err(lam0.cpu().numpy(), olam0) <= TOL
    assert abs(float(dLdD[0]) - odLdD[0]) <= 1e-10 * abs(odLdD[0])
