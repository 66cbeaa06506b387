"""The two-variable Karma model (Eq. karma) on the GPU against the oracle:
every stencil, scheme and ghost rule on ragged shapes, the tanh variant of
Sect. 6, integer and non-integer M, tangent-linear and adjoint runs, the
linearized tangents, temporal blocking (bitwise equal to the stage kernel),
batches, and the first 100 steps of the 256 x 256 workload of the paper's
timing experiments."""
import numpy as np
import pytest

from helpers import field_rel_err, gpu_run, oracle_problem, oracle_run
from paper_1309_1720_gb300 import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _karma(nx, ny, stencil=0, scheme=2, bc=0, dt=0.05, **kw):
    from paper_1309_1720_gb300 import Problem, KARMA
    return Problem(model=KARMA, nx=nx, ny=ny, dx=I.KARMA_DX, stencil=stencil, scheme=scheme, bc=bc, dt=dt,
                   **kw)


def _state(nx, ny, seed=0):
    """A broken wave advanced a little, so u and v take intermediate values
    (front, plateau, recovery) and every branch of the model is visited."""
    z = I.karma_broken_wave(nx, ny, width=max(1, nx // 6), seed=seed)
    z[1] += 0.4 * I.uniform01(seed + 11, nx * ny).reshape(ny, nx)
    z[0] += 2.0 * (I.uniform01(seed + 12, nx * ny).reshape(ny, nx) > 0.8)
    return z


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("shape", [(67, 45), (3, 7), (2, 2), (130, 66)])
def test_karma_parity(cuda_ok, stencil, scheme, bc, shape):
    nx, ny = shape
    p = _karma(nx, ny, stencil, scheme, bc)
    z0 = _state(nx, ny)
    n = 25
    assert field_rel_err(gpu_run(p, z0, n), oracle_run(p, z0, n)) <= TOL


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 2])
def test_karma_tanh_variant(cuda_ok, stencil, scheme):
    from paper_1309_1720_gb300 import FLAG_TANH_AS_HK
    p = _karma(90, 61, stencil, scheme, flags=FLAG_TANH_AS_HK)
    z0 = _state(90, 61, seed=3)
    g = gpu_run(p, z0, 40)
    assert field_rel_err(g, oracle_run(p, z0, 40)) <= TOL
    assert field_rel_err(g, oracle_run(_karma(90, 61, stencil, scheme), z0, 40)) > 1e-6


@pytest.mark.parametrize("M", [6.0, 1.0, 0.0, 4.5, 10.0])
def test_karma_powers(cuda_ok, M):
    """v^M by repeated squaring for integer M, by pow() otherwise.  For
    M = 10 the recovery variable is scaled below 1: with v up to 1.6,
    v^10 = 110 drives u negative and the model itself (oracle included)
    blows up within the run."""
    from paper_1309_1720_gb300 import KARMA, default_params
    prm = default_params(KARMA)
    prm[6] = M
    p = _karma(77, 40, 1, 2, params=prm)
    z0 = _state(77, 40, seed=5)
    if M > 6:
        z0[1] *= 0.6
    assert field_rel_err(gpu_run(p, z0, 30), oracle_run(p, z0, 30)) <= TOL


def test_karma_anisotropic_and_tunings(cuda_ok):
    from paper_1309_1720_gb300 import FLAG_NEIGHBOR_SYNC, FLAG_PER_STAGE_LAUNCH
    z0 = _state(150, 97, seed=7)
    ref = None
    for tuning, flags in [(None, 0), (dict(cells_x=1, threads=256), 0), (None, FLAG_NEIGHBOR_SYNC),
                          (None, FLAG_PER_STAGE_LAUNCH), (dict(schedule=1, rows=4), 0)]:
        p = _karma(150, 97, 1, 2, D=(1.1e-3,), Dyy=(1.1e-3 / 4,), flags=flags)
        g = gpu_run(p, z0, 20, tuning=tuning)
        if ref is None:
            ref = g
            assert field_rel_err(g, oracle_run(p, z0, 20)) <= TOL
        assert np.array_equal(g, ref)


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_karma_tlm_adjoint(cuda_ok, stencil, scheme):
    import torch
    from paper_1309_1720_gb300 import Plan
    p = _karma(70, 45, stencil, scheme)
    z0 = _state(70, 45, seed=9)
    steps = 15
    op = oracle_problem(p)
    plan = Plan(p)
    dz0 = np.stack([I.unit_direction(z0.shape, 30 + i) for i in range(2)])
    zd = torch.from_numpy(z0).cuda()
    zT, dzT = plan.tlm(zd, torch.from_numpy(dz0).cuda(), steps)
    for i in range(2):
        assert field_rel_err(dzT[i].cpu().numpy(), O.tlm(op, z0, dz0[i], steps)[1]) <= TOL
    assert np.array_equal(zT.cpu().numpy(), plan.run(zd, steps).cpu().numpy())
    lin = plan.linearize(zd, steps, max_tangents=2)
    assert torch.equal(lin.apply(torch.from_numpy(dz0).cuda()), dzT)
    lamT = I.unit_direction(z0.shape, 78)
    lam0, dLdD = plan.adjoint(zd, torch.from_numpy(lamT).cuda(), steps)
    plan.status()
    lin.status()
    olam0, odLdD = O.adjoint(op, z0, lamT, steps)
    assert field_rel_err(lam0.cpu().numpy(), olam0) <= TOL
    assert abs(float(dLdD[0]) - odLdD[0]) <= 1e-10 * abs(odLdD[0])


@pytest.mark.parametrize("shape", [(128, 128), (67, 45), (3, 7)])
@pytest.mark.parametrize("scheme", [0, 2])
def test_karma_temporal_blocking_bitwise(cuda_ok, shape, scheme):
    nx, ny = shape
    p = _karma(nx, ny, 1, scheme)
    z0 = _state(nx, ny, seed=2)
    ref = gpu_run(p, z0, 9)
    for k in (2, 4):
        assert np.array_equal(gpu_run(p, z0, 9, tuning=dict(schedule=2, rows=k)), ref)


def test_karma_batch(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan
    shapes = [(64, 64), (33, 90), (128, 20), (5, 5)]
    probs = [_karma(nx, ny, 0, 2, D=(1.1e-3 * (1 + 0.1 * i),)) for i, (nx, ny) in enumerate(shapes)]
    states = [_state(nx, ny, seed=i) for i, (nx, ny) in enumerate(shapes)]
    plan = Plan(probs)
    outs = [g.cpu().numpy() for g in plan.unpack(plan.run(plan.pack(states), 12))]
    plan.status()
    for p, s, got in zip(probs, states, outs):
        assert np.array_equal(got, gpu_run(p, s, 12))
        assert field_rel_err(got, oracle_run(p, s, 12)) <= TOL


def test_karma_256_first_100_steps(cuda_ok):
    """The 256 x 256 grid of the paper's Karma timing runs (Figs. 3-4), RK4,
    dt = 0.05 ms, from the seeded broken wave."""
    p = _karma(256, 256, 0, 2)
    z0 = I.karma_broken_wave(256, 256, seed=0)
    assert field_rel_err(gpu_run(p, z0, 100), oracle_run(p, z0, 100)) <= TOL
