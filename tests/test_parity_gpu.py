"""Parity of the CUDA stepper (through the C ABI) with the CPU oracle.

Metric: per field max|gpu - oracle| / max|oracle| (the max-norm relative
error), bound 1e-12 after up to 100 steps: the two sides differ only in FMA
contraction, summation order and libm-vs-CUDA transcendental rounding.
"""
import numpy as np
import pytest

from helpers import field_rel_err, gpu_run, oracle_problem, oracle_run
from paper_1309_1720_gb300 import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _fhn(nx, ny, **kw):
    from paper_1309_1720_gb300 import Problem, FHN
    base = dict(model=FHN, nx=nx, ny=ny, dx=0.04, dt=2e-4)
    base.update(kw)
    return Problem(**base)


def _bocf(nx, ny, **kw):
    from paper_1309_1720_gb300 import Problem, BOCF, STENCIL9, RK4
    base = dict(model=BOCF, nx=nx, ny=ny, dx=0.03, D=(1.171e-3,), Dyy=(1.171e-3 / 4,),
                stencil=STENCIL9, scheme=RK4, dt=0.05)
    base.update(kw)
    return Problem(**base)


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("shape", [(67, 45), (2, 2), (3, 7), (129, 65)])
def test_fhn_matrix(cuda_ok, stencil, scheme, bc, shape):
    nx, ny = shape
    p = _fhn(nx, ny, stencil=stencil, scheme=scheme, bc=bc, dt=1e-4)
    z0 = I.fhn_broken_wave(nx, ny, width=max(1, nx // 8))
    n = 100
    g = gpu_run(p, z0, n)
    o = oracle_run(p, z0, n)
    assert field_rel_err(g, o) <= TOL


@pytest.mark.parametrize("tuning", [
    dict(cells_x=1, rows=1, threads=128, schedule=1), dict(cells_x=2, rows=3, threads=512, schedule=1),
    dict(cells_x=1, rows=16, threads=256, blocks_per_sm=1, schedule=1), dict(cells_x=2, rows=64, threads=128, schedule=1),
    dict(cells_x=1, threads=256), dict(cells_x=2, threads=128, blocks_per_sm=2), dict(cells_x=1, threads=512),
])
@pytest.mark.parametrize("mode", ["barrier", "per_stage", "neighbor"])
def test_fhn_tunings_and_launch_modes(cuda_ok, tuning, mode):
    from paper_1309_1720_gb300 import FLAG_PER_STAGE_LAUNCH, FLAG_NEIGHBOR_SYNC, RK4, STENCIL9
    flags = {"barrier": 0, "per_stage": FLAG_PER_STAGE_LAUNCH, "neighbor": FLAG_NEIGHBOR_SYNC}[mode]
    p = _fhn(150, 97, stencil=STENCIL9, scheme=RK4, dt=2e-4, flags=flags)
    z0 = I.fhn_broken_wave(150, 97, width=20)
    g = gpu_run(p, z0, 60, tuning=tuning)
    o = oracle_run(p, z0, 60)
    assert field_rel_err(g, o) <= TOL


@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("n", [0, 1, 2, 7])
def test_in_place_and_step_counts(cuda_ok, scheme, n):
    p = _fhn(70, 33, scheme=scheme, dt=1e-4)
    z0 = I.fhn_broken_wave(70, 33, width=9)
    g = gpu_run(p, z0, n, inplace=True)
    o = oracle_run(p, z0, n)
    if n == 0:
        assert np.array_equal(g, z0)
    else:
        assert field_rel_err(g, o) <= TOL


@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("bc", [0, 1])
def test_bocf_matrix(cuda_ok, stencil, scheme, bc):
    nx, ny = 77, 41
    p = _bocf(nx, ny, stencil=stencil, scheme=scheme, bc=bc)
    z0 = I.bocf_spiral_cores(nx, ny, n_cores=3)
    g = gpu_run(p, z0, 100)
    o = oracle_run(p, z0, 100)
    assert field_rel_err(g, o) <= TOL


def test_c1_full_run(cuda_ok):
    """128^2 two-field model, 5-point, mirror, explicit Euler, dt 2e-4,
    1000 steps from the seeded broken wave: the whole run."""
    p = _fhn(128, 128, dt=2e-4)
    z0 = I.fhn_broken_wave(128, 128, seed=0)
    g = gpu_run(p, z0, 1000)
    o = oracle_run(p, z0, 1000)
    assert field_rel_err(g, o) <= TOL


def test_c2_first_100_steps(cuda_ok):
    """1024^2 two-field model, 9-point isotropic, RK4, dt 4e-4: first 100
    steps against the oracle on the full grid."""
    from paper_1309_1720_gb300 import RK4, STENCIL9
    p = _fhn(1024, 1024, stencil=STENCIL9, scheme=RK4, dt=4e-4)
    z0 = I.fhn_broken_wave(1024, 1024, seed=0)
    g = gpu_run(p, z0, 100)
    o = oracle_run(p, z0, 100)
    assert field_rel_err(g, o) <= TOL


def test_c3_sampled_windows_100_steps(cuda_ok):
    """2048^2 four-field model, anisotropic 9-point, RK4, the first 100 steps
    of the 5000-step workload, with the library's default launch shape, the
    tile-queue shapes the autotuner chooses among for the bench and
    neighbour-only synchronisation: the oracle recomputes windows whose margin (4 cells
    per step: one per RK stage) covers the domain of dependence, so each
    window's interior is exact; windows at the four corners, on the edges
    and in the interior (six oracle runs in parallel threads)."""
    import threading
    from paper_1309_1720_gb300 import FLAG_NEIGHBOR_SYNC
    n, steps, w = 2048, 100, 32
    p = _bocf(n, n)
    z0 = I.bocf_spiral_cores(n, n, seed=0)
    margin = 4 * steps + 2
    corners = [(0, 0), (0, 1000), (1000, 0), (900, 1300), (n - w, n - w), (0, n - w)]
    ref = {}

    def oracle_window(y0, x0):
        ys, xs = max(0, y0 - margin), max(0, x0 - margin)
        ye, xe = min(n, y0 + w + margin), min(n, x0 + w + margin)
        sub = np.ascontiguousarray(z0[:, ys:ye, xs:xe])
        o = oracle_run(_bocf(xe - xs, ye - ys), sub, steps)
        ref[(y0, x0)] = o[:, y0 - ys:y0 - ys + w, x0 - xs:x0 - xs + w].copy()
    threads = [threading.Thread(target=oracle_window, args=c) for c in corners]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert len(ref) == len(corners)
    shapes = [(p, None)] + [(p, dict(cells_x=1, threads=thr, blocks_per_sm=bps, schedule=1, rows=r))
                            for thr, bps, r in ((512, 1, 4), (512, 1, 8), (512, 1, 16), (256, 2, 8))] + \
             [(_bocf(n, n, flags=FLAG_NEIGHBOR_SYNC), dict(cells_x=2, threads=256, blocks_per_sm=2, schedule=0))]
    for q, tuning in shapes:
        g = gpu_run(q, z0, steps, tuning=tuning)
        for (y0, x0) in corners:
            assert field_rel_err(g[:, y0:y0 + w, x0:x0 + w], ref[(y0, x0)]) <= TOL, (tuning, y0, x0)


def test_diffusion_fourier_mode(cuda_ok):
    """Closed form on the GPU path: a cosine mode decays by G(dt lambda)^n."""
    import math
    from paper_1309_1720_gb300 import Problem, DIFFUSION, RK4, STENCIL9
    nx, ny, h = 200, 150, 0.1
    tx, ty = math.pi * 5 / (nx - 1), math.pi * 3 / (ny - 1)
    u0 = np.outer(np.cos(ty * np.arange(ny)), np.cos(tx * np.arange(nx)))[None].copy()
    a, b = 1.0 / h ** 2, 0.5 / h ** 2
    kappa = (1 / 6) * (a + b) / 2
    ex, ey = 2 * math.cos(tx) - 2, 2 * math.cos(ty) - 2
    lam = a * ex + b * ey + kappa * ex * ey
    dt = 0.002
    p = Problem(model=DIFFUSION, nx=nx, ny=ny, dx=h, D=(1.0,), Dyy=(0.5,), stencil=STENCIL9, scheme=RK4, dt=dt)
    g = gpu_run(p, u0, 50)
    z = dt * lam
    G = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    assert np.max(np.abs(g - G ** 50 * u0)) <= 1e-13


def test_reflection_symmetry_bitwise(cuda_ok):
    """x- and y-flips of a symmetric state stay bitwise symmetric on the GPU
    (the kernel sums mirror-image neighbours in pairs)."""
    from paper_1309_1720_gb300 import RK4, STENCIL9
    n = 96
    r = I.uniform01(3, n * n).reshape(n, n)
    base = r + r[:, ::-1]
    base = base + base[::-1, :]
    z = np.stack([0.4 * base - 0.5, 0.1 * base])
    for st in (0, 1):
        g = gpu_run(_fhn(n, n, stencil=st, scheme=RK4, dt=2e-4), z, 50)
        assert np.array_equal(g, g[:, :, ::-1])
        assert np.array_equal(g, g[:, ::-1, :])


def test_status_nonfinite(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, DEV_NONFINITE, CGError
    p = _fhn(64, 64)
    z0 = I.fhn_broken_wave(64, 64)
    z0[0, 10, 10] = np.nan
    plan = Plan(p)
    out = plan.run(torch.from_numpy(z0).cuda(), 5)
    with pytest.raises(CGError) as ei:
        plan.status()
    assert ei.value.status == 5
    assert plan.status(raise_on_error=False) & DEV_NONFINITE
    # the next clean run clears the word
    plan.run(torch.from_numpy(I.fhn_broken_wave(64, 64)).cuda(), 5, out=out)
    assert plan.status() == 0


def test_barrier_timeout_reports_status(cuda_ok):
    """The testing knob makes the first grid barrier wait for a block that
    does not exist; the bounded wait gives up after 0.2 s, every block
    returns, the status word says CG_DEV_TIMEOUT and the context stays usable."""
    import torch
    from paper_1309_1720_gb300 import Plan, FLAG_TEST_STUCK_BARRIER, DEV_TIMEOUT, CGError, RK4
    p = _fhn(64, 64, scheme=RK4, flags=FLAG_TEST_STUCK_BARRIER, barrier_timeout_s=0.2)
    plan = Plan(p)
    plan.run(torch.from_numpy(I.fhn_broken_wave(64, 64)).cuda(), 3)
    with pytest.raises(CGError) as ei:
        plan.status()
    assert ei.value.status == 6
    assert plan.status(raise_on_error=False) & DEV_TIMEOUT
    # context still usable
    q = _fhn(64, 64, scheme=RK4)
    g = gpu_run(q, I.fhn_broken_wave(64, 64), 3)
    o = oracle_run(q, I.fhn_broken_wave(64, 64), 3)
    assert field_rel_err(g, o) <= TOL


@pytest.mark.parametrize("scheme", [0, 2])
@pytest.mark.parametrize("tho", [0.02, 0.0061])
def test_bocf_distinct_switch_thresholds(cuda_ok, scheme, tho):
    """Constants with theta_o != theta_v^- (0.006): the plan evaluates the
    v^- and o switches apart (it shares them only when the two switch
    constants are equal bit for bit).  Forward, tangent-linear and adjoint
    against the oracle on a ragged grid, 1e-12."""
    import torch
    from paper_1309_1720_gb300 import Plan, BOCF, default_params
    prm = default_params(BOCF)
    prm[5] = tho
    p = _bocf(67, 45, params=prm, scheme=scheme)
    z0 = I.bocf_spiral_cores(67, 45, n_cores=2)
    op = oracle_problem(p)
    assert field_rel_err(gpu_run(p, z0, 60), O.step(op, z0, 60)) <= TOL
    plan = Plan(p)
    dz0 = I.unit_direction(z0.shape, 41)
    zT, dzT = plan.tlm(torch.from_numpy(z0).cuda(), torch.from_numpy(dz0[None].copy()).cuda(), 20)
    plan.status()
    assert field_rel_err(dzT[0].cpu().numpy(), O.tlm(op, z0, dz0, 20)[1]) <= TOL
    lamT = I.unit_direction(z0.shape, 42)
    lam0, _ = plan.adjoint(torch.from_numpy(z0).cuda(), torch.from_numpy(lamT).cuda(), 20)
    plan.status()
    assert field_rel_err(lam0.cpu().numpy(), O.adjoint(op, z0, lamT, 20)[0]) <= TOL
