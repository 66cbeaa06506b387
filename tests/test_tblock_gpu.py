"""Temporally blocked stepping (tuning schedule 2): each block advances its
tiles (of one instance or of a batch) with a halo through k steps in shared
memory between grid barriers.
Its results must equal the stage kernel's bit for bit (same per-cell
arithmetic) and the oracle's to 1e-12, for every model, stencil, explicit
scheme and ghost rule, on ragged shapes, with step counts that leave a
partial last pass, in place, and with the device-side checks."""
import numpy as np
import pytest

from helpers import field_rel_err, oracle_run
from paper_1309_1720_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _problem(model, nx, ny, stencil, scheme, bc):
    from paper_1309_1720_gb300 import Problem, FHN, BOCF
    if model == FHN:
        return Problem(model=FHN, nx=nx, ny=ny, dx=0.04, stencil=stencil, scheme=scheme, bc=bc, dt=1e-4)
    if model == BOCF:
        return Problem(model=BOCF, nx=nx, ny=ny, dx=0.03, D=(1.171e-3,), Dyy=(1.171e-3 / 4,), stencil=stencil,
                       scheme=scheme, bc=bc, dt=0.05)
    return Problem(model=3, nx=nx, ny=ny, dx=0.1, D=(1.0,), Dyy=(0.6,), stencil=stencil, scheme=scheme, bc=bc,
                   dt=1e-3)


def _state(model, nx, ny):
    if model == 0:
        return I.fhn_broken_wave(nx, ny, width=max(1, nx // 8))
    if model == 1:
        return I.bocf_spiral_cores(nx, ny, n_cores=2)
    return (1.0 + 0.3 * I.uniform_pm1(9, nx * ny)).reshape(1, ny, nx)


def _run(p, z0, n, tuning=None, inplace=False):
    import torch
    from paper_1309_1720_gb300 import Plan
    plan = Plan(p, tuning=tuning)
    z = torch.from_numpy(np.ascontiguousarray(z0)).cuda()
    out = plan.run(z, n, out=z if inplace else None)
    plan.status()
    return out.cpu().numpy()


@pytest.mark.parametrize("model", [0, 1, 3])
@pytest.mark.parametrize("stencil", [0, 1])
@pytest.mark.parametrize("scheme", [0, 1, 2])
@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("shape", [(128, 128), (67, 45), (3, 7), (2, 2), (512, 2)])
def test_tblock_bitwise_and_oracle(cuda_ok, model, stencil, scheme, bc, shape):
    nx, ny = shape
    p = _problem(model, nx, ny, stencil, scheme, bc)
    z0 = _state(model, nx, ny)
    n = 7
    ref = _run(p, z0, n)
    for k in (1, 2, 3):
        g = _run(p, z0, n, tuning=dict(schedule=2, rows=k, threads=256))
        assert np.array_equal(g, ref), k
    assert field_rel_err(ref, oracle_run(p, z0, n)) <= TOL


@pytest.mark.parametrize("k", [1, 2, 4])
@pytest.mark.parametrize("n", [0, 1, 2, 5, 8])
def test_tblock_in_place_and_step_counts(cuda_ok, k, n):
    from paper_1309_1720_gb300 import FHN, RK4, STENCIL9
    p = _problem(FHN, 70, 33, STENCIL9, RK4, 0)
    z0 = _state(FHN, 70, 33)
    ref = _run(p, z0, n)
    assert np.array_equal(_run(p, z0, n, tuning=dict(schedule=2, rows=k), inplace=True), ref)
    assert np.array_equal(_run(p, z0, n, tuning=dict(schedule=2, rows=k, threads=128)), ref)


def test_tblock_c1_full_run(cuda_ok):
    """The 128^2 explicit-Euler workload, 1000 steps, 4 steps per pass."""
    from paper_1309_1720_gb300 import FHN
    p = _problem(FHN, 128, 128, 0, 0, 0)
    p.dt = 2e-4
    z0 = I.fhn_broken_wave(128, 128, seed=0)
    g = _run(p, z0, 1000, tuning=dict(schedule=2, rows=4))
    assert np.array_equal(g, _run(p, z0, 1000))
    assert field_rel_err(g, oracle_run(p, z0, 1000)) <= TOL


def test_tblock_rejections(cuda_ok):
    from paper_1309_1720_gb300 import CGError, Plan, FHN, BOCF, PERIODIC, RUSH_LARSEN
    with pytest.raises(CGError):
        Plan(_problem(FHN, 64, 64, 0, 2, PERIODIC), tuning=dict(schedule=2, rows=2))
    with pytest.raises(CGError):
        Plan(_problem(BOCF, 64, 64, 0, RUSH_LARSEN, 0), tuning=dict(schedule=2, rows=2))
    with pytest.raises(CGError):                      # tile and halo exceed shared memory
        Plan(_problem(BOCF, 2048, 2048, 1, 2, 0), tuning=dict(schedule=2, rows=8))


def test_tblock_plan_keeps_tangents_and_adjoint(cuda_ok):
    """A plan tuned for temporal blocking still runs the tangent-linear and
    adjoint kernels (with the default launch shape)."""
    import torch
    from paper_1309_1720_gb300 import Plan, FHN
    p = _problem(FHN, 96, 80, 1, 2, 0)
    z0 = torch.from_numpy(_state(FHN, 96, 80)).cuda()
    dz = torch.from_numpy(I.unit_direction(z0.shape, 3)[None].copy()).cuda()
    a, b = Plan(p), Plan(p, tuning=dict(schedule=2, rows=2))
    for x, y in zip(a.tlm(z0, dz, 6), b.tlm(z0, dz, 6)):
        assert torch.equal(x, y)
    for x, y in zip(a.adjoint(z0, z0.clone(), 6), b.adjoint(z0, z0.clone(), 6)):
        assert torch.equal(x, y)


def test_tblock_device_checks(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import CGError, Plan, FHN, FLAG_TEST_STUCK_BARRIER
    p = _problem(FHN, 64, 64, 0, 2, 0)
    z0 = _state(FHN, 64, 64)
    z0[0, 10, 10] = np.nan
    plan = Plan(p, tuning=dict(schedule=2, rows=2))
    plan.run(torch.from_numpy(z0).cuda(), 5)
    with pytest.raises(CGError) as ei:
        plan.status()
    assert ei.value.status == 5                      # CG_ENAN
    q = _problem(FHN, 64, 64, 0, 2, 0)
    q.flags = FLAG_TEST_STUCK_BARRIER
    q.barrier_timeout_s = 0.2
    stuck = Plan(q, tuning=dict(schedule=2, rows=2))
    good = torch.from_numpy(_state(FHN, 64, 64)).cuda()
    stuck.run(good, 6)
    with pytest.raises(CGError) as ei:
        stuck.status()
    assert ei.value.status == 6                      # CG_ETIMEOUT
    # the context is still usable
    assert np.array_equal(_run(p, _state(FHN, 64, 64), 6, tuning=dict(schedule=2, rows=2)),
                          _run(p, _state(FHN, 64, 64), 6))


@pytest.mark.parametrize("model", [0, 1, 3])
@pytest.mark.parametrize("scheme", [0, 2])
@pytest.mark.parametrize("shape", [(128, 128), (67, 45), (3, 7), (2, 2), (512, 2), (300, 17)])
def test_tblock_neighbor_sync_bitwise(cuda_ok, model, scheme, shape):
    """Neighbour waits between passes (each block waits for the tiles its
    window covers, not for the whole grid): results equal the stage
    kernel's bit for bit for several steps per pass and block sizes (a
    multiple of four warps deals cells to sub-partitions, three warps do
    not), out of place and in place."""
    from paper_1309_1720_gb300 import CGError, FLAG_NEIGHBOR_SYNC
    nx, ny = shape
    p = _problem(model, nx, ny, 1, scheme, 0)
    z0 = _state(model, nx, ny)
    n = 9
    ref = _run(p, z0, n)
    q = _problem(model, nx, ny, 1, scheme, 0)
    q.flags = FLAG_NEIGHBOR_SYNC
    ran = 0
    for k, thr in ((1, 256), (2, 512), (4, 128), (3, 384), (2, 96)):
        try:
            g = _run(q, z0, n, tuning=dict(schedule=2, rows=k, threads=thr))
        except CGError as e:
            # a tile and its halo that do not fit shared memory (four-field
            # RK4 with deep passes) are refused at plan creation
            assert e.status == 7, e
            continue
        assert np.array_equal(g, ref), (k, thr)
        ran += 1
    assert ran >= 3
    assert np.array_equal(_run(q, z0, n, tuning=dict(schedule=2, rows=1), inplace=True), ref)


def test_tblock_neighbor_sync_c1_and_timeout(cuda_ok):
    """The 128^2 Euler workload with neighbour waits, 1000 steps, against the
    stage kernel and the oracle; and the testing knob: the first wait
    expects a pass that never comes, gives up after 0.2 s with
    CG_ETIMEOUT, and the context stays usable."""
    import torch
    from paper_1309_1720_gb300 import CGError, Plan, FHN, FLAG_NEIGHBOR_SYNC, FLAG_TEST_STUCK_BARRIER
    p = _problem(FHN, 128, 128, 0, 0, 0)
    p.dt = 2e-4
    z0 = I.fhn_broken_wave(128, 128, seed=0)
    ref = _run(p, z0, 1000)
    q = _problem(FHN, 128, 128, 0, 0, 0)
    q.dt = 2e-4
    q.flags = FLAG_NEIGHBOR_SYNC
    for k, thr in ((4, 512), (8, 512), (2, 256)):
        assert np.array_equal(_run(q, z0, 1000, tuning=dict(schedule=2, rows=k, threads=thr)), ref), k
    assert field_rel_err(ref, oracle_run(p, z0, 1000)) <= TOL
    s = _problem(FHN, 64, 64, 0, 2, 0)
    s.flags = FLAG_NEIGHBOR_SYNC | FLAG_TEST_STUCK_BARRIER
    s.barrier_timeout_s = 0.2
    stuck = Plan(s, tuning=dict(schedule=2, rows=2))
    stuck.run(torch.from_numpy(_state(FHN, 64, 64)).cuda(), 6)
    with pytest.raises(CGError) as ei:
        stuck.status()
    assert ei.value.status == 6                      # CG_ETIMEOUT
    good = _problem(FHN, 64, 64, 0, 2, 0)
    good.flags = FLAG_NEIGHBOR_SYNC
    assert np.array_equal(_run(good, _state(FHN, 64, 64), 6, tuning=dict(schedule=2, rows=2)),
                          _run(good, _state(FHN, 64, 64), 6))


@pytest.mark.parametrize("model", [0, 1, 2])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_tblock_batch_bitwise(cuda_ok, model, k):
    """Uneven instances in one temporally blocked launch (blocks loop over the
    tiles of all instances): packed out of place and in place, and with
    separate per-instance buffers (cg_batch_run, some in place), bit for bit
    the stage kernel's batch results."""
    import torch
    from paper_1309_1720_gb300 import Plan, KARMA, inputs as I2
    shapes = [(64, 64), (33, 90), (128, 20), (5, 5), (2, 3), (150, 97)]

    def prob(nx, ny):
        if model == KARMA:
            from paper_1309_1720_gb300 import Problem
            return Problem(model=KARMA, nx=nx, ny=ny, dx=I2.KARMA_DX, stencil=1, scheme=2, dt=0.05)
        return _problem(model, nx, ny, 1, 2, 0)

    def state(nx, ny, i):
        if model == KARMA:
            return I2.karma_broken_wave(nx, ny, width=max(1, nx // 6), seed=i)
        return _state(model, nx, ny)

    probs = [prob(nx, ny) for nx, ny in shapes]
    states = [state(nx, ny, i) for i, (nx, ny) in enumerate(shapes)]
    n = 7
    ref = Plan(probs)
    want = [g.cpu().numpy() for g in ref.unpack(ref.run(ref.pack(states), n))]
    ref.status()
    tb = Plan(probs, tuning=dict(schedule=2, rows=k))
    got = [g.cpu().numpy() for g in tb.unpack(tb.run(tb.pack(states), n))]
    tb.status()
    for g, w in zip(got, want):
        assert np.array_equal(g, w)
    z = tb.pack(states)
    tb.run(z, n, out=z)
    tb.status()
    for g, w in zip(tb.unpack(z), want):
        assert np.array_equal(g.cpu().numpy(), w)
    ins = [torch.from_numpy(s_).cuda() for s_ in states]
    outs = [x if i % 2 == 0 else torch.empty_like(x) for i, x in enumerate(ins)]
    res = tb.run_batch(ins, n, outs=outs)
    tb.status()
    for g, w in zip(res, want):
        assert np.array_equal(g.cpu().numpy(), w)
    assert field_rel_err(want[3], oracle_run(probs[3], states[3], n)) <= TOL


def test_tblock_batch_many_small_instances(cuda_ok):
    """256 instances of 32 x 32 (more tiles than resident blocks), Euler,
    1000 steps with 4 steps per pass: bit for bit the stage kernel's batch."""
    from paper_1309_1720_gb300 import Plan, FHN
    probs = [_problem(FHN, 32, 32, 0, 0, 0) for _ in range(256)]
    for p in probs:
        p.dt = 2e-4
    states = [_state(FHN, 32, 32) * (1.0 + 1e-3 * i) for i in range(256)]
    ref = Plan(probs)
    want = ref.run(ref.pack(states), 1000).cpu().numpy()
    ref.status()
    tb = Plan(probs, tuning=dict(schedule=2, rows=4))
    got = tb.run(tb.pack(states), 1000).cpu().numpy()
    tb.status()
    assert np.array_equal(got, want)
