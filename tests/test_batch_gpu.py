"""Batched persistent stepping: many uneven instances in one launch must give
bitwise the same result as stepping each instance alone (same kernel
arithmetic per cell), and the run must replay from a CUDA graph."""
import numpy as np
import pytest

from helpers import field_rel_err, oracle_run
from paper_1309_1720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _problems(sizes, dus, scheme=2, stencil=0):
    from paper_1309_1720_gb300 import Problem, FHN
    return [Problem(model=FHN, nx=int(n), ny=int(n), dx=0.04, D=(float(d), 1.5), stencil=stencil,
                    scheme=scheme, dt=2.5e-4) for n, d in zip(sizes, dus)]


@pytest.mark.parametrize("scheme", [0, 2])
@pytest.mark.parametrize("stencil", [0, 1])
def test_batch_equals_sequential_bitwise(cuda_ok, scheme, stencil):
    import torch
    from paper_1309_1720_gb300 import Plan
    sizes, states, dus = I.batch_workload(n_inst=12, lo=17, hi=90, seed=1)
    probs = _problems(sizes, dus, scheme=scheme, stencil=stencil)
    bp = Plan(probs)
    zb = bp.pack(states)
    out = bp.run(zb, 30)
    bp.status()
    got = [g.cpu().numpy() for g in bp.unpack(out)]
    for i, (p, z) in enumerate(zip(probs, states)):
        sp = Plan(p)
        o = sp.run(torch.from_numpy(z).cuda(), 30)
        sp.status()
        assert np.array_equal(o.cpu().numpy(), got[i]), i
        sp.close()
    # and two instances against the oracle
    for i in (0, 7):
        assert field_rel_err(got[i], oracle_run(probs[i], states[i], 30)) <= 1e-12


def test_batch_full_size_sample(cuda_ok):
    """The 256-instance workload (sizes 64..512 from seed 1, D sweep +/-20%,
    RK4, 5-point): 20 steps batched; sampled instances equal their own
    single-instance runs bitwise."""
    import torch
    from paper_1309_1720_gb300 import Plan
    sizes, states, dus = I.batch_workload(n_inst=256, seed=1)
    probs = _problems(sizes, dus)
    bp = Plan(probs)
    out = bp.run(bp.pack(states), 20)
    bp.status()
    parts = bp.unpack(out)
    for i in (0, 100, 128, 255):
        sp = Plan(probs[i])
        o = sp.run(torch.from_numpy(states[i]).cuda(), 20)
        assert torch.equal(o, parts[i]), i
        sp.close()


def test_graph_capture_replay(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan
    sizes, states, dus = I.batch_workload(n_inst=9, lo=40, hi=130, seed=4)
    bp = Plan(_problems(sizes, dus))
    zin = bp.pack(states)
    eager = bp.run(zin, 25).clone()
    out = torch.empty_like(zin)
    ws = bp.workspace()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        bp.run(zin, 25, out=out, stream=s)      # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        bp.run(zin, 25, out=out, stream=torch.cuda.current_stream())
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)


@pytest.mark.parametrize("scheme", [0, 2])
def test_batch_run_separate_buffers(cuda_ok, scheme):
    """cg_batch_run with one buffer per instance (some in place, some not)
    equals the packed run bit for bit, for odd and even step counts."""
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN
    sizes = [(70, 33), (3, 5), (129, 64), (40, 40), (64, 2)]
    probs = [Problem(model=FHN, nx=nx, ny=ny, dx=0.04, scheme=scheme, dt=1e-4, D=(1.0 + 0.1 * i, 1.5))
             for i, (nx, ny) in enumerate(sizes)]
    zs = [I.fhn_broken_wave(nx, ny, width=4, seed=i) for i, (nx, ny) in enumerate(sizes)]
    plan = Plan(probs)
    for n in (0, 1, 6, 7):
        ref = [g.cpu().numpy() for g in plan.unpack(plan.run(plan.pack(zs), n))]
        ins = [torch.from_numpy(z.copy()).cuda() for z in zs]
        outs = [ins[i] if i % 2 == 0 else torch.empty_like(ins[i]) for i in range(len(ins))]
        got = plan.run_batch(ins, n, outs=outs)
        plan.status()
        for g, r in zip(got, ref):
            assert np.array_equal(g.cpu().numpy(), r), n


@pytest.mark.parametrize("tuning", [None, dict(cells_x=2, threads=256, blocks_per_sm=2, schedule=1, rows=8)])
def test_batch_full_size_against_oracle(cuda_ok, tuning):
    """The full 256-instance workload in one launch (default shape and the
    tile-queue shape the autotuner picks for the bench), 20 RK4 steps: the
    smallest, the largest and two other instances against the oracle."""
    import torch
    from helpers import field_rel_err, oracle_run
    from paper_1309_1720_gb300 import Plan
    sizes, states, dus = I.batch_workload(n_inst=256, seed=1)
    probs = _problems(sizes, dus)
    bp = Plan(probs, tuning=tuning)
    parts = bp.unpack(bp.run(bp.pack(states), 20))
    bp.status()
    order = sorted(range(len(sizes)), key=lambda i: int(sizes[i]))
    for i in (order[0], order[-1], 37, 200):
        assert field_rel_err(parts[i].cpu().numpy(), oracle_run(probs[i], states[i], 20)) <= 1e-12, i
