"""cg_run_noalloc: stepping without any device allocation, for callers that
cannot allocate at run time (inside CUDA-graph capture, under a foreign pool
allocator, in allocation-free real-time loops).  Its scratch is a fixed
static device array; the result must equal cg_run's with a caller
workspace, call after call.  This file sorts last so that a run stopping at
the first failure has already run every other test."""

import pytest

from helpers import field_rel_err
from paper_1309_1720_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _noalloc(plan, z_in, z_out, n_steps, status):
    import torch
    from paper_1309_1720_gb300 import _lib
    st = _lib.lib().cg_run_noalloc(plan.handle, z_in.data_ptr(), z_out.data_ptr(), int(n_steps),
                                   status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st


def test_noalloc_matches_cg_run_twice(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, RK4, STENCIL9
    n = 256
    plan = Plan(Problem(model=FHN, nx=n, ny=n - 13, dx=0.04, stencil=STENCIL9, scheme=RK4, dt=2e-4))
    status = torch.full((1,), 0xFFFF, dtype=torch.int32, device="cuda")
    for call, (seed, steps) in enumerate([(0, 37), (5, 20)]):
        z0 = torch.from_numpy(I.fhn_broken_wave(n, n - 13, width=30, seed=seed)).cuda()
        ref = plan.run(z0, steps)
        plan.status()
        out = torch.full_like(z0, float("nan"))
        assert _noalloc(plan, z0, out, steps, status) == 0
        torch.cuda.synchronize()
        assert int(status.item()) == 0, call
        # the same kernel on the same inputs: equal bit for bit (so within
        # the 1e-12 parity tolerance as well)
        assert torch.equal(out, ref), call
        assert field_rel_err(out.cpu().numpy(), ref.cpu().numpy()) <= TOL, call


def test_noalloc_rejects_oversized_plan(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, _lib
    plan = Plan(Problem(model=FHN, nx=1024, ny=1024, dx=0.04, dt=2e-4))
    z = torch.zeros(plan.offsets[-1], dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _noalloc(plan, z, z, 1, status) == 1
    assert "32" in _lib.lib().cg_last_error().decode()
