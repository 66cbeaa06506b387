"""cg_run_host: stepping a state held in host memory (copy in, run, copy
out, wait) gives cg_run's result bit for bit, for pinned and pageable
buffers, in place, for a batch, and reports device errors on return."""
import numpy as np
import pytest

from helpers import field_rel_err, oracle_run
from paper_1309_1720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("scheme", [0, 2])
def test_run_host_equals_run(cuda_ok, pinned, scheme):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, STENCIL9
    p = Problem(model=FHN, nx=130, ny=67, dx=0.04, stencil=STENCIL9, scheme=scheme, dt=1e-4)
    z0 = I.fhn_broken_wave(130, 67, width=12)
    plan = Plan(p)
    dev = plan.run(torch.from_numpy(z0).cuda(), 37).cpu().numpy()
    h = torch.from_numpy(z0.copy())
    if pinned:
        h = h.pin_memory()
    out = plan.run_host(h, 37)
    assert np.array_equal(out.numpy(), dev)
    assert field_rel_err(out.numpy(), oracle_run(p, z0, 37)) <= 1e-12
    # in place, odd and even step counts
    for n in (1, 4):
        hh = torch.from_numpy(z0.copy())
        plan.run_host(hh, n, out=hh)
        assert np.array_equal(hh.numpy(), plan.run(torch.from_numpy(z0).cuda(), n).cpu().numpy())
    assert np.array_equal(plan.run_host(h, 0).numpy(), z0)


def test_run_host_batch(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, RK4
    sizes = [(64, 64), (3, 9), (101, 77)]
    probs = [Problem(model=FHN, nx=nx, ny=ny, dx=0.04, scheme=RK4, dt=1e-4) for nx, ny in sizes]
    plan = Plan(probs)
    zs = [I.fhn_broken_wave(nx, ny, width=4, seed=i) for i, (nx, ny) in enumerate(sizes)]
    packed = plan.pack(zs).cpu()
    out = plan.run_host(packed, 20)
    dev = plan.run(packed.cuda(), 20).cpu()
    assert torch.equal(out, dev)


def test_run_host_reports_nan(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import CGError, Plan, Problem, FHN
    p = Problem(model=FHN, nx=40, ny=30, dx=0.04, dt=1e-4)
    z0 = I.fhn_broken_wave(40, 30)
    z0[0, 5, 7] = np.nan
    plan = Plan(p)
    with pytest.raises(CGError) as ei:
        plan.run_host(torch.from_numpy(z0), 3)
    assert ei.value.status == 5          # CG_ENAN
    # the context stays usable
    good = I.fhn_broken_wave(40, 30)
    assert np.array_equal(plan.run_host(torch.from_numpy(good), 3).numpy(),
                          plan.run(torch.from_numpy(good).cuda(), 3).cpu().numpy())
