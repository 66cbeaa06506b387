"""A single grid of more than 2^31 cells (46341^2 with scalar row access,
46342^2 with 16-byte vector access; the diffusion model, in place): every
address computation must be 64-bit.  The initial
state varies along x only; under mirror ghosts in y every row then follows
the same arithmetic, so each of the n rows must equal, bit for bit, the
rows of the same problem on an n x 2 grid, which in turn matches the
oracle.  Needs about 90 GB of device memory (skipped on smaller devices)."""
import numpy as np
import pytest

from helpers import field_rel_err, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,stencil,scheme", [(46341, 1, 2), (46342, 0, 0)])
def test_more_than_2_pow_31_cells(cuda_ok, n, stencil, scheme):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, DIFFUSION
    free, _ = torch.cuda.mem_get_info()
    if free < 100e9:
        pytest.skip("needs about 90 GB of free device memory")
    assert n * n > 2 ** 31
    dt = 2e-4 if scheme == 2 else 1e-4
    kw = dict(model=DIFFUSION, dx=0.05, D=(0.1,), Dyy=(0.07,), stencil=stencil, scheme=scheme, dt=dt)
    x = np.arange(n, dtype=np.float64)
    prof = np.cos(2 * np.pi * x / 977.0) + 0.25 * np.sin(2 * np.pi * x / 131.0) + 1e-3 * (x % 17)
    small = np.ascontiguousarray(np.broadcast_to(prof, (1, 2, n)))
    steps = 3
    ps = Problem(nx=n, ny=2, **kw)
    splan = Plan(ps)
    ref = splan.run(torch.from_numpy(small).cuda(), steps)
    splan.status()
    assert torch.equal(ref[0, 0], ref[0, 1])
    assert field_rel_err(ref.cpu().numpy(), oracle_run(ps, small, steps)) <= 1e-12
    row = ref[0, 0].contiguous()
    del ref
    big = torch.from_numpy(prof).cuda().expand(n, n).contiguous().view(1, n, n)
    plan = Plan(Problem(nx=n, ny=n, **kw))
    plan.run(big, steps, out=big)
    plan.status()
    bad = 0
    for y0 in range(0, n, 2048):
        blk = big[0, y0:y0 + 2048]
        bad += int((blk != row).sum())
    assert bad == 0
    plan._ws = None
    plan.close()
    del big
    torch.cuda.empty_cache()
