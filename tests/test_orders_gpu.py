"""Observed convergence orders of the CUDA integrators (Table 2): relative
L2 error of u against a fine-step RK4 run of the same kernels, fitted over
halving dt.  Explicit Euler, Rush-Larsen and implicit Euler 1, Heun 2,
RK4 4 (two-field model); Karma 1, 2, 4 inside one smooth piece of H_k and
RK4 below 3.5 across its band edges (the table's order 3)."""
import math

import numpy as np
import pytest

from paper_1309_1720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _errors(prob_kw, z0, T, dts, scheme):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, RK4
    z = torch.from_numpy(z0).cuda()
    dref = dts[-1] / 8
    ref = Plan(Problem(scheme=RK4, dt=dref, **prob_kw)).run(z, int(round(T / dref)))[0]
    errs = []
    for dt in dts:
        u = Plan(Problem(scheme=scheme, dt=dt, **prob_kw)).run(z, int(round(T / dt)))[0]
        errs.append(float(torch.linalg.norm(u - ref) / torch.linalg.norm(ref)))
    return errs


@pytest.mark.parametrize("scheme,order", [(0, 1), (1, 2), (2, 4)])
def test_fhn_orders(cuda_ok, scheme, order):
    from paper_1309_1720_gb300 import FHN
    from scipy.ndimage import gaussian_filter
    n = 48
    z0 = I.fhn_broken_wave(n, n, width=8, noise=0.0)
    z0 = np.ascontiguousarray(np.stack([gaussian_filter(z0[k], 2.0, mode="nearest") for k in range(2)]))
    kw = dict(model=FHN, nx=n, ny=n, dx=0.5)
    errs = _errors(kw, z0, 0.4, [0.4 / 16, 0.4 / 32, 0.4 / 64], scheme)
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(s - order) < 0.2 for s in slopes), (errs, slopes)


@pytest.mark.parametrize("scheme", [0, 3, 4])
def test_bocf_first_order_schemes(cuda_ok, scheme):
    from paper_1309_1720_gb300 import BOCF
    n = 40
    z0 = I.bocf_spiral_cores(n, n, n_cores=1, seed=2)
    kw = dict(model=BOCF, nx=n, ny=n, dx=0.03, D=(1.171e-3,))
    errs = _errors(kw, z0, 1.0, [1 / 128, 1 / 256, 1 / 512], scheme)
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(s - 1.0) < 0.1 for s in slopes), (errs, slopes)


def _karma_uniform_errors(z0, T, dts, scheme):
    """Errors of u on a gradient-free 8 x 8 Karma state (the model's ODE in
    every cell) against RK4 at dt/16 of the finest step."""
    from paper_1309_1720_gb300 import KARMA
    z = np.empty((2, 8, 8))
    z[0], z[1] = z0
    kw = dict(model=KARMA, nx=8, ny=8, dx=I.KARMA_DX)
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, RK4
    zt = torch.from_numpy(z).cuda()
    dref = dts[-1] / 16
    ref = Plan(Problem(scheme=RK4, dt=dref, **kw)).run(zt, int(round(T / dref)))
    errs = []
    for dt in dts:
        out = Plan(Problem(scheme=scheme, dt=dt, **kw)).run(zt, int(round(T / dt)))
        errs.append(float(torch.linalg.norm(out - ref)))
    return errs


@pytest.mark.parametrize("scheme,order", [(0, 1), (1, 2), (2, 4)])
def test_karma_orders_inside_one_smooth_piece(cuda_ok, scheme, order):
    """An upstroke that stays away from the band edges of H_k: orders 1, 2, 4."""
    errs = _karma_uniform_errors((1.02, 0.3), 10.0, [0.1, 0.05, 0.025], scheme)
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(s - order) < 0.2 for s in slopes), (errs, slopes)


def test_karma_rk4_order_drops_across_the_step_band(cuda_ok):
    """Table 2's order 3 for RK4 on the Karma model: across the band edges of
    the C^1 smoothed step (recovery through u = u_v) the fitted order falls
    below 3.5, on the GPU as in the oracle."""
    dts = [0.1, 0.05, 0.025, 0.0125, 0.00625]
    errs = _karma_uniform_errors((3.5, 1.02), 60.0, dts, 2)
    fit = float(np.polyfit(np.log(dts), np.log(errs), 1)[0])
    assert 2.0 < fit < 3.5, (errs, fit)
