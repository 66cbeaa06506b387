"""Newton-Krylov search for a periodic orbit (Sect. 1's motivating use): a
FitzHugh-Nagumo pulse travelling round a periodic ring returns to itself
after one period.  Checks: Newton converges (quadratically at the end) to a
relative residual |Phi_T(z) - z| / |z| below 1e-11, and the oracle, stepping
the converged state independently, confirms the orbit; also cg_rhs against
the oracle's right-hand side."""

import numpy as np
import pytest

from helpers import field_rel_err, oracle_problem
from paper_1309_1720_gb300 import inputs as I
import oracle as O

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("model,stencil,bc", [(0, 0, 0), (0, 1, 2), (1, 1, 0), (1, 0, 2), (3, 1, 1)])
def test_rhs_matches_oracle(cuda_ok, model, stencil, bc):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem
    nx, ny = 131, 66
    if model == 0:
        p = Problem(model=0, nx=nx, ny=ny, dx=0.04, stencil=stencil, bc=bc, dt=1e-4)
        z = I.fhn_broken_wave(nx, ny, width=9)
    elif model == 1:
        p = Problem(model=1, nx=nx, ny=ny, dx=0.03, D=(1.171e-3,), Dyy=(1.171e-3 / 4,), stencil=stencil, bc=bc,
                    dt=0.05)
        z = I.bocf_spiral_cores(nx, ny, n_cores=3)
    else:
        p = Problem(model=3, nx=nx, ny=ny, dx=0.1, D=(1.0,), Dyy=(0.6,), stencil=stencil, bc=bc, dt=1e-3)
        z = (1.0 + 0.3 * I.uniform_pm1(4, nx * ny)).reshape(1, ny, nx)
    plan = Plan(p)
    f = plan.rhs(torch.from_numpy(z).cuda())
    plan.status()
    assert field_rel_err(f.cpu().numpy(), O.rhs(oracle_problem(p), z)) <= 1e-12


def _pulse(nx, ny):
    z = np.empty((2, ny, nx))
    z[0] = I.FHN_U_REST
    z[1] = I.FHN_V_REST
    z[0, :, 10:20] = 1.0
    z[1, :, 0:10] = 0.6          # refractory behind the bump: it travels one way
    z[1, :, -30:] = 0.6
    return z


def _front(u, level=0.0):
    """Sub-cell position of the pulse's leading edge (first upward-then-down
    crossing of `level` going right from the maximum, wrapped)."""
    n = u.size
    k = int(np.argmax(u))
    for j in range(n):
        a, b = u[(k + j) % n], u[(k + j + 1) % n]
        if a >= level > b:
            return k + j + (a - level) / (a - b)
    raise AssertionError("no front")


def test_travelling_pulse_is_a_periodic_orbit(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, PERIODIC, RK4
    from paper_1309_1720_gb300.newton import periodic_orbit
    nx, ny, h, dt = 512, 2, 0.5, 0.05
    base = Problem(model=FHN, nx=nx, ny=ny, dx=h, bc=PERIODIC, scheme=RK4, dt=dt)
    plan = Plan(base)
    z = plan.run(torch.from_numpy(_pulse(nx, ny)).cuda(), 6000)       # settle the pulse
    x0 = _front(z[0, 0].cpu().numpy())
    z1 = plan.run(z, 2000)
    x1 = _front(z1[0, 0].cpu().numpy())
    plan.status()
    speed = ((x1 - x0) % nx) / (2000 * dt)                             # cells per unit time
    T0 = nx / speed
    n = int(round(T0 / dt))
    zc, T, hist = periodic_orbit(base, z1, T0, n, tol=1e-11)
    res = [hh["rel_residual"] for hh in hist]
    assert res[-1] <= 1e-11, hist
    assert len(res) <= 8, hist
    # quadratic convergence at the end: each of the last residuals below
    # 1e-3 is at most (10 x the previous)^2
    tail = [r for r in res if r < 1e-3]
    for a, b in zip(tail, tail[1:]):
        assert b <= max(100 * a * a, 1e-11), res
    assert abs(T - T0) / T0 < 0.05
    # the oracle, stepping the converged state on its own, closes the orbit
    op = oracle_problem(Problem(model=FHN, nx=nx, ny=ny, dx=h, bc=PERIODIC, scheme=RK4, dt=T / n))
    zc_h = zc.cpu().numpy()
    zo = O.step(op, zc_h, n)
    assert np.linalg.norm(zo - zc_h) / np.linalg.norm(zc_h) <= 1e-9
