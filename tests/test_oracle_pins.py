"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
eigen-solutions, conservation laws, exact polynomial consistency, roots found
by numpy, hand-worked values of the paper's formulas, measured convergence
orders (Table 2 of the paper), symmetry, and finite differences.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1309_1720_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- P1 decay
def _amp(scheme, z):
    """Amplification polynomial of the explicit scheme for dz/dt = lambda z."""
    if scheme == O.EULER:
        return 1 + z
    if scheme == O.HEUN:
        return 1 + z + z * z / 2
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


@pytest.mark.parametrize("bc", [O.MIRROR, O.CLAMP])
@pytest.mark.parametrize("stencil,alpha_d", [(O.ST5, 0.0), (O.ST9, 1 / 6), (O.ST9, 0.25)])
@pytest.mark.parametrize("scheme", [O.EULER, O.HEUN, O.RK4])
@pytest.mark.parametrize("aniso", [1.0, 0.25])
def test_fourier_mode_decay(bc, stencil, alpha_d, scheme, aniso):
    """P1: with N = 0 a cosine mode is an exact eigenvector of the no-flux
    Laplacian (Eq. diffusion with the ghost points of Fig. 1); n steps scale
    it by G(dt*lambda)^n with G the scheme's stability polynomial."""
    nx, ny, h = 23, 17, 0.1
    Dxx, Dyy = 1.0, aniso
    px, py = 3, 2
    if bc == O.MIRROR:
        tx, ty = math.pi * px / (nx - 1), math.pi * py / (ny - 1)
        cx = np.cos(tx * np.arange(nx)); cy = np.cos(ty * np.arange(ny))
    else:
        tx, ty = math.pi * px / nx, math.pi * py / ny
        cx = np.cos(tx * (np.arange(nx) + 0.5)); cy = np.cos(ty * (np.arange(ny) + 0.5))
    u0 = np.outer(cy, cx)[None].copy()
    a, b = Dxx / h ** 2, Dyy / h ** 2
    kappa = alpha_d * (a + b) / 2 if stencil == O.ST9 else 0.0
    # symbol of Dxx d_xx + Dyy d_yy + kappa h^2 d_xx d_yy
    ex, ey = 2 * math.cos(tx) - 2, 2 * math.cos(ty) - 2
    lam = a * ex + b * ey + kappa * ex * ey
    dt = 0.2 * h * h / (Dxx + Dyy)
    n = 40
    p = O.problem(O.DIFFUSION, nx=nx, ny=ny, dx=h, Dxx=[Dxx], Dyy=[Dyy], stencil=stencil,
                  alpha_d=alpha_d, bc=bc, scheme=scheme, dt=dt)
    un = O.step(p, u0, n)
    expect = _amp(scheme, dt * lam) ** n * u0
    assert np.max(np.abs(un - expect)) <= 1e-13 * np.max(np.abs(u0))


def test_isotropic_weights_match_paper_form():
    """Eq. (diffusion): alpha_pm_pm = alpha_d, alpha_a on axes, balanced
    centre; with alpha_a + 2 alpha_d = 1 the operator is exact on quadratics."""
    nx = ny = 9
    h = 0.5
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    X, Y = np.meshgrid(x, y)
    for st, ad in [(O.ST5, 0.0), (O.ST9, 1 / 6), (O.ST9, 0.3)]:
        p = O.problem(O.DIFFUSION, nx=nx, ny=ny, dx=h, stencil=st, alpha_d=ad)
        u = 3 * X ** 2 + 2 * Y ** 2 + X * Y + X - 7 * Y
        L = O.apply_L(p, u, 1.0)
        # interior value of the continuous Laplacian: 6 + 4 = 10
        assert np.allclose(L[1:-1, 1:-1], 10.0, rtol=0, atol=1e-11)
        # the paper's explicit weights summed by hand at one interior node
        aa, a00 = 1 - 2 * ad, -4 * (1 - ad)
        i, j = 4, 4
        s = (ad * (u[i - 1, j - 1] + u[i - 1, j + 1] + u[i + 1, j - 1] + u[i + 1, j + 1])
             + aa * (u[i - 1, j] + u[i + 1, j] + u[i, j - 1] + u[i, j + 1]) + a00 * u[i, j])
        assert abs(L[i, j] - s / (h * h)) < 1e-11


# ---------------------------------------------------------- P2 conservation
@pytest.mark.parametrize("stencil", [O.ST5, O.ST9])
@pytest.mark.parametrize("scheme", [O.EULER, O.RK4])
def test_conservation(stencil, scheme):
    """P2: pure no-flux diffusion conserves the trapezoid-weighted sum of u
    under MIRROR ghosts and the plain sum under CLAMP ghosts."""
    nx, ny = 19, 14
    u0 = (1.0 + 0.3 * I.uniform_pm1(5, nx * ny)).reshape(1, ny, nx)
    wx = np.ones(nx); wx[[0, -1]] = 0.5
    wy = np.ones(ny); wy[[0, -1]] = 0.5
    W = np.outer(wy, wx)
    for bc, Wt in [(O.MIRROR, W), (O.CLAMP, np.ones((ny, nx)))]:
        p = O.problem(O.DIFFUSION, nx=nx, ny=ny, dx=0.1, Dxx=[1.0], Dyy=[0.6], stencil=stencil,
                      bc=bc, scheme=scheme, dt=0.0015)
        u = O.step(p, u0, 200)
        s0 = math.fsum((Wt * u0[0]).ravel())
        s1 = math.fsum((Wt * u[0]).ravel())
        assert abs(s1 - s0) <= 1e-13 * abs(s0)
        assert np.max(np.abs(u - u0)) > 1e-3   # it did diffuse


def test_transpose_and_weighted_symmetry():
    """The scattered transpose equals the dense transpose, and W L is
    symmetric under MIRROR with trapezoid weights (L^T = W L W^-1)."""
    nx, ny = 6, 5
    for st in (O.ST5, O.ST9):
        for bc in (O.MIRROR, O.CLAMP):
            p = O.problem(O.DIFFUSION, nx=nx, ny=ny, dx=0.3, stencil=st, bc=bc)
            n = nx * ny
            M = np.zeros((n, n))
            for k in range(n):
                e = np.zeros(n); e[k] = 1
                M[:, k] = O.apply_L(p, e.reshape(ny, nx), 1.3, 0.7).ravel()
            MT = np.zeros((n, n))
            for k in range(n):
                e = np.zeros(n); e[k] = 1
                MT[:, k] = O.apply_LT(p, e.reshape(ny, nx), 1.3, 0.7).ravel()
            assert np.allclose(MT, M.T, rtol=0, atol=1e-12)
            if bc == O.MIRROR:
                wx = np.ones(nx); wx[[0, -1]] = 0.5
                wy = np.ones(ny); wy[[0, -1]] = 0.5
                Wd = np.diag(np.outer(wy, wx).ravel())
                WM = Wd @ M
                assert np.allclose(WM, WM.T, rtol=0, atol=1e-12)
            else:
                assert np.allclose(M, M.T, rtol=0, atol=1e-12)


# ----------------------------------------------------------- P3, P6, golden
def test_fhn_golden_points():
    """Eq. (fhn) evaluated by hand at five points (tests/golden)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "fhn_pointwise.txt"))
    p = O.problem(O.FHN)
    for u, v, nu, nv in rows:
        f = O.pointwise(p, [u, v])
        assert abs(f[0] - nu) <= 1e-15 * max(1, abs(nu))
        assert abs(f[1] - nv) <= 1e-16 * max(1, abs(nv)) + 1e-17


def test_fhn_rest_state():
    """P6: the rest point (root of 1.5u^3 - 0.5u + 0.1 found by numpy) is a
    fixed point of the oracle's N[z]; the stored IC constants equal it."""
    r = np.roots([1.5, 0.0, -0.5, 0.1])
    u = float(np.real(r[np.argmin(np.real(r))]))
    v = (u + 0.1) / 1.5
    p = O.problem(O.FHN)
    f = O.pointwise(p, [u, v])
    assert np.max(np.abs(f)) <= 1e-15
    assert abs(u - I.FHN_U_REST) < 1e-14 and abs(v - I.FHN_V_REST) < 1e-14


@pytest.mark.parametrize("model,z0,dt,T", [
    (O.FHN, [0.3, -0.2], 0.02, 4.0),
    (O.BOCF, [0.5, 1.0, 1.0, 0.0], 0.05, 20.0),
])
def test_uniform_field_is_ode(model, z0, dt, T):
    """P3: a uniform field stays exactly uniform (L 1 = 0) and follows the
    model ODE: RK4 matches scipy's DOP853 at tight tolerance to scheme error."""
    from scipy.integrate import solve_ivp
    nv = O.n_fields(model)
    nx, ny = 7, 6
    z = np.empty((nv, ny, nx))
    for c in range(nv):
        z[c] = z0[c]
    p = O.problem(model, nx=nx, ny=ny, dx=0.04 if model == O.FHN else 0.03, scheme=O.RK4, dt=dt)
    n = int(round(T / dt))
    zT = O.step(p, z, n)
    for c in range(nv):
        assert np.all(zT[c] == zT[c, 0, 0])
    pt = O.problem(model)
    sol = solve_ivp(lambda t, y: O.pointwise(pt, y), (0, T), np.asarray(z0, float),
                    method="DOP853", rtol=1e-12, atol=1e-13)
    ref = sol.y[:, -1]
    got = zT[:, 0, 0]
    assert np.max(np.abs(got - ref)) < 1e-6 * max(1.0, np.max(np.abs(ref)))


# --------------------------------------------------------------- P7 H_k
def test_smoothed_step():
    """P7: the cubic step of Sect. 2 is 0, 1/2, 1 at kx = -1/2, 0, 1/2, is
    odd about 1/2, C^1 at the band edges, width 1/k."""
    k = 28.4
    assert O.Hk(-0.5 / k, k) == 0.0
    assert O.Hk(0.0, k) == 0.5
    assert abs(O.Hk(0.5 / k, k) - 1.0) < 1e-15
    assert O.Hk(-1.0, k) == 0.0 and O.Hk(1.0, k) == 1.0
    for x in np.linspace(-0.03, 0.03, 61):
        assert abs(O.Hk(x, k) + O.Hk(-x, k) - 1.0) < 1e-15
    e = 1e-9
    for edge in (-0.5 / k, 0.5 / k):
        assert abs(O.dHk(edge, k)) < 1e-12
        assert abs((O.Hk(edge + e, k) - O.Hk(edge - e, k)) / (2 * e)) < 1e-5
    assert abs(O.dHk(0.0, k) - 1.5 * k) < 1e-12   # slope 3k/2 at the centre


# ------------------------------------------------- BOCF saturated reductions
def test_bocf_saturated_limits():
    """Where every H_k is saturated the model reduces to the piecewise forms of
    the cited minimal model: checked at u = -0.1 (all switches off), u = 0.2
    (v switch off; w, v-, o switches on) and u = 1.0 (all on)."""
    P = O.default_params(O.BOCF)
    (uo, uu, thv, thw, thvm, tho, tv1m, tv2m, tvp, tw1m, tw2m, kwm, uwm, twp,
     tfi, to1, to2, tso1, tso2, kso, uso, ts1, ts2, ks, us, tsi, twinf, wstar, k) = P
    p = O.problem(O.BOCF)
    v, w, s = 0.6, 0.7, 0.3
    th = lambda a: math.tanh(a)
    tau_wm = lambda u: tw1m + (tw2m - tw1m) * (1 + th(kwm * (u - uwm))) / 2
    tau_so = lambda u: tso1 + (tso2 - tso1) * (1 + th(kso * (u - uso))) / 2
    sinf = lambda u: (1 + th(ks * (u - us))) / 2
    # all switches off
    u = -0.1
    f = O.pointwise(p, [u, v, w, s])
    exp = [-(u - uo) / to1, (1 - v) / tv1m, ((1 - u / twinf) - w) / tau_wm(u), (sinf(u) - s) / ts1]
    assert np.allclose(f, exp, rtol=1e-14, atol=1e-16)
    # u = 0.2
    u = 0.2
    f = O.pointwise(p, [u, v, w, s])
    exp = [-(1 / tau_so(u) - w * s / tsi), (0 - v) / tv2m,      # v_inf = 0 once the v- switch is on
           -w / twp, (sinf(u) - s) / ts2]
    assert np.allclose(f, exp, rtol=1e-14, atol=1e-16)
    # u = 1.0
    u = 1.0
    f = O.pointwise(p, [u, v, w, s])
    jfi = -v * (u - thv) * (uu - u) / tfi
    exp = [-(jfi + 1 / tau_so(u) - w * s / tsi), -v / tvp, -w / twp, (sinf(u) - s) / ts2]
    assert np.allclose(f, exp, rtol=1e-14, atol=1e-16)


def test_bocf_action_potential_shape():
    """Sanity of the recalled constants: a 0-D RK4 run from (0.5, 1, 1, 0)
    fires an action potential that peaks in (1.3, 1.55) (the voltage range
    (0, 1.55) of Sect. 2) and repolarises within 500 ms."""
    p = O.problem(O.BOCF, nx=2, ny=2, dx=0.03, scheme=O.RK4, dt=0.05)
    z = np.empty((4, 2, 2))
    for c, val in enumerate([0.5, 1.0, 1.0, 0.0]):
        z[c] = val
    peak, t_above = 0.0, 0.0
    for _ in range(200):                  # first 10 ms step by step: the upstroke
        z = O.step(p, z, 1)
        peak = max(peak, z[0, 0, 0])
        t_above += 0.05 if z[0, 0, 0] > 0.3 else 0.0
    for _ in range(490):                  # then 490 ms in 1 ms strides
        z = O.step(p, z, 20)
        peak = max(peak, z[0, 0, 0])
        t_above += 1.0 if z[0, 0, 0] > 0.3 else 0.0
    assert 1.3 < peak < 1.55
    assert 100.0 < t_above < 400.0
    assert z[0, 0, 0] < 0.1


# ------------------------------------------------------------ P4 orders
@pytest.mark.parametrize("scheme,order", [(O.EULER, 1), (O.HEUN, 2), (O.RK4, 4)])
def test_convergence_order_fhn(scheme, order):
    """P4 / Table 2: observed orders 1, 2 and 4 for FitzHugh-Nagumo with the
    relative L2 error of u (Fig. 5 metric)."""
    n = 24
    z0 = I.fhn_broken_wave(n, n, width=4, noise=0.0)
    # smooth the IC a little so the solution is smooth in time
    from scipy.ndimage import gaussian_filter
    z0 = np.stack([gaussian_filter(z0[0], 2.0, mode="nearest"),
                   gaussian_filter(z0[1], 2.0, mode="nearest")])
    T = 0.4
    ref_p = O.problem(O.FHN, nx=n, ny=n, dx=0.5, scheme=O.RK4, dt=T / 2048)
    ref = O.step(ref_p, z0, 2048)[0]
    errs = []
    for k in (16, 32, 64):
        p = O.problem(O.FHN, nx=n, ny=n, dx=0.5, scheme=scheme, dt=T / k)
        u = O.step(p, z0, k)[0]
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(s - order) < 0.2 for s in slopes), (errs, slopes)


# --------------------------------------------------------- P5 symmetry
def test_reflection_symmetry_bitwise():
    """P5: a reflection-symmetric state stays bitwise symmetric under the x and
    y flips (and the transpose for isotropic D), because the oracle sums
    mirror-image neighbours in pairs."""
    n = 16
    r = I.uniform01(3, n * n).reshape(n, n)
    base = r + r[:, ::-1]
    base = base + base[::-1, :]
    base = base + base.T
    z = np.stack([0.4 * base - 0.5, 0.1 * base])
    for st in (O.ST5, O.ST9):
        p = O.problem(O.FHN, nx=n, ny=n, stencil=st, scheme=O.RK4, dt=2e-4)
        zt = O.step(p, z, 50)
        assert np.array_equal(zt, zt[:, :, ::-1])
        assert np.array_equal(zt, zt[:, ::-1, :])
        assert np.array_equal(zt, np.transpose(zt, (0, 2, 1)))


# ------------------------------------------------------ P8 TLM / adjoint
@pytest.mark.parametrize("model", [O.FHN, O.BOCF])
@pytest.mark.parametrize("stencil", [O.ST5, O.ST9])
@pytest.mark.parametrize("scheme", [O.EULER, O.HEUN, O.RK4])
def test_tlm_fd_and_adjoint_dot(model, stencil, scheme):
    """P8: tangent-linear vs central finite differences (eps = 1e-6) and the
    adjoint dot-product identity <J v, w> = <v, J^T w>."""
    n, steps = 10, 6
    if model == O.FHN:
        z0 = I.fhn_broken_wave(n, n, width=3)
        kw = dict(dx=0.04, dt=2e-4)
    else:
        z0 = I.bocf_spiral_cores(n, n, n_cores=2)
        kw = dict(dx=0.03, dt=0.05, Dxx=[1.171e-3, 0, 0, 0], Dyy=[1.171e-3 / 4, 0, 0, 0])
    p = O.problem(model, nx=n, ny=n, stencil=stencil, scheme=scheme, **kw)
    v = I.unit_direction(z0.shape, 11)
    w = I.unit_direction(z0.shape, 12)
    zT, Jv = O.tlm(p, z0, v, steps)
    eps = 1e-6
    fd = (O.step(p, z0 + eps * v, steps) - O.step(p, z0 - eps * v, steps)) / (2 * eps)
    assert np.linalg.norm(Jv - fd) <= 1e-7 * np.linalg.norm(fd)
    assert np.allclose(zT, O.step(p, z0, steps), rtol=0, atol=1e-14)
    JTw, dLdD = O.adjoint(p, z0, w, steps)
    lhs, rhs = float(np.sum(Jv * w)), float(np.sum(v * JTw))
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(Jv) * np.linalg.norm(w) * 10


def test_adjoint_dD_fd():
    """P8: dL/dD_u from the adjoint vs central FD on D_u for
    L = sum (u_T - u_tgt)^2."""
    n, steps = 12, 20
    z0 = I.fhn_broken_wave(n, n, width=3)
    base = dict(nx=n, ny=n, dx=0.04, scheme=O.RK4, dt=2e-4, stencil=O.ST9)
    tgt = O.step(O.problem(O.FHN, Dxx=[1.05, 1.5], **base), z0, steps)[0]
    p = O.problem(O.FHN, **base)
    zT = O.step(p, z0, steps)
    lam = np.zeros_like(zT)
    lam[0] = 2 * (zT[0] - tgt)
    lam0, dLdD = O.adjoint(p, z0, lam, steps)
    loss = lambda D: float(np.sum((O.step(O.problem(O.FHN, Dxx=[D, 1.5], **base), z0, steps)[0] - tgt) ** 2))
    eps = 1e-6
    fd = (loss(1 + eps) - loss(1 - eps)) / (2 * eps)
    assert abs(dLdD[0] - fd) <= 1e-6 * abs(fd)
    # gradient w.r.t. z0 along a direction
    d = I.unit_direction(z0.shape, 21)
    lz = lambda zz: float(np.sum((O.step(p, zz, steps)[0] - tgt) ** 2))
    fdz = (lz(z0 + eps * d) - lz(z0 - eps * d)) / (2 * eps)
    assert abs(np.sum(lam0 * d) - fdz) <= 1e-6 * abs(fdz)


def test_splitmix64_published_vector():
    """SplitMix64 from seed 0 starts 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4."""
    z = I.splitmix64(0, 2)
    assert int(z[0]) == 0xE220A8397B1DCDAF and int(z[1]) == 0x6E789E6AA1B965F4
