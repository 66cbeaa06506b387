"""Pins of the oracle's two-variable Karma model (Eq. karma, Sect. 2).

The paper prints the form of the model and (Re, M, gamma); the remaining
constants come from the cited model paper, so these pins fix the FORM for
chosen constants: closed-form solutions of the discrete scheme where the
model reduces to a linear equation, the exact solution of the Bernoulli
equation it reduces to when the tanh saturates, exact fixed points, the
scale of the paper's voltage range, the tanh variant of Sect. 6, the hand Jacobian
against central differences, and the tangent-linear / adjoint pair."""
import math

import numpy as np
import pytest

import oracle as O

TU, TV, USTAR, UH, UV, RE, M, K = range(8)


def _amp(scheme, z):
    if scheme == O.EULER:
        return 1 + z
    if scheme == O.HEUN:
        return 1 + z + z * z / 2
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def _uniform(u, v, nx=5, ny=4):
    z = np.empty((2, ny, nx))
    z[0] = u
    z[1] = v
    return z


def _params(**kw):
    q = O.default_params(O.KARMA).copy()
    names = dict(tau_u=TU, tau_v=TV, u_star=USTAR, u_h=UH, u_v=UV, Re=RE, M=M, k=K)
    for k, v in kw.items():
        q[names[k]] = v
    return q


def test_defaults_and_fields():
    """Sect. 2: (Re, M) = (1, 6), k = 28.4; two fields, only u diffuses."""
    q = O.default_params(O.KARMA)
    assert len(q) == 8 and q[RE] == 1.0 and q[M] == 6.0 and q[K] == 28.4
    assert O.n_fields(O.KARMA) == 2
    p = O.problem(O.KARMA)
    assert p.Dxx[0] == pytest.approx(1.1e-3) and p.Dxx[1] == 0.0


@pytest.mark.parametrize("scheme", [O.EULER, O.HEUN, O.RK4])
def test_resting_state_v_decay_closed_form(scheme):
    """At u = 0 the u-equation vanishes exactly (every term carries u) and,
    with H_k(-u_v) = 0, H_k(u_v) = 1, the v-equation is dv/dt = -v/tau_v:
    n steps multiply v by the scheme's amplification polynomial at
    -dt/tau_v, for any gradient-free state."""
    dt, n = 0.5, 60
    p = O.problem(O.KARMA, nx=5, ny=4, dx=0.0262, scheme=scheme, dt=dt)
    z = O.step(p, _uniform(0.0, 1.3), n)
    assert np.all(z[0] == 0.0)
    q = O.default_params(O.KARMA)
    expect = 1.3 * _amp(scheme, -dt / q[TV]) ** n
    assert np.max(np.abs(z[1] - expect)) <= 1e-13


@pytest.mark.parametrize("scheme", [O.EULER, O.HEUN, O.RK4])
@pytest.mark.parametrize("Re", [1.0, 0.5])
def test_excited_v_relaxes_to_recovery_level(scheme, Re):
    """With u frozen above u_v + 1/(2k) (tau_u huge) the v-equation is
    dv/dt = (a - v)/tau_v, a = 1/(1 - e^-Re): v_n = a + (v_0 - a) G^n."""
    dt, n = 2.0, 40
    q = _params(tau_u=1e300, Re=Re)
    p = O.problem(O.KARMA, nx=5, ny=4, dx=0.0262, scheme=scheme, dt=dt, params=q)
    z = O.step(p, _uniform(2.0, 0.1), n)
    a = 1.0 / (1.0 - math.exp(-Re))
    assert np.all(z[0] == 2.0)
    expect = a + (0.1 - a) * _amp(scheme, -dt / q[TV]) ** n
    assert np.max(np.abs(z[1] - expect)) <= 1e-13 * a


def test_v_at_threshold_uses_both_steps():
    """At u = u_v both smoothed steps are 1/2: dv/dt = (a/2 - v)/tau_v."""
    dt, n = 2.0, 30
    q = _params(tau_u=1e300)
    p = O.problem(O.KARMA, nx=3, ny=3, dx=0.0262, scheme=O.RK4, dt=dt, params=q)
    z = O.step(p, _uniform(q[UV], 0.2, 3, 3), n)
    a2 = 0.5 / (1.0 - math.exp(-1.0))
    expect = a2 + (0.2 - a2) * _amp(O.RK4, -dt / q[TV]) ** n
    assert np.max(np.abs(z[1] - expect)) <= 1e-14


@pytest.mark.parametrize("v0,Mv", [(0.5, 6.0), (0.8, 3.0), (0.0, 6.0)])
def test_bernoulli_solution_when_tanh_saturates(v0, Mv):
    """u_h = 1e6 makes tanh(u - u_h) = -1 exactly; with v frozen (tau_v
    huge) the u-equation becomes du/dt = (g u^2 - u)/tau_u, g = u* - v^M,
    whose solution is u(t) = 1/(g + (1/u_0 - g) e^{t/tau_u}).  RK4 at
    dt = tau_u/400 reproduces it to 1e-10."""
    q = _params(u_h=1e6, tau_v=1e300, M=Mv)
    tau = q[TU]
    dt, n = tau / 400, 1200
    p = O.problem(O.KARMA, nx=4, ny=3, dx=0.0262, scheme=O.RK4, dt=dt, params=q)
    u0 = 0.4
    z = O.step(p, _uniform(u0, v0, 4, 3), n)
    g = q[USTAR] - v0 ** Mv
    t = n * dt
    exact = 1.0 / (g + (1.0 / u0 - g) * math.exp(t / tau))
    assert np.all(z[1] == v0)
    assert np.max(np.abs(z[0] - exact)) <= 1e-10 * u0


@pytest.mark.parametrize("variant", [O.AS_WRITTEN, O.TANH_AS_HK])
def test_fixed_point_at_u_h(variant):
    """At u = u_h, tanh(0) = 0 (and 2 H(0) - 1 = 0) so f_u = (u_h^2/2 g -
    u_h)/tau_u, which vanishes for u_h = 2, g = u* - v^M = 1: with v frozen,
    u = 2 stays put under every scheme.  Pins the 1/2, the u^2 and v^M."""
    q = _params(u_h=2.0, u_star=1.0 + 0.5 ** 6, tau_v=1e300)
    for scheme in (O.EULER, O.HEUN, O.RK4):
        p = O.problem(O.KARMA, nx=3, ny=3, dx=0.0262, scheme=scheme, dt=0.1, params=q, variant=variant)
        z = O.step(p, _uniform(2.0, 0.5, 3, 3), 50)
        assert np.max(np.abs(z[0] - 2.0)) <= 1e-14
        f = O.pointwise(p, [2.0, 0.5])
        assert abs(f[0]) <= 1e-16


def test_action_potential_scale():
    """Sect. 2 gives the Karma voltage a range of about (0, 3.5): a stimulated
    cell (u = 1.5 on the resting v = 0) rises above 3 (to 3.79 with these
    constants, the upper root of u (1 - tanh(u - u_h)) u*/2 = 1 while v is
    still small), stays non-negative and returns to rest as v recovers."""
    p = O.problem(O.KARMA, nx=3, ny=3, dx=0.0262, scheme=O.RK4, dt=0.05)
    z = _uniform(1.5, 0.0, 3, 3)
    umax, umin = 0.0, 10.0
    for _ in range(1000):
        z = O.step(p, z, 20)
        umax = max(umax, z[0, 0, 0])
        umin = min(umin, z[0, 0, 0])
    assert 3.0 < umax < 4.0
    assert umin >= 0.0 and z[0, 0, 0] < 1e-3


def test_tanh_variant_values():
    """Sect. 6's replacement of tanh(x) by 2 H_{1/3}(x) - 1: same value and
    slope at x = 0, exactly -1 / +1 beyond |x| = 3/2, and 0.6875 at x = 3/4
    (t = 3/4: 2 t^2 (3 - 2t) - 1)."""
    for x, th in [(0.0, 0.0), (-1.6, -1.0), (1.6, 1.0), (0.75, 0.6875)]:
        q = _params(u_h=0.0, u_star=1.0, tau_u=1.0, tau_v=1e300)
        p = O.problem(O.KARMA, nx=1, ny=1, scheme=O.EULER, params=q, variant=O.TANH_AS_HK)
        u = x
        f = O.pointwise(p, [u, 0.0])
        assert f[0] == pytest.approx(u * u / 2 * (1 - th) - u, abs=1e-15)
    # slope of f_u at u = u_h: d/du[u^2/2 (1 - th)] - 1 = u_h (1 - 0) - u_h^2/2 th'(0) - 1
    q = _params(u_h=1.0, u_star=1.0, tau_u=1.0, tau_v=1e300)
    for variant in (O.AS_WRITTEN, O.TANH_AS_HK):
        p = O.problem(O.KARMA, nx=1, ny=1, scheme=O.EULER, params=q, variant=variant)
        J = O.pointwise_jac(p, [1.0, 0.0])
        assert J[0, 0] == pytest.approx(1.0 - 0.5 * 1.0 - 1.0, abs=1e-15)


@pytest.mark.parametrize("variant", [O.AS_WRITTEN, O.TANH_AS_HK])
def test_jacobian_against_central_differences(variant):
    p = O.problem(O.KARMA, nx=1, ny=1, scheme=O.EULER, variant=variant)
    rng = np.random.default_rng(3)
    for _ in range(40):
        zc = np.array([rng.uniform(0.0, 3.6), rng.uniform(0.05, 1.5)])
        J = O.pointwise_jac(p, zc)
        for j in range(2):
            h = 1e-6
            e = np.zeros(2)
            e[j] = h
            fd = (O.pointwise(p, zc + e) - O.pointwise(p, zc - e)) / (2 * h)
            assert np.allclose(J[:, j], fd, rtol=1e-6, atol=1e-7), (zc, j)


@pytest.mark.parametrize("stencil", [O.ST5, O.ST9])
@pytest.mark.parametrize("scheme", [O.EULER, O.HEUN, O.RK4])
def test_tlm_fd_and_adjoint_dot(stencil, scheme):
    """Tangent-linear run against central differences of the oracle's own
    step, and <lam_T, J dz> = <J^T lam_T, dz> for the adjoint."""
    nx, ny, n = 9, 7, 12
    p = O.problem(O.KARMA, nx=nx, ny=ny, dx=0.0262, stencil=stencil, scheme=scheme, dt=0.05)
    rng = np.random.default_rng(5)
    z0 = np.empty((2, ny, nx))
    z0[0] = rng.uniform(0.0, 3.2, (ny, nx))
    z0[1] = rng.uniform(0.1, 1.2, (ny, nx))
    dz = rng.standard_normal(z0.shape)
    _, jdz = O.tlm(p, z0, dz, n)
    eps = 1e-6
    fd = (O.step(p, z0 + eps * dz, n) - O.step(p, z0 - eps * dz, n)) / (2 * eps)
    assert np.linalg.norm(jdz - fd) <= 1e-6 * np.linalg.norm(fd)
    lamT = rng.standard_normal(z0.shape)
    lam0, dLdD = O.adjoint(p, z0, lamT, n)
    assert abs(np.vdot(lamT, jdz) - np.vdot(lam0, dz)) <= 1e-11 * abs(np.vdot(lamT, jdz))
    assert len(dLdD) == 2


def test_adjoint_dD_fd():
    """dL/dgamma from the adjoint against central differences in gamma."""
    nx, ny, n = 8, 6, 10
    rng = np.random.default_rng(7)
    z0 = np.empty((2, ny, nx))
    z0[0] = rng.uniform(0.0, 3.2, (ny, nx))
    z0[1] = rng.uniform(0.1, 1.2, (ny, nx))
    lamT = rng.standard_normal(z0.shape)
    g0 = 1.1e-3

    def L(g):
        p = O.problem(O.KARMA, nx=nx, ny=ny, dx=0.0262, stencil=O.ST9, scheme=O.RK4, dt=0.05, Dxx=[g, 0])
        return np.vdot(lamT, O.step(p, z0, n))

    p = O.problem(O.KARMA, nx=nx, ny=ny, dx=0.0262, stencil=O.ST9, scheme=O.RK4, dt=0.05, Dxx=[g0, 0])
    _, dLdD = O.adjoint(p, z0, lamT, n)
    h = 1e-7
    fd = (L(g0 + h) - L(g0 - h)) / (2 * h)
    assert dLdD[0] == pytest.approx(fd, rel=1e-6)


def test_rk4_order_and_the_smoothed_step():
    """Table 2 reports order 3 instead of 4 for RK4 on the Karma and
    Bueno-Orovio models, which the paper leaves unexplained.  Both models
    switch through the cubic H_k, which is only C^1: its second derivative
    jumps at k x = +-1/2.  On a gradient-free state (the model's ODE): while
    u stays inside one smooth piece the observed order is 4; on a trajectory
    whose u falls through the band edges of H_k(u - u_v) at the end of the
    action potential it drops below 3.5 (a step that straddles an edge makes
    a local error of order dt^3)."""
    def run(z0, T, dt):
        p = O.problem(O.KARMA, nx=3, ny=3, dx=0.0262, scheme=O.RK4, dt=dt)
        return O.step(p, _uniform(z0[0], z0[1], 3, 3), int(round(T / dt)))[:, 0, 0]

    dts = [0.1, 0.05, 0.025, 0.0125, 0.00625]
    smooth = ((1.02, 0.3), 10.0)             # upstroke away from the band edges
    ref = run(*smooth, dts[-1] / 16)
    errs = [np.linalg.norm(run(*smooth, d) - ref) for d in dts[:3]]
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(slopes) > 3.9, slopes
    across = ((3.5, 1.02), 60.0)             # plateau, recovery through u = u_v
    ref = run(*across, dts[-1] / 16)
    errs = [np.linalg.norm(run(*across, d) - ref) for d in dts]
    fit = np.polyfit(np.log(dts), np.log(errs), 1)[0]
    assert 2.0 < fit < 3.5, fit
