"""Pins of the oracle's periodic ghosts, its gate integrators (Rush-Larsen and
implicit Euler on the Bueno-Orovio gates) and its tanh-as-smoothed-step
variant of the Bueno-Orovio model, each against something other than the
oracle itself: exact Fourier eigen-solutions, translation invariance, the
method of images, an adaptive ODE integrator, the implicit equation's
residual, measured convergence orders (Table 2), and closed-form values of the
smoothed step."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1309_1720_gb300 import inputs as I


def _amp(scheme, z):
    if scheme == O.EULER:
        return 1 + z
    if scheme == O.HEUN:
        return 1 + z + z * z / 2
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


# ------------------------------------------------------------ periodic ghosts
@pytest.mark.parametrize("stencil,alpha_d", [(O.ST5, 0.0), (O.ST9, 1 / 6), (O.ST9, 0.25)])
@pytest.mark.parametrize("scheme", [O.EULER, O.HEUN, O.RK4])
@pytest.mark.parametrize("aniso", [1.0, 0.25])
def test_periodic_fourier_mode_decay(stencil, alpha_d, scheme, aniso):
    """Sect. 3 (opposite-edge ghosts): a shifted cosine cos(2 pi p x/n + phi)
    is an exact eigenvector of the periodic Laplacian; n steps scale it by
    G(dt lambda)^n."""
    nx, ny, h = 24, 18, 0.1
    px, py = 5, 2
    tx, ty = 2 * math.pi * px / nx, 2 * math.pi * py / ny
    cx = np.cos(tx * np.arange(nx) + 0.3)
    cy = np.cos(ty * np.arange(ny) - 1.1)
    u0 = np.outer(cy, cx)[None].copy()
    a, b = 1.0 / h ** 2, aniso / h ** 2
    kappa = alpha_d * (a + b) / 2 if stencil == O.ST9 else 0.0
    ex, ey = 2 * math.cos(tx) - 2, 2 * math.cos(ty) - 2
    lam = a * ex + b * ey + kappa * ex * ey
    dt = 0.2 * h * h / (1.0 + aniso)
    p = O.problem(O.DIFFUSION, nx=nx, ny=ny, dx=h, Dxx=[1.0], Dyy=[aniso], stencil=stencil,
                  alpha_d=alpha_d, bc=O.PERIODIC, scheme=scheme, dt=dt)
    un = O.step(p, u0, 40)
    assert np.max(np.abs(un - _amp(scheme, dt * lam) ** 40 * u0)) <= 1e-13


@pytest.mark.parametrize("model", [O.FHN, O.BOCF])
def test_periodic_translation_invariance_bitwise(model):
    """Every cell of a periodic grid sees the same arithmetic, so stepping a
    rolled state gives the rolled result bit for bit."""
    n = 20
    if model == O.FHN:
        z = I.fhn_broken_wave(n, n, width=5, seed=4)
        p = O.problem(O.FHN, nx=n, ny=n, stencil=O.ST9, bc=O.PERIODIC, scheme=O.RK4, dt=2e-4)
    else:
        z = I.bocf_spiral_cores(n, n, n_cores=2, seed=4)
        p = O.problem(O.BOCF, nx=n, ny=n, dx=0.03, Dxx=[1.171e-3], Dyy=[1.171e-3 / 4],
                      stencil=O.ST9, bc=O.PERIODIC, scheme=O.RK4, dt=0.05)
    base = O.step(p, z, 10)
    for sy, sx in [(3, 0), (0, 7), (5, 11)]:
        zr = np.roll(z, (sy, sx), axis=(1, 2))
        assert np.array_equal(O.step(p, zr, 10), np.roll(base, (sy, sx), axis=(1, 2)))


def test_periodic_method_of_images():
    """Mirror ghosts on n points equal periodic ghosts on the even extension
    of period 2(n-1), restricted to the first n points (bit for bit: the same
    neighbour values are summed in the same order)."""
    nx, ny = 13, 9
    z = I.fhn_broken_wave(nx, ny, width=4, seed=6)
    ext = lambda a, n, ax: np.concatenate([a, np.flip(np.take(a, range(1, n - 1), axis=ax), axis=ax)], axis=ax)
    Z = ext(ext(z, nx, 2), ny, 1)
    assert Z.shape == (2, 2 * (ny - 1), 2 * (nx - 1))
    for st in (O.ST5, O.ST9):
        pm = O.problem(O.FHN, nx=nx, ny=ny, stencil=st, bc=O.MIRROR, scheme=O.RK4, dt=2e-4)
        pp = O.problem(O.FHN, nx=2 * (nx - 1), ny=2 * (ny - 1), stencil=st, bc=O.PERIODIC, scheme=O.RK4,
                       dt=2e-4)
        assert np.array_equal(O.step(pm, z, 15), O.step(pp, Z, 15)[:, :ny, :nx])


@pytest.mark.parametrize("shape", [(6, 5), (2, 3), (3, 2), (2, 2)])
def test_periodic_operator_symmetric_and_conservative(shape):
    """The periodic operator is a symmetric circulant: the scattered transpose
    equals it, its dense matrix is symmetric, and its columns sum to 0 (plain
    sum conserved), including the degenerate widths 2 and 3."""
    nx, ny = shape
    for st in (O.ST5, O.ST9):
        p = O.problem(O.DIFFUSION, nx=nx, ny=ny, dx=0.3, stencil=st, bc=O.PERIODIC)
        n = nx * ny
        M = np.zeros((n, n))
        MT = np.zeros((n, n))
        for k in range(n):
            e = np.zeros(n); e[k] = 1
            M[:, k] = O.apply_L(p, e.reshape(ny, nx), 1.3, 0.7).ravel()
            MT[:, k] = O.apply_LT(p, e.reshape(ny, nx), 1.3, 0.7).ravel()
        assert np.allclose(M, M.T, rtol=0, atol=1e-12)
        assert np.allclose(MT, M, rtol=0, atol=1e-12)
        assert np.allclose(M.sum(axis=0), 0.0, atol=1e-11)


# ------------------------------------------------------------ gate integrators
def _gate_coefficients(p, zc):
    """alpha, beta of dx/dt = alpha x + beta for x = v, w, s, recovered from
    the right-hand side at x = 0 and x = 1 (the gate equations are linear in
    their own gate)."""
    al, be = [], []
    for g in (1, 2, 3):
        z0 = np.array(zc, dtype=float); z0[g] = 0.0
        z1 = np.array(zc, dtype=float); z1[g] = 1.0
        f0 = O.pointwise(p, z0)[g]
        f1 = O.pointwise(p, z1)[g]
        al.append(f1 - f0)
        be.append(f0)
    return np.array(al), np.array(be)


CELLS = [(-0.05, 0.9, 0.8, 0.1), (0.01, 0.7, 0.9, 0.2), (0.12, 0.5, 0.6, 0.3), (0.2, 0.3, 0.5, 0.4),
         (0.31, 0.2, 0.4, 0.5), (0.9, 0.05, 0.3, 0.6), (1.4, 0.0, 0.2, 0.9)]


def _uniform(zc, n=2):
    z = np.empty((4, n, n))
    for c in range(4):
        z[c] = zc[c]
    return z


@pytest.mark.parametrize("scheme", [O.RUSH_LARSEN, O.IMPLICIT_EULER])
def test_gate_schemes_take_an_euler_step_in_u(scheme):
    """Both gate integrators advance u exactly as explicit Euler does."""
    n = 12
    z = I.bocf_spiral_cores(n, n, n_cores=2, seed=3)
    kw = dict(nx=n, ny=n, dx=0.03, Dxx=[1.171e-3], Dyy=[1.171e-3 / 4], stencil=O.ST9, dt=0.05)
    fe = O.step(O.problem(O.BOCF, scheme=O.EULER, **kw), z, 1)
    gs = O.step(O.problem(O.BOCF, scheme=scheme, **kw), z, 1)
    assert np.array_equal(fe[0], gs[0])
    assert not np.array_equal(fe[1:], gs[1:])


@pytest.mark.parametrize("dt", [0.05, 2.0, 40.0])
def test_rush_larsen_is_the_exact_frozen_u_gate_flow(dt):
    """Rush-Larsen: the gates after one step equal an adaptive high-order
    integration of dx/dt = alpha x + beta over dt with u frozen (uniform
    field, so no diffusion enters)."""
    from scipy.integrate import solve_ivp
    p = O.problem(O.BOCF, nx=2, ny=2, dx=0.03, scheme=O.RUSH_LARSEN, dt=dt)
    for zc in CELLS:
        al, be = _gate_coefficients(p, zc)
        out = O.step(p, _uniform(zc), 1)[:, 0, 0]
        sol = solve_ivp(lambda t, x: al * x + be, (0.0, dt), np.array(zc[1:]), method="DOP853",
                        rtol=1e-13, atol=1e-15)
        assert np.allclose(out[1:], sol.y[:, -1], rtol=1e-10, atol=1e-13), (zc, out, sol.y[:, -1])


@pytest.mark.parametrize("dt", [0.05, 2.0, 40.0])
def test_implicit_euler_solves_its_equation(dt):
    """Implicit Euler: x' - x = dt (alpha x' + beta) holds to rounding, and x'
    lies between x and the frozen steady state -beta/alpha for any dt."""
    p = O.problem(O.BOCF, nx=2, ny=2, dx=0.03, scheme=O.IMPLICIT_EULER, dt=dt)
    for zc in CELLS:
        al, be = _gate_coefficients(p, zc)
        x0 = np.array(zc[1:])
        x1 = O.step(p, _uniform(zc), 1)[1:, 0, 0]
        res = x1 - x0 - dt * (al * x1 + be)
        assert np.all(np.abs(res) <= 1e-13 * (1 + np.abs(x0) + dt * (np.abs(al) + np.abs(be)))), res
        xinf = -be / al
        assert np.all(x1 >= np.minimum(x0, xinf) - 1e-15) and np.all(x1 <= np.maximum(x0, xinf) + 1e-15)


@pytest.mark.parametrize("scheme", [O.RUSH_LARSEN, O.IMPLICIT_EULER])
def test_gate_schemes_first_order(scheme):
    """Table 2: implicit Euler and Rush-Larsen converge with order 1 (relative
    L2 error of u against a fine RK4 reference, the Fig. 5 metric)."""
    n = 10
    z0 = I.bocf_spiral_cores(n, n, n_cores=1, seed=2)
    kw = dict(nx=n, ny=n, dx=0.03, Dxx=[1.171e-3], Dyy=[1.171e-3])
    T = 1.0
    ref = O.step(O.problem(O.BOCF, scheme=O.RK4, dt=T / 4096, **kw), z0, 4096)[0]
    errs = []
    for k in (128, 256, 512):
        u = O.step(O.problem(O.BOCF, scheme=scheme, dt=T / k, **kw), z0, k)[0]
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(s - 1.0) < 0.1 for s in slopes), (errs, slopes)


def test_gate_schemes_reject_other_models_and_tangents():
    z = I.fhn_broken_wave(8, 8)
    with pytest.raises(ValueError):
        O.step(O.problem(O.FHN, nx=8, ny=8, scheme=O.RUSH_LARSEN), z, 1)
    zb = I.bocf_spiral_cores(8, 8, n_cores=1)
    pb = O.problem(O.BOCF, nx=8, ny=8, dx=0.03, scheme=O.IMPLICIT_EULER, dt=0.05)
    with pytest.raises(ValueError):
        O.tlm(pb, zb, zb, 1)
    with pytest.raises(ValueError):
        O.adjoint(pb, zb, zb, 1)


# ---------------------------------------------------- tanh as smoothed step
def _s_inf(p, u):
    """s_inf(u) from the s equation at s = 0 where the w switch is on
    (tau_s = tau_s2)."""
    ts2 = O.default_params(O.BOCF)[22]
    return O.pointwise(p, [u, 0.0, 0.0, 0.0])[3] * ts2


def _tau_wm(p, u):
    """tau_w^-(u) from the w equation at w = 0 where H_o = 1 and H_w = 0."""
    wstar = O.default_params(O.BOCF)[27]
    return wstar / O.pointwise(p, [u, 0.0, 0.0, 0.0])[2]


def test_tanh_variant_smoothed_step_values():
    """Sect. 6 replaces (1 + tanh(k x))/2 by a smoothed step; with H_{k/3} it
    keeps the value 1/2 and the slope k/2 at x = 0, is exactly 0 and 1 beyond
    |x| = 3/(2k), and stays within 0.07 of the tanh form (0.056 at most)."""
    P = O.default_params(O.BOCF)
    ks, us, kwm, uwm, tw1m, tw2m = P[23], P[24], P[11], P[12], P[9], P[10]
    pv = O.problem(O.BOCF, variant=O.TANH_AS_HK)
    pt = O.problem(O.BOCF)
    assert abs(_s_inf(pv, us) - 0.5) < 1e-14
    e = 1e-6
    assert abs((_s_inf(pv, us + e) - _s_inf(pv, us - e)) / (2 * e) - ks / 2) < 1e-6
    half = 1.5 / ks
    assert _s_inf(pv, us + half + 1e-3) == 1.0 or abs(_s_inf(pv, us + half + 1e-3) - 1.0) < 1e-15
    assert abs(_s_inf(pv, us - half - 1e-3)) < 1e-15
    us_grid = np.linspace(0.2, 1.6, 141)
    dev = max(abs(_s_inf(pv, u) - _s_inf(pt, u)) for u in us_grid)
    assert 0.03 < dev < 0.07
    # tau_w^- switches between tw1m and tw2m about uwm
    assert abs(_tau_wm(pv, uwm) - (tw1m + tw2m) / 2) < 1e-12
    assert abs(_tau_wm(pv, uwm + 1.5 / kwm + 1e-3) - tw2m) < 1e-12
    assert abs(_tau_wm(pt, uwm + 1.5 / kwm + 1e-3) - tw2m) > 1e-3


def test_tanh_variant_jacobian_and_adjoint():
    """The variant's hand Jacobian against central differences of its right
    side, and its tangent/adjoint pair through the dot-product identity."""
    p = O.problem(O.BOCF, variant=O.TANH_AS_HK)
    for zc in CELLS:
        J = O.pointwise_jac(p, zc)
        for j in range(4):
            e = 1e-7
            zp = np.array(zc, dtype=float); zp[j] += e
            zm = np.array(zc, dtype=float); zm[j] -= e
            fd = (O.pointwise(p, zp) - O.pointwise(p, zm)) / (2 * e)
            assert np.allclose(J[:, j], fd, rtol=1e-5, atol=1e-6 * (1 + np.abs(fd).max())), (zc, j)
    n = 8
    z = I.bocf_spiral_cores(n, n, n_cores=1, seed=9)
    pg = O.problem(O.BOCF, nx=n, ny=n, dx=0.03, stencil=O.ST9, scheme=O.RK4, dt=0.05, variant=O.TANH_AS_HK)
    dz = I.uniform_pm1(21, z.size).reshape(z.shape)
    lam = I.uniform_pm1(22, z.size).reshape(z.shape)
    _, dzT = O.tlm(pg, z, dz, 5)
    lam0, _ = O.adjoint(pg, z, lam, 5)
    lhs, rhs = float(np.sum(lam * dzT)), float(np.sum(lam0 * dz))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
    eps = 1e-6
    fd = (O.step(pg, z + eps * dz, 5) - O.step(pg, z - eps * dz, 5)) / (2 * eps)
    assert np.linalg.norm(fd - dzT) <= 1e-6 * np.linalg.norm(dzT)
