"""Seeded synthetic inputs for the cardiac reaction-diffusion stepper.

This module only *builds inputs*: initial states, grid-size draws, random
directions and parameter sweeps.  It contains none of the stepping arithmetic
(no stencil, no ionic model, no integrator), so that the CUDA path and the CPU
oracle can both consume the same arrays without sharing any of the method.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), implemented here from its
published definition with numpy uint64 arithmetic.  Uniforms take the top 53
bits of each output.

Layout of every state: a C-contiguous float64 array ``[n_v, ny, nx]``; ``x`` is
the column index (contiguous), ``y`` the row index.  "Left" means small ``x``
and "lower half" means ``y < ny/2`` (y grows upward).

The workloads follow the paper's two-dimensional tissue simulations (Sect. 2,
Fig. 3): FitzHugh-Nagumo with dx = 0.04 and the Bueno-Orovio-Cherry-Fenton
model with dx = 0.03 cm.  No dataset is involved.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# FitzHugh-Nagumo rest point for (eps, a1, a0) = (0.05, 1.5, -0.1), Eq. (fhn):
# the real root near -0.659 of 1.5 u^3 - 0.5 u + 0.1 = 0 and v = (u - a0)/a1.
# Stored as plain numbers (input values, not model arithmetic).
FHN_U_REST = -0.6591465811607408
FHN_V_REST = -0.37276438744049384

FHN_DX = 0.04          # Sect. 2, FitzHugh-Nagumo spatial step
BOCF_DX = 0.03         # Sect. 2, Bueno-Orovio spatial step [cm]
BOCF_D = 1.171e-3      # Sect. 2, D = 1.171 cm^2/s expressed in cm^2/ms
KARMA_DX = 0.0262      # Sect. 2, Karma spatial step [cm]
KARMA_GAMMA = 1.1e-3   # Sect. 2, gamma = 0.0011 (cm^2/ms)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+n-1`` of the SplitMix64 stream for ``seed``.

    Output i mixes state ``seed + (i+1)*0x9E3779B97F4A7C15`` (mod 2^64).
    """
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of SplitMix64 outputs."""
    z = splitmix64(seed, n, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles in [-1, 1)."""
    return 2.0 * uniform01(seed, n, offset) - 1.0


def gaussian(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform01(seed, 2 * m, offset)
    u1 = 1.0 - u[0::2]            # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    g = np.empty(2 * m)
    g[0::2] = r * np.cos(2.0 * math.pi * u2)
    g[1::2] = r * np.sin(2.0 * math.pi * u2)
    return g[:n]


def fhn_broken_wave(nx: int, ny: int, width: int | None = None, seed: int = 0,
                    noise: float = 1e-3) -> np.ndarray:
    """Broken plane wave for the two-field model, shape ``[2, ny, nx]``.

    u is excited (u = 1) in the ``width`` left columns, v is refractory
    (v = 0.6) in the lower half ``y < ny/2``; elsewhere the rest point.  Then
    ``u += noise * U[-1, 1)`` drawn in row-major (y, x) order from ``seed``.
    ``width`` defaults to 10 columns per 128 (10 at 128^2, 80 at 1024^2).
    """
    if width is None:
        width = max(1, (10 * nx) // 128)
    z = np.empty((2, ny, nx), dtype=np.float64)
    z[0] = FHN_U_REST
    z[1] = FHN_V_REST
    z[0, :, :width] = 1.0
    z[1, : ny // 2, :] = 0.6
    z[0] += noise * uniform_pm1(seed, nx * ny).reshape(ny, nx)
    return z


def karma_broken_wave(nx: int, ny: int, width: int | None = None, seed: int = 0,
                      noise: float = 1e-3) -> np.ndarray:
    """Broken plane wave for the Karma model, shape ``[2, ny, nx]``.

    u is excited (u = 3) in the ``width`` left columns and rests at 0
    elsewhere; v is refractory (v = 1.2, so v^6 > u* blocks excitation) in
    the lower half ``y < ny/2`` and 0 elsewhere.  Then ``u += noise *
    U[0, 1)`` drawn in row-major (y, x) order from ``seed``.  ``width``
    defaults to 10 columns per 128.
    """
    if width is None:
        width = max(1, (10 * nx) // 128)
    z = np.zeros((2, ny, nx), dtype=np.float64)
    z[0, :, :width] = 3.0
    z[1, : ny // 2, :] = 1.2
    z[0] += noise * uniform01(seed, nx * ny).reshape(ny, nx)
    return z


def bocf_spiral_cores(nx: int, ny: int, n_cores: int = 8, seed: int = 0,
                      noise: float = 1e-3) -> np.ndarray:
    """Seeded multi-core initial state for the four-field model, ``[4, ny, nx]``.

    ``n_cores`` phase singularities are placed uniformly in the inner 80% of
    the domain with random chirality; the phase is
    ``theta = sum_c chi_c * atan2(y - y_c, x - x_c)`` and ``phi = (theta mod
    2 pi) / 2 pi``.  Fields are smooth synthetic profiles of ``phi`` that put
    cells in excited (u ~ 1.5, v ~ 0), recovering and resting (u ~ 0, v ~ 1)
    states, so every branch of the gating switches is visited.  Then
    ``u += noise * U[-1, 1)``.
    """
    r = uniform01(seed, 3 * n_cores)
    xc = (0.1 + 0.8 * r[0::3]) * (nx - 1)
    yc = (0.1 + 0.8 * r[1::3]) * (ny - 1)
    chi = np.where(r[2::3] < 0.5, -1.0, 1.0)
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64),
                       np.arange(nx, dtype=np.float64), indexing="ij")
    theta = np.zeros((ny, nx))
    for c in range(n_cores):
        theta += chi[c] * np.arctan2(y - yc[c], x - xc[c])
    phi = np.mod(theta, 2.0 * math.pi) / (2.0 * math.pi)
    z = np.empty((4, ny, nx), dtype=np.float64)
    z[0] = 1.5 * np.exp(-(phi / 0.22) ** 2)                      # voltage
    z[1] = np.clip((phi - 0.35) / 0.55, 0.0, 1.0)                 # fast gate
    z[2] = 0.45 + 0.5 * phi                                       # slow gate
    z[3] = 0.85 * np.exp(-(phi / 0.45) ** 2)                      # s gate
    z[0] += noise * uniform_pm1(seed + 1, nx * ny).reshape(ny, nx)
    return z


def batch_sizes(n_inst: int = 256, lo: int = 64, hi: int = 512, seed: int = 1) -> np.ndarray:
    """Square instance sizes drawn uniformly from ``lo..hi`` (inclusive)."""
    u = uniform01(seed, n_inst)
    return lo + np.floor(u * (hi - lo + 1)).astype(np.int64)


def unit_direction(shape, seed: int, offset: int = 0, norm: float = 1.0) -> np.ndarray:
    """A Gaussian random direction of the given shape with 2-norm ``norm``."""
    n = int(np.prod(shape))
    g = gaussian(seed, n, offset).reshape(shape)
    return g * (norm / np.sqrt(np.sum(g * g)))


def batch_workload(n_inst: int = 256, seed: int = 1, lo: int = 64, hi: int = 512,
                   d_u: float = 1.0, sizes=None):
    """Uneven batch of two-field instances.

    Returns ``(sizes, states, d_u_per_instance)``.  The first half are the
    broken-wave base state of their own size plus a Krylov-style perturbation
    of 2-norm 1e-7 in a Gaussian direction; the second half are the base
    state with ``D_u * (1 + 0.2 U[-1, 1))`` (a +/-20% parameter sweep).
    """
    if sizes is None:
        sizes = batch_sizes(n_inst, lo, hi, seed)
    half = n_inst // 2
    sweep = uniform_pm1(seed + 1000, n_inst)
    states, dus = [], []
    for i, n in enumerate(sizes):
        n = int(n)
        z = fhn_broken_wave(n, n, seed=0)
        if i < half:
            z = z + unit_direction(z.shape, seed, offset=i * 4 * 512 * 512, norm=1e-7)
            dus.append(d_u)
        else:
            dus.append(d_u * (1.0 + 0.2 * sweep[i]))
        states.append(np.ascontiguousarray(z))
    return np.asarray(sizes, dtype=np.int64), states, np.asarray(dus)
