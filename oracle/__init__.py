"""CPU oracle for the cardiac reaction-diffusion step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it.

The arithmetic lives in ``cardiac_oracle.c`` (plain single-threaded FP64 C,
built with ``-O2 -ffp-contract=off``); this module only loads it with ctypes
and converts numpy arrays.  See the header of ``cardiac_oracle.c`` for the
paper passages each function restates.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cardiac_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FHN, BOCF, KARMA, DIFFUSION = 0, 1, 2, 3
ST5, ST9 = 0, 1
MIRROR, CLAMP, PERIODIC = 0, 1, 2
EULER, HEUN, RK4, RUSH_LARSEN, IMPLICIT_EULER = 0, 1, 2, 3, 4
AS_WRITTEN, TANH_AS_HK = 0, 1

MAXF, MAXP = 4, 32


class Problem(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int), ("stencil", ctypes.c_int),
        ("bc", ctypes.c_int), ("scheme", ctypes.c_int),
        ("nx", ctypes.c_long), ("ny", ctypes.c_long),
        ("dx", ctypes.c_double), ("dy", ctypes.c_double),
        ("alpha_d", ctypes.c_double), ("dt", ctypes.c_double),
        ("Dxx", ctypes.c_double * MAXF), ("Dyy", ctypes.c_double * MAXF),
        ("params", ctypes.c_double * MAXP),
        ("variant", ctypes.c_int),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (seconds)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(Problem)
            L.orc_n_fields.argtypes = [ctypes.c_int]; L.orc_n_fields.restype = ctypes.c_int
            L.orc_n_params.argtypes = [ctypes.c_int]; L.orc_n_params.restype = ctypes.c_int
            L.orc_default_params.argtypes = [ctypes.c_int, dp]; L.orc_default_params.restype = ctypes.c_int
            L.orc_Hk.argtypes = [ctypes.c_double, ctypes.c_double]; L.orc_Hk.restype = ctypes.c_double
            L.orc_dHk.argtypes = [ctypes.c_double, ctypes.c_double]; L.orc_dHk.restype = ctypes.c_double
            L.orc_pointwise.argtypes = [pp, dp, dp]; L.orc_pointwise.restype = None
            L.orc_pointwise_jac.argtypes = [pp, dp, dp]; L.orc_pointwise_jac.restype = None
            L.orc_apply_L.argtypes = [pp, ctypes.c_double, ctypes.c_double, dp, dp]
            L.orc_apply_L.restype = None
            L.orc_apply_LT.argtypes = [pp, ctypes.c_double, ctypes.c_double, dp, dp]
            L.orc_apply_LT.restype = None
            L.orc_rhs.argtypes = [pp, dp, dp]; L.orc_rhs.restype = ctypes.c_int
            L.orc_step.argtypes = [pp, dp, ctypes.c_long]; L.orc_step.restype = ctypes.c_int
            L.orc_tlm.argtypes = [pp, dp, dp, ctypes.c_long]; L.orc_tlm.restype = ctypes.c_int
            L.orc_adjoint.argtypes = [pp, dp, dp, dp, dp, ctypes.c_long]
            L.orc_adjoint.restype = ctypes.c_int
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def n_fields(model: int) -> int:
    return lib().orc_n_fields(model)


def default_params(model: int) -> np.ndarray:
    out = np.zeros(MAXP)
    n = lib().orc_default_params(model, _ptr(out))
    return out[:n].copy()


def problem(model=FHN, nx=64, ny=64, dx=0.04, dy=None, Dxx=None, Dyy=None,
            stencil=ST5, alpha_d=1.0 / 6.0, bc=MIRROR, scheme=EULER, dt=1e-4,
            params=None, variant=AS_WRITTEN) -> Problem:
    """Build the oracle's problem record.  Defaults: FHN diffusivities
    (D_u, D_v) = (1, 1.5); BOCF D_u = 1.171e-3 cm^2/ms, gates not diffusive;
    Karma gamma = D_u = 1.1e-3 cm^2/ms, v not diffusive.
    ``variant=TANH_AS_HK`` selects the Bueno-Orovio or Karma model with its
    tanh terms replaced by smoothed steps (Sect. 6)."""
    p = Problem()
    p.variant = variant
    p.model, p.stencil, p.bc, p.scheme = model, stencil, bc, scheme
    p.nx, p.ny = nx, ny
    p.dx = dx
    p.dy = dx if dy is None else dy
    p.alpha_d = alpha_d
    p.dt = dt
    if Dxx is None:
        Dxx = {FHN: [1.0, 1.5], BOCF: [1.171e-3, 0, 0, 0], KARMA: [1.1e-3, 0], DIFFUSION: [1.0]}[model]
    if Dyy is None:
        Dyy = Dxx
    for i in range(MAXF):
        p.Dxx[i] = Dxx[i] if i < len(Dxx) else 0.0
        p.Dyy[i] = Dyy[i] if i < len(Dyy) else 0.0
    prm = default_params(model) if params is None else np.asarray(params, dtype=np.float64)
    for i, v in enumerate(prm):
        p.params[i] = v
    return p


def Hk(x: float, k: float = 28.4) -> float:
    return lib().orc_Hk(x, k)


def dHk(x: float, k: float = 28.4) -> float:
    return lib().orc_dHk(x, k)


def pointwise(p: Problem, zc) -> np.ndarray:
    nv = n_fields(p.model)
    zc = np.ascontiguousarray(zc, dtype=np.float64)
    f = np.zeros(nv)
    lib().orc_pointwise(ctypes.byref(p), _ptr(zc), _ptr(f))
    return f


def pointwise_jac(p: Problem, zc) -> np.ndarray:
    nv = n_fields(p.model)
    zc = np.ascontiguousarray(zc, dtype=np.float64)
    J = np.zeros(nv * nv)
    lib().orc_pointwise_jac(ctypes.byref(p), _ptr(zc), _ptr(J))
    return J.reshape(nv, nv)


def apply_L(p: Problem, u: np.ndarray, Dxx: float, Dyy: float | None = None) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    lib().orc_apply_L(ctypes.byref(p), Dxx, Dxx if Dyy is None else Dyy, _ptr(u), _ptr(out))
    return out


def apply_LT(p: Problem, u: np.ndarray, Dxx: float, Dyy: float | None = None) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros_like(u)
    lib().orc_apply_LT(ctypes.byref(p), Dxx, Dxx if Dyy is None else Dyy, _ptr(u), _ptr(out))
    return out


def rhs(p: Problem, z: np.ndarray) -> np.ndarray:
    z = np.ascontiguousarray(z, dtype=np.float64)
    f = np.zeros_like(z)
    rc = lib().orc_rhs(ctypes.byref(p), _ptr(z), _ptr(f))
    assert rc == 0
    return f


def step(p: Problem, z: np.ndarray, n_steps: int) -> np.ndarray:
    """Return z advanced by n_steps (input untouched)."""
    z = np.array(z, dtype=np.float64, order="C", copy=True)
    rc = lib().orc_step(ctypes.byref(p), _ptr(z), n_steps)
    if rc != 0:
        raise ValueError("orc_step failed: %d" % rc)
    return z


def tlm(p: Problem, z: np.ndarray, dz: np.ndarray, n_steps: int):
    z = np.array(z, dtype=np.float64, order="C", copy=True)
    dz = np.array(dz, dtype=np.float64, order="C", copy=True)
    rc = lib().orc_tlm(ctypes.byref(p), _ptr(z), _ptr(dz), n_steps)
    if rc != 0:
        raise ValueError("orc_tlm failed: %d" % rc)
    return z, dz


def adjoint(p: Problem, z0: np.ndarray, lamT: np.ndarray, n_steps: int):
    z0 = np.ascontiguousarray(z0, dtype=np.float64)
    lamT = np.ascontiguousarray(lamT, dtype=np.float64)
    lam0 = np.zeros_like(z0)
    dLdD = np.zeros(MAXF)
    rc = lib().orc_adjoint(ctypes.byref(p), _ptr(z0), _ptr(lamT), _ptr(lam0), _ptr(dLdD), n_steps)
    if rc != 0:
        raise ValueError("orc_adjoint failed: %d" % rc)
    return lam0, dLdD[: n_fields(p.model)].copy()
