"""Newton-Krylov solver for periodic orbits of the discrete flow.

Sect. 1 of the paper names matrix-free Newton-Krylov solvers for unstable
periodic orbits as the use that needs double precision.  This module finds
(z, T) with Phi_T(z) = z, Phi_T being n_steps steps of the plan's scheme with
dt = T / n_steps, by Newton's method on the bordered system

    [ J - I   F(Phi_T z) ] [dz]   [ -(Phi_T(z) - z) ]
    [ F(z)^T      0      ] [dT] = [        0        ]

(J = dPhi_T/dz at z; the last row is the phase condition that removes the
shift along the orbit; F(Phi_T z) is dPhi_T/dT of the continuous flow).
Each Newton step solves it by restarted GMRES with modified Gram-Schmidt.
Every vector operation runs in the library's kernels: J v by the
tangent-linear run (exact, not a difference of nearby solutions; from the
stage Jacobians one linearizing run keeps per iterate when they fit), F by
cg_rhs, inner products by cg_dot (fixed summation order) and updates by
cg_axpby; only the (m+1) x m Hessenberg least-squares problem and the
bordering scalars live on the host.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import replace
from typing import List, Optional

import numpy as np
import torch

from . import _lib, api


class _Vec:
    """Device vector kernels of the library on flat float64 CUDA tensors."""

    def __init__(self):
        self._ws = torch.empty(256, dtype=torch.float64, device="cuda")
        self._res = torch.empty(1, dtype=torch.float64, device="cuda")

    def dot(self, x: torch.Tensor, y: torch.Tensor) -> float:
        _lib.check(_lib.lib().cg_dot(x.data_ptr(), y.data_ptr(), x.numel(), self._res.data_ptr(),
                                     self._ws.data_ptr(), torch.cuda.current_stream().cuda_stream))
        return float(self._res.item())

    def axpby(self, a: float, x: torch.Tensor, b: float, y: torch.Tensor) -> None:
        """y = a x + b y"""
        _lib.check(_lib.lib().cg_axpby(float(a), x.data_ptr(), float(b), y.data_ptr(), x.numel(),
                                       torch.cuda.current_stream().cuda_stream))


def _givens(a: float, b: float):
    if b == 0.0:
        return 1.0, 0.0
    r = math.hypot(a, b)
    return a / r, b / r


def periodic_orbit(problem: api.Problem, z0: torch.Tensor, T0: float, n_steps: int, tol: float = 1e-11,
                   max_newton: int = 12, restart: int = 30, max_restarts: int = 4, gmres_rtol: float = 1e-7,
                   linearized: Optional[bool] = None, verbose: bool = False):
    """Newton-Krylov search for a periodic orbit through (z0, T0).

    ``problem`` is a single-instance problem whose ``dt`` is ignored (each
    iterate uses dt = T / n_steps).  ``linearized``: each Newton iterate
    keeps the stage Jacobians of its trajectory (n_steps x stages x NJ
    planes of device memory) so that every J v advances the tangent alone;
    otherwise each J v re-runs the primal.  Both give the same iterates bit
    for bit; None (the default) linearizes when that store takes at most
    half of the free device memory.  Returns (z, T, history) with history a list of dicts (Newton
    iteration, relative residual |Phi_T(z) - z| / |z|, T, GMRES iterations,
    final GMRES relative residual).
    """
    if not (isinstance(z0, torch.Tensor) and z0.is_cuda and z0.dtype == torch.float64):
        raise TypeError("z0 must be a float64 CUDA tensor")
    vec = _Vec()
    z = z0.contiguous().clone().reshape(-1)
    shape = z0.shape
    T = float(T0)
    hist: List[dict] = []

    def plan_for(T_):
        return api.Plan(replace(problem, dt=T_ / n_steps))

    if linearized is None:
        probe = plan_for(T)
        sz = ctypes.c_size_t()
        _lib.check(_lib.lib().cg_tlm_linearized_workspace_size(probe.handle, 1, int(n_steps), ctypes.byref(sz)))
        probe.close()
        linearized = sz.value <= torch.cuda.mem_get_info()[0] // 2

    for it in range(max_newton + 1):
        plan = plan_for(T)
        zs = z.view(shape)
        lin = plan.linearize(zs, n_steps) if linearized else None
        zT = (lin.zT if linearized else plan.run(zs, n_steps)).reshape(-1)
        r = zT.clone()
        vec.axpby(-1.0, z, 1.0, r)                        # r = Phi_T(z) - z
        rn = math.sqrt(vec.dot(r, r))
        zn = math.sqrt(vec.dot(z, z))
        rec = {"newton": it, "rel_residual": rn / zn, "T": T}
        hist.append(rec)
        if verbose:
            print("newton %d  |r|/|z| = %.3e  T = %.12g" % (it, rn / zn, T))
        if rn / zn <= tol or it == max_newton:
            if lin is not None:
                lin.status()
            plan.status()
            plan.close()
            break
        b = plan.rhs(zT.view(shape)).reshape(-1)          # dPhi/dT
        c = plan.rhs(zs).reshape(-1)                      # phase condition
        plan.status()

        def apply(v: torch.Tensor, s: float):
            v1 = v.view((1,) + tuple(shape))
            jv = lin.apply(v1) if linearized else plan.tlm(zs, v1, n_steps)[1]
            w = jv.reshape(-1)
            vec.axpby(-1.0, v, 1.0, w)                    # (J - I) v
            vec.axpby(s, b, 1.0, w)                       # + F(Phi_T z) s
            return w, vec.dot(c, v)

        # GMRES(restart) on A x = (-r, 0), x = (dz, dT), from x = 0
        dz = torch.zeros_like(z)
        dT = 0.0
        beta0 = rn
        n_it = 0
        gres = 1.0
        for _ in range(max_restarts):
            # residual of the current iterate
            if n_it == 0:
                q0 = r.clone()
                vec.axpby(0.0, r, -1.0, q0)               # -r
                q0s = 0.0
            else:
                w, ws_ = apply(dz, dT)
                q0 = r.clone()
                vec.axpby(-1.0, w, -1.0, q0)              # -r - A x
                q0s = -ws_
            beta = math.sqrt(vec.dot(q0, q0) + q0s * q0s)
            if beta <= gmres_rtol * beta0:
                break
            Q = [q0]
            Qs = [q0s / beta]
            vec.axpby(0.0, q0, 1.0 / beta, Q[0])
            H = np.zeros((restart + 1, restart))
            cs, sn = np.zeros(restart), np.zeros(restart)
            g = np.zeros(restart + 1)
            g[0] = beta
            k_done = 0
            for j in range(restart):
                w, ws_ = apply(Q[j], Qs[j])
                n_it += 1
                for i in range(j + 1):
                    h = vec.dot(w, Q[i]) + ws_ * Qs[i]
                    H[i, j] = h
                    vec.axpby(-h, Q[i], 1.0, w)
                    ws_ -= h * Qs[i]
                hn = math.sqrt(vec.dot(w, w) + ws_ * ws_)
                H[j + 1, j] = hn
                for i in range(j):
                    t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                    H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                    H[i, j] = t
                cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
                H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
                H[j + 1, j] = 0.0
                g[j + 1] = -sn[j] * g[j]
                g[j] = cs[j] * g[j]
                k_done = j + 1
                gres = abs(g[j + 1]) / beta0
                if gres <= gmres_rtol or hn == 0.0:
                    break
                vec.axpby(0.0, w, 1.0 / hn, w)
                Q.append(w)
                Qs.append(ws_ / hn)
            y = np.linalg.solve(np.triu(H[:k_done, :k_done]), g[:k_done])
            for i in range(k_done):
                vec.axpby(y[i], Q[i], 1.0, dz)
                dT += y[i] * Qs[i]
            if gres <= gmres_rtol:
                break
        rec["gmres_iterations"] = n_it
        rec["gmres_rel_residual"] = gres
        if lin is not None:
            lin.status()
            lin = None
        plan.close()
        vec.axpby(1.0, dz, 1.0, z)
        T += dT
    return z.view(shape), T, hist
