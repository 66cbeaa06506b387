"""Workloads shared by the checked-build test: every kernel family (forward
stage kernels of all models, stencils, schemes and ghost rules; the tile
queue, neighbour-synchronised, per-stage and temporally blocked launches;
batches; tangent-linear, linearized and adjoint runs; the right-hand side)
on ragged shapes.  ``run_all()`` returns a dict of result arrays; run as a
script it writes them to the .npz file named on the command line after
checking that no run reported a device error (with the checked library,
that includes CG_EBOUNDS).  Not a test module itself."""
from __future__ import annotations

import sys

import numpy as np


def _problem(model, nx, ny, stencil, scheme, bc, **kw):
    from paper_1309_1720_gb300 import Problem, inputs as I
    if model == 0:
        return Problem(model=0, nx=nx, ny=ny, dx=0.04, stencil=stencil, scheme=scheme, bc=bc, dt=1e-4, **kw)
    if model == 1:
        return Problem(model=1, nx=nx, ny=ny, dx=0.03, D=(1.171e-3,), Dyy=(1.171e-3 / 4,), stencil=stencil,
                       scheme=scheme, bc=bc, dt=0.05, **kw)
    if model == 2:
        return Problem(model=2, nx=nx, ny=ny, dx=I.KARMA_DX, stencil=stencil, scheme=scheme, bc=bc, dt=0.05, **kw)
    return Problem(model=3, nx=nx, ny=ny, dx=0.1, D=(1.0,), Dyy=(0.6,), stencil=stencil, scheme=scheme, bc=bc,
                   dt=1e-3, **kw)


def _state(model, nx, ny, seed=0):
    from paper_1309_1720_gb300 import inputs as I
    if model == 0:
        return I.fhn_broken_wave(nx, ny, width=max(1, nx // 6), seed=seed)
    if model == 1:
        return I.bocf_spiral_cores(nx, ny, n_cores=2, seed=seed)
    if model == 2:
        z = I.karma_broken_wave(nx, ny, width=max(1, nx // 6), seed=seed)
        z[1] += 0.4 * I.uniform01(seed + 11, nx * ny).reshape(ny, nx)
        return z
    return (1.0 + 0.3 * I.uniform_pm1(9 + seed, nx * ny)).reshape(1, ny, nx)


def run_all() -> dict:
    import torch
    from paper_1309_1720_gb300 import Plan, inputs as I
    out = {}

    def run(name, p, z0, n, tuning=None):
        plan = Plan(p, tuning=tuning)
        r = plan.run(torch.from_numpy(np.ascontiguousarray(z0)).cuda(), n)
        plan.status()
        out[name] = r.cpu().numpy()
        plan.close()

    shapes = [(2, 2), (3, 7), (67, 45), (130, 66)]
    for model in (0, 1, 2, 3):
        for stencil in (0, 1):
            schemes = (0, 1, 2, 3, 4) if model == 1 else (0, 1, 2)
            for scheme in schemes:
                for bc in (0, 1, 2):
                    for nx, ny in shapes:
                        name = "fwd_m%d_s%d_i%d_b%d_%dx%d" % (model, stencil, scheme, bc, nx, ny)
                        run(name, _problem(model, nx, ny, stencil, scheme, bc), _state(model, nx, ny), 5)
    # launch shapes and synchronisation modes
    from paper_1309_1720_gb300 import FLAG_NEIGHBOR_SYNC, FLAG_PER_STAGE_LAUNCH
    tunings = [dict(cells_x=1, threads=128), dict(cells_x=2, threads=256, blocks_per_sm=2),
               dict(schedule=1, rows=1), dict(schedule=1, rows=8, cells_x=1), dict(threads=384, cells_x=1)]
    for i, tun in enumerate(tunings):
        for model in (0, 1):
            run("tun%d_m%d" % (i, model), _problem(model, 150, 97, 1, 2, 0), _state(model, 150, 97), 4, tun)
    for flags, tag in ((FLAG_NEIGHBOR_SYNC, "nbr"), (FLAG_PER_STAGE_LAUNCH, "pstage")):
        run("mode_%s" % tag, _problem(0, 150, 97, 1, 2, 0, flags=flags), _state(0, 150, 97), 4)
    # temporal blocking
    for model in (0, 1, 2):
        for nx, ny in ((128, 128), (67, 45), (3, 7), (512, 2)):
            for k in (1, 3):
                run("tb_m%d_%dx%d_k%d" % (model, nx, ny, k), _problem(model, nx, ny, 1, 2, 0),
                    _state(model, nx, ny), 7, dict(schedule=2, rows=k))
    # temporal blocking with neighbour waits between passes
    for model in (0, 1):
        for nx, ny in ((128, 128), (67, 45), (3, 7)):
            run("tbn_m%d_%dx%d" % (model, nx, ny), _problem(model, nx, ny, 1, 2, 0, flags=FLAG_NEIGHBOR_SYNC),
                _state(model, nx, ny), 7, dict(schedule=2, rows=2))
    # four-field constants whose v^- and o switches differ (evaluated apart)
    from paper_1309_1720_gb300 import default_params
    prm = default_params(1)
    prm[5] = 0.02
    run("bocf_tho", _problem(1, 67, 45, 1, 2, 0, params=prm), _state(1, 67, 45), 6)
    # batch of uneven instances
    probs = [_problem(0, nx, ny, 0, 2, 0) for nx, ny in ((64, 64), (33, 90), (128, 20), (5, 5))]
    plan = Plan(probs)
    res = plan.unpack(plan.run(plan.pack([_state(0, p.nx, p.ny, seed=i) for i, p in enumerate(probs)]), 6))
    plan.status()
    for i, r in enumerate(res):
        out["batch_%d" % i] = r.cpu().numpy()
    for k in (1, 2):
        tplan = Plan(probs, tuning=dict(schedule=2, rows=k))
        res = tplan.unpack(tplan.run(tplan.pack([_state(0, p.nx, p.ny, seed=i) for i, p in enumerate(probs)]), 6))
        tplan.status()
        for i, r in enumerate(res):
            out["tbatch_k%d_%d" % (k, i)] = r.cpu().numpy()
    # tangent-linear, linearized, adjoint and right-hand side
    for model in (0, 1, 2):
        for stencil in (0, 1):
            p = _problem(model, 70, 45, stencil, 2, 0)
            z0 = torch.from_numpy(_state(model, 70, 45)).cuda()
            dz = torch.from_numpy(np.stack([I.unit_direction(tuple(z0.shape), 30 + i) for i in range(3)])).cuda()
            plan = Plan(p)
            zT, dzT = plan.tlm(z0, dz, 6)
            plan.status()
            lin = plan.linearize(z0, 6, max_tangents=3)
            dzL = lin.apply(dz)
            lin.status()
            lam0, dLdD = plan.adjoint(z0, zT.clone(), 6)
            plan.status()
            lamA, dLdDA = plan.adjoint(z0, zT.clone(), 6, checkpoint_every=6)
            plan.status()
            f = plan.rhs(z0)
            plan.status()
            tag = "m%d_s%d" % (model, stencil)
            out["tlm_z_" + tag] = zT.cpu().numpy()
            out["tlm_dz_" + tag] = dzT.cpu().numpy()
            out["lin_dz_" + tag] = dzL.cpu().numpy()
            out["adj_lam_" + tag] = lam0.cpu().numpy()
            out["adj_dD_" + tag] = dLdD.cpu().numpy()
            out["adjall_lam_" + tag] = lamA.cpu().numpy()
            out["rhs_" + tag] = f.cpu().numpy()
            plan.close()
    return out


if __name__ == "__main__":
    from paper_1309_1720_gb300 import _lib
    assert _lib.lib().cg_bounds_checked() == (1 if _lib.CHECKED else 0)
    np.savez(sys.argv[1], **run_all())
