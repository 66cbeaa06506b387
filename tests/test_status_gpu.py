"""cg_get_device_status: the device status of the latest run issued with a
plan, read without naming its workspace."""
import ctypes

import numpy as np
import pytest

from paper_1309_1720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_device_status_of_latest_run(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, _lib
    L = _lib.lib()
    plan = Plan(Problem(model=FHN, nx=64, ny=48, dx=0.04, dt=1e-4))
    flags = ctypes.c_uint32(7)
    assert L.cg_get_device_status(plan.handle, ctypes.byref(flags)) == 0 and flags.value == 0
    z = I.fhn_broken_wave(64, 48)
    plan.run(torch.from_numpy(z).cuda(), 5)
    assert L.cg_get_device_status(plan.handle, ctypes.byref(flags)) == 0 and flags.value == 0
    bad = z.copy()
    bad[0, 3, 3] = np.nan
    plan.run(torch.from_numpy(bad).cuda(), 5)
    assert L.cg_get_device_status(plan.handle, ctypes.byref(flags)) == 5 and flags.value == 1
    # a tangent-linear run with its own workspace becomes the latest run
    zd = torch.from_numpy(z).cuda()
    plan.tlm(zd, zd[None].clone(), 3)
    assert L.cg_get_device_status(plan.handle, ctypes.byref(flags)) == 0 and flags.value == 0
