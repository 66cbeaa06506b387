"""Step-count and workspace-size limits of the C ABI: step counts above
CG_MAX_STEPS and workspace layouts whose byte count would not fit are
rejected with CG_EINVAL before anything is launched; a checkpoint interval
longer than the horizon is clamped to it."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

MAX_STEPS = 1 << 56
EINVAL = 1


def test_step_and_workspace_limits(cuda_ok):
    import torch
    from paper_1309_1720_gb300 import Plan, Problem, FHN, RK4, _lib
    L = _lib.lib()
    plan = Plan(Problem(model=FHN, nx=64, ny=48, dx=0.04, scheme=RK4, dt=1e-4))
    h = plan.handle
    sz = ctypes.c_size_t()
    # counts beyond the limit
    assert L.cg_adjoint_workspace_size(h, MAX_STEPS + 1, 0, ctypes.byref(sz)) == EINVAL
    assert L.cg_tlm_linearized_workspace_size(h, 1, MAX_STEPS + 1, ctypes.byref(sz)) == EINVAL
    assert L.cg_newton_linearized_workspace_size(h, 30, MAX_STEPS + 1, ctypes.byref(sz)) == EINVAL
    # counts within it whose layouts would overflow: 2^56 checkpoints, 2^58 stage Jacobians
    assert L.cg_adjoint_workspace_size(h, MAX_STEPS, 1, ctypes.byref(sz)) == EINVAL
    assert L.cg_tlm_linearized_workspace_size(h, 1, MAX_STEPS, ctypes.byref(sz)) == EINVAL
    assert L.cg_newton_linearized_workspace_size(h, 30, MAX_STEPS, ctypes.byref(sz)) == EINVAL
    # the largest tangent count has a representable size
    assert L.cg_tlm_workspace_size(h, 2 ** 31 - 1, ctypes.byref(sz)) == 0 and sz.value > 2 ** 40
    # a checkpoint interval beyond the horizon costs no more than the horizon
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    assert L.cg_adjoint_workspace_size(h, 10, 10, ctypes.byref(a)) == 0
    assert L.cg_adjoint_workspace_size(h, 10, 1000, ctypes.byref(b)) == 0
    assert a.value == b.value
    # run entry points
    z = torch.zeros(2 * 48 * 64, dtype=torch.float64, device="cuda")
    ws = plan.workspace()
    assert L.cg_run(h, z.data_ptr(), z.data_ptr(), MAX_STEPS + 1, ws.data_ptr(), None) == EINVAL
    assert L.cg_run(h, z.data_ptr(), z.data_ptr(), -1, ws.data_ptr(), None) == EINVAL
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.close()
