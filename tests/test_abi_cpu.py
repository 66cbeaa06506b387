"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point the public header declares, validates problems before any
device call, and carries the same model constants as the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1309_1720_gb300 import build, _lib
    build.build()
    return _lib.lib()


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(cg_[a-z0-9_]+)\s*\(",
                                src, flags=re.M)
    return names


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n


def test_abi_version(L):
    assert L.cg_abi_version() == 1


def test_default_params_match_oracle(L):
    import oracle as O
    from paper_1309_1720_gb300 import api
    for m_abi, m_orc in [(api.FHN, O.FHN), (api.BOCF, O.BOCF), (api.KARMA, O.KARMA)]:
        assert api.n_fields(m_abi) == O.n_fields(m_orc)
        assert np.array_equal(np.array(api.default_params(m_abi)), O.default_params(m_orc))


def _create(prob):
    from paper_1309_1720_gb300 import _lib
    c = prob.to_c()
    h = ctypes.c_void_p()
    st = _lib.lib().cg_plan_create(ctypes.byref(c), ctypes.byref(h))
    return st, _lib.lib().cg_last_error().decode()


@pytest.mark.parametrize("kw,status", [
    (dict(nx=1), 1), (dict(ny=0), 1), (dict(dx=0.0), 1), (dict(dt=-1.0), 1),
    (dict(stencil=7), 1), (dict(bc=5), 1), (dict(scheme=9), 1), (dict(model=42), 1),
    (dict(model=2, dx=0.0262, dt=0.05, D=(1.1e-3, 1e-3)), 7),   # Karma: v does not diffuse
    (dict(model=2, dx=0.0262, dt=0.05, scheme=3), 7),            # Karma: no gate integrators
    (dict(model=2, dx=0.0262, dt=0.05, params=[2.5, 250, 1.5415, 3, 1, 0, 6, 28.4]), 1),  # Re = 0
    (dict(model=2, dx=0.0262, dt=0.2), 4),  # FE bound h^2/(4 gamma) = 0.156 ms
    (dict(dt=3e-4), 4),                     # FE bound for FHN at dx=0.04 is 2.67e-4
    (dict(scheme=2, dt=5.6e-4), 4),         # RK4 5-point bound 3.71e-4
    (dict(stencil=1, alpha_d=0.4), 1),
    (dict(params=[0.05, 1.5]), 1),
    (dict(scheme=3), 7), (dict(scheme=4), 7),   # gate integrators: four-field model only
    (dict(flags=1 << 3), 7),                # tanh variant: four-field and Karma models only
    (dict(bc=3), 1), (dict(scheme=5), 1),
])
def test_validation_errors(L, kw, status):
    from paper_1309_1720_gb300 import Problem
    st, msg = _create(Problem(**kw))
    assert st == status, msg
    assert msg


def test_bocf_gate_diffusion_rejected(L):
    from paper_1309_1720_gb300 import Problem, BOCF
    st, msg = _create(Problem(model=BOCF, dx=0.03, dt=0.05, D=(1e-3, 1e-3)))
    assert st == 7 and "diffuse" in msg


def test_gate_integrators_need_positive_time_constants(L):
    from paper_1309_1720_gb300 import Problem, BOCF, RUSH_LARSEN, default_params
    prm = default_params(BOCF)
    prm[8] = -1.0                           # tau_v+ < 0
    st, msg = _create(Problem(model=BOCF, dx=0.03, dt=0.05, scheme=RUSH_LARSEN, params=prm))
    assert st == 1 and "positive" in msg


def test_temporal_blocking_rejected_before_device_work(L):
    """Temporal blocking needs one instance, mirror or clamp ghosts and an
    explicit scheme; the checks come before any device call."""
    from paper_1309_1720_gb300 import Problem, FHN, BOCF, PERIODIC, RUSH_LARSEN, _lib
    from paper_1309_1720_gb300._lib import CTuning
    for prob in (Problem(model=FHN, bc=PERIODIC), Problem(model=BOCF, dx=0.03, dt=0.05, scheme=RUSH_LARSEN)):
        c = prob.to_c()
        tun = CTuning(0, 2, 256, 0, 2)
        h = ctypes.c_void_p()
        st = _lib.lib().cg_plan_create_tuned(ctypes.byref(c), ctypes.byref(tun), ctypes.byref(h))
        assert st == 7, _lib.lib().cg_last_error().decode()
    c = Problem(model=FHN).to_c()
    h = ctypes.c_void_p()
    st = _lib.lib().cg_plan_create_tuned(ctypes.byref(c), ctypes.byref(CTuning(0, 65, 256, 0, 2)), ctypes.byref(h))
    assert st == 1


def test_linearized_tangent_entry_points_reject_null_plan(L):
    """The linearized tangent-linear and Newton entry points check their
    arguments before touching the device."""
    sz = ctypes.c_size_t()
    assert L.cg_tlm_linearized_workspace_size(None, 1, 10, ctypes.byref(sz)) == 1
    assert L.cg_tlm_linearize(None, None, None, 10, None, None) == 1
    assert L.cg_tlm_apply(None, None, None, 1, 10, None, None) == 1
    assert L.cg_newton_linearized_workspace_size(None, 30, 10, ctypes.byref(sz)) == 1
    hist = (ctypes.c_double * 2)()
    nit = ctypes.c_int32()
    assert L.cg_newton_gmres_step_linearized(None, None, 10, 30, 1, 1e-8, None, hist, ctypes.byref(nit),
                                             None, None) == 1


def test_checkpointed_adjoint_entry_points_reject_null_plan(L):
    """The split adjoint (forward keeping checkpoints, reverse from them)
    checks its arguments before touching the device."""
    sz = ctypes.c_size_t()
    assert L.cg_adjoint_checkpoint_size(None, 10, 0, ctypes.byref(sz)) == 1
    assert L.cg_adjoint_forward(None, None, None, 10, 0, None, None, None) == 1
    assert L.cg_adjoint_reverse(None, None, None, None, None, 10, 0, None, None) == 1


def test_checked_build_loads_and_exports(L):
    """The checked build (index checks in every stage worker) is a drop-in
    replacement: same exported symbols, selected by CG_BOUNDS_CHECK=1."""
    import subprocess
    import sys
    from paper_1309_1720_gb300 import build, _lib
    build.build(checked=True)
    assert L.cg_bounds_checked() == (1 if _lib.CHECKED else 0)
    chk = ctypes.CDLL(build.LIB_CHECKED)
    chk.cg_bounds_checked.restype = ctypes.c_int32
    assert chk.cg_bounds_checked() == 1
    for n in declared_functions():
        assert hasattr(chk, n), n
    code = ("from paper_1309_1720_gb300 import _lib; import sys; "
            "sys.exit(0 if _lib.lib().cg_bounds_checked() == 1 else 3)")
    env = dict(os.environ, CG_BOUNDS_CHECK="1")
    assert subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env).returncode == 0


def test_bocf_sharpness_must_be_positive(L):
    from paper_1309_1720_gb300 import Problem, BOCF, default_params
    prm = default_params(BOCF)
    prm[28] = 0.0
    st, msg = _create(Problem(model=BOCF, dx=0.03, dt=0.05, params=prm))
    assert st == 1 and "sharpness" in msg
