"""The checked build (libcardiac_gb300_checked.so, -DCG_BOUNDS_CHECK): every
stage worker of the forward, tangent-linear, adjoint and temporally blocked
kernels checks the grid and window indices it is about to use.  Run in a
child process over the workloads of checked_cases.py, no run may report a
device error (CG_EBOUNDS included), and every result must equal the plain
build's bit for bit (the checks add integer compares only)."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_checked_build_clean_and_bitwise_equal(cuda_ok, tmp_path):
    from paper_1309_1720_gb300 import build, _lib
    import checked_cases
    if _lib.CHECKED:
        pytest.skip("this process already runs the checked build")
    build.build(checked=True)
    npz = str(tmp_path / "checked.npz")
    env = dict(os.environ, CG_BOUNDS_CHECK="1")
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py"), npz], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-4000:], r.stderr[-4000:])
    assert _lib.lib().cg_bounds_checked() == 0
    plain = checked_cases.run_all()
    chk = np.load(npz)
    assert set(chk.files) == set(plain)
    assert len(plain) > 400
    for k, v in plain.items():
        assert np.array_equal(chk[k], v), k
