"""The library's own FP64 reciprocal, exponential and sigmoid against CUDA's
functions on the device and against numpy on the host."""
import numpy as np
import pytest

from paper_1309_1720_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _eval(fn, x):
    import torch
    from paper_1309_1720_gb300 import _lib
    xd = torch.from_numpy(x).cuda()
    own = torch.empty_like(xd)
    ref = torch.empty_like(xd)
    assert _lib.lib().cg_check_fastmath(fn, xd.data_ptr(), own.data_ptr(), ref.data_ptr(), xd.numel()) == 0
    return own.cpu().numpy(), ref.cpu().numpy()


def _ulps(a, b):
    return np.abs(a - b) / np.spacing(np.abs(b))


def test_reciprocal(cuda_ok):
    x = np.exp(np.log(0.5) + (np.log(2000.0) - np.log(0.5)) * I.uniform01(1, 1 << 20))
    own, ref = _eval(0, x)
    assert np.max(_ulps(own, ref)) <= 1.0
    assert np.max(_ulps(own, 1.0 / x)) <= 1.0


def test_exp(cuda_ok):
    x = -700.0 * I.uniform01(2, 1 << 20)
    x[:5] = [0.0, -1e-300, -708.0, -0.5, -1.0]
    own, ref = _eval(1, x)
    assert np.max(np.abs(own - ref) / ref) <= 4e-16
    assert np.max(np.abs(own - np.exp(x)) / np.exp(x)) <= 4e-16


def test_sigmoid(cuda_ok):
    x = 120.0 * (I.uniform01(3, 1 << 20) - 0.5)
    x[:4] = [0.0, -0.0, 40.0, -745.0]
    own, ref = _eval(2, x)
    exact = 1.0 / (1.0 + np.exp(-x))
    ok = x >= -700.0
    assert np.max(np.abs(own[ok] - exact[ok]) / exact[ok]) <= 6e-16
    # below -708 the exponential is held at e^-708: the value is within
    # 4e-308 of the true (subnormal or zero) one
    assert np.all(np.abs(own[~ok] - exact[~ok]) <= 4e-308)
    # (1 + tanh(x/2))/2 cancels for large negative x, so against CUDA's form
    # the comparison is absolute
    assert np.max(np.abs(own - ref)) <= 2.5e-16
