"""Argument checks of the Python binding that need no GPU: the helper that
every Plan entry point runs before handing pointers to the C ABI rejects
wrong dtypes, devices, layouts and element counts with an exception (not
an assert, so the checks survive ``python -O``)."""
import pytest
import torch

from paper_1309_1720_gb300.api import _state


def test_state_accepts_a_matching_tensor():
    t = torch.zeros(3, 4, 5, dtype=torch.float64)
    assert _state(t, 60, "z", cuda=False) is t
    assert _state(t, None, "z", cuda=False) is t


@pytest.mark.parametrize("bad,cuda,exc", [
    (torch.zeros(60, dtype=torch.float32), False, TypeError),           # wrong dtype
    (torch.zeros(59, dtype=torch.float64), False, ValueError),          # wrong element count
    (torch.zeros(6, 10, dtype=torch.float64).t(), False, ValueError),   # not contiguous
    (torch.zeros(60, dtype=torch.float64), True, ValueError),           # host tensor where a device one is needed
    ([0.0] * 60, False, TypeError),                                     # not a tensor
])
def test_state_rejects(bad, cuda, exc):
    with pytest.raises(exc):
        _state(bad, 60, "z", cuda=cuda)
