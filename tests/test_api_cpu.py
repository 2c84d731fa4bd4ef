"""Host side of the Python binding, without a GPU: argument errors surface
before any device work, and a call on a machine without a GPU fails loudly
-- the binding has no CPU path to fall back to."""
import pytest
import torch

import paper_1907_04834_gb300 as gs


def test_dtype_and_shape_checked_before_device_work():
    q32 = torch.zeros((10, 3), dtype=torch.float32)
    with pytest.raises(TypeError):
        gs.shoot(q32, q32, 1.0, 4)
    q2 = torch.zeros((10, 2), dtype=torch.float64)
    with pytest.raises(ValueError):
        gs.shoot(q2, q2, 1.0, 4)
    a = torch.zeros((10, 3), dtype=torch.float64)
    b = torch.zeros((9, 3), dtype=torch.float64)
    with pytest.raises(ValueError):
        gs.shoot_grad(a, a, b, 1.0, 4)
    with pytest.raises(ValueError):
        gs.rhs(a, b, 1.0)


@pytest.mark.skipif(torch.cuda.is_available(), reason="the behaviour without a GPU")
def test_no_cpu_fallback_without_a_gpu():
    from paper_1907_04834_gb300 import native
    native.build()
    a = torch.zeros((10, 3), dtype=torch.float64)
    with pytest.raises(gs.GSError):
        gs.shoot(a, a, 1.0, 4)
    with pytest.raises(gs.GSError):
        gs.shoot_grad(a, a, a, 1.0, 4, mode="bh")
