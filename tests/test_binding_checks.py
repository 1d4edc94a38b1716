"""Argument checks of the Python binding, which guard the C ABI against buffers of the wrong size (CPU)."""
import numpy as np
import pytest

from paper_2509_23945_gb300 import tnmc


def test_items_must_pair_up():
    c, s = tnmc._items([0, 1, 2], [0, 2, 4])
    assert c.dtype == np.int32 and s.dtype == np.int32 and c.shape == (3,)
    with pytest.raises(ValueError):
        tnmc._items([0, 1, 2], [0, 2])
    with pytest.raises(ValueError):
        tnmc._items([[0, 1]], [[0, 2]])


def test_shape_check():
    tnmc._expect_shape("spins", (2, 4, 5, 6), (2, 4, 5, 6))
    with pytest.raises(ValueError):
        tnmc._expect_shape("spins", (2, 6, 5, 4), (2, 4, 5, 6))


def test_accept_counter_must_be_a_large_enough_int32_device_tensor():
    torch = pytest.importorskip("torch")
    tnmc._check_counter(None, 8)
    with pytest.raises(ValueError):                      # host tensor
        tnmc._check_counter(torch.zeros(8, dtype=torch.int32), 8)

    class FakeDeviceTensor:                               # stands in for a CUDA tensor on a CPU-only machine
        is_cuda = True

        def __init__(self, n, dtype):
            self.n, self.dtype = n, dtype

        def is_contiguous(self):
            return True

        def numel(self):
            return self.n

    tnmc._check_counter(FakeDeviceTensor(8, torch.int32), 8)
    with pytest.raises(ValueError):
        tnmc._check_counter(FakeDeviceTensor(7, torch.int32), 8)
    with pytest.raises(ValueError):
        tnmc._check_counter(FakeDeviceTensor(8, torch.int64), 8)


def test_noalloc_binding_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    spins = torch.zeros((4, 4, 4), dtype=torch.int8)
    with pytest.raises(ValueError):
        tnmc._check_device_tensor("spins", spins, torch.int8, (4, 4, 4))
    with pytest.raises(ValueError):
        tnmc._check_device_tensor("spins", np.zeros((4, 4, 4), dtype=np.int8), torch.int8, (4, 4, 4))
