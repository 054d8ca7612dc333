"""The binding refuses device and host buffers that do not match what the kernels
behind the pointer read or write (dtype, device, contiguity, exact shape), before
anything reaches the library: a wrong buffer would make a kernel access memory
outside it. Runs on the CPU: CUDA tensors are stood in for by objects with the
same attributes, and the library is never loaded."""
import numpy as np
import pytest
import torch

from paper_1404_3816_gb300 import binding as B


class FakeCuda:
    """Duck-typed stand-in for a CUDA tensor (the checks read only these attributes)."""

    def __init__(self, shape, dtype=torch.float64, contiguous=True, index=0):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.is_cuda = True
        self._contig = contiguous
        self.device = type("Dev", (), {"index": index})()

    def is_contiguous(self):
        return self._contig

    def data_ptr(self):
        return 4096


@pytest.fixture(autouse=True)
def no_library(monkeypatch):
    def boom(*a, **k):
        raise AssertionError("the library was reached with a rejected buffer")
    monkeypatch.setattr(B, "load", boom)


def _einval(fn, *args):
    with pytest.raises(B.HikfError) as e:
        fn(*args)
    assert e.value.code == B.HIKF_EINVAL
    return str(e.value)


@pytest.mark.parametrize("S,M,word", [
    (torch.eye(4, dtype=torch.float64), torch.eye(4, dtype=torch.float64), "not on a CUDA"),
    (FakeCuda((4, 4), torch.float32), FakeCuda((4, 4)), "dtype"),
    (FakeCuda((4, 4)), FakeCuda((4, 4), torch.float32), "dtype"),
    (FakeCuda((4, 4)), FakeCuda((4, 3)), "shape"),
    (FakeCuda((4, 4)), FakeCuda((16,)), "shape"),
    (FakeCuda((4, 4), contiguous=False), FakeCuda((4, 4)), "contiguous"),
    (FakeCuda((4, 4)), FakeCuda((4, 4), index=1), "cuda:1"),
    (FakeCuda((4, 5)), FakeCuda((4, 5)), "shape"),
    (np.eye(4), np.eye(4), "torch CUDA tensor"),
])
@pytest.mark.parametrize("fn", ["spd_inverse", "spd_inverse_noalloc"])
def test_spd_inverse_rejects_wrong_buffers(fn, S, M, word):
    msg = _einval(getattr(B, fn), S, M)
    assert word in msg


def _filter(m=10, n=3, device=0):
    f = object.__new__(B.Filter)
    f.h, f.m, f.n, f.dim, f.device = None, m, n, 2, device
    return f


@pytest.mark.parametrize("y,word", [
    (FakeCuda((4,)), "shape"),
    (FakeCuda((3,), torch.float32), "dtype"),
    (FakeCuda((3,), contiguous=False), "contiguous"),
    (FakeCuda((3,), index=2), "cuda:2"),
    (torch.zeros(3, dtype=torch.float64), "not on a CUDA"),
])
def test_assimilate_device_rejects_wrong_y(y, word):
    assert word in _einval(_filter().assimilate_device, y)


def test_assimilate_rejects_wrong_length():
    assert "shape" in _einval(_filter().assimilate, np.zeros(4))


@pytest.mark.parametrize("out", [
    np.zeros(9), np.zeros(10, dtype=np.float32), np.zeros((10, 2))[:, 0], torch.zeros(10, dtype=torch.float32),
    torch.zeros(11, dtype=torch.float64), FakeCuda((9,)), FakeCuda((10,), torch.float32), FakeCuda((10,), index=1),
])
@pytest.mark.parametrize("method", ["mean_into", "variance_into"])
def test_outputs_reject_wrong_buffers(method, out):
    _einval(getattr(_filter(), method), out)
