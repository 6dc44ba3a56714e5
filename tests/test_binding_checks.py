"""Argument checks of the Python binding, which run before any library call:
a state, cotangent or field pointer handed to a kernel must be contiguous
memory of the lattice's GPU with the right dtype and shape (a host pointer
would otherwise be dereferenced on the device).  The helper is device-agnostic,
so its accept and reject paths are checked here on CPU tensors."""
import pytest

torch = pytest.importorskip("torch")

from paper_1703_00186_gb300.lbm import _check_tensor  # noqa: E402

SHAPE = (37, 10, 8)
CPU = torch.device("cpu")


def test_matching_tensor_is_accepted():
    t = torch.zeros(SHAPE, dtype=torch.float64)
    assert _check_tensor(t, "f", torch.float64, SHAPE, CPU) is t


def test_host_tensor_is_refused_for_a_gpu_lattice():
    t = torch.zeros(SHAPE, dtype=torch.float64)
    with pytest.raises(ValueError, match="lives on cuda:0"):
        _check_tensor(t, "f", torch.float64, SHAPE, torch.device("cuda", 0))


@pytest.mark.parametrize("bad,match", [
    (lambda: torch.zeros(SHAPE, dtype=torch.float32), "dtype"),
    (lambda: torch.zeros((37, 10, 9), dtype=torch.float64), "shape"),
    (lambda: torch.zeros((37, 8, 10), dtype=torch.float64).transpose(1, 2), "contiguous"),
])
def test_wrong_dtype_shape_or_layout_is_refused(bad, match):
    with pytest.raises(ValueError, match=match):
        _check_tensor(bad(), "f", torch.float64, SHAPE, CPU)


def test_non_tensor_is_refused():
    import numpy as np
    with pytest.raises(TypeError):
        _check_tensor(np.zeros(SHAPE), "f", torch.float64, SHAPE, CPU)
