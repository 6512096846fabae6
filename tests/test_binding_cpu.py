"""Argument checks of the Python binding that need no GPU: tensors on the
wrong side of the host/device boundary and float tensors of mismatched shape
are refused before anything reaches the library."""
import pytest
import torch

from paper_1702_00817_gb300 import codec as C


def test_device_calls_refuse_host_tensors():
    src = torch.zeros((16, 16), dtype=torch.uint8)
    coef = torch.zeros((1, 2, 2, 8, 8), dtype=torch.int16)
    with pytest.raises(ValueError, match="CUDA tensor"):
        C.image_array([C.Image(src, None, coef)], None, 0)
    with pytest.raises(ValueError, match="CUDA tensor"):
        C._f32(torch.zeros((1, 8, 8)), "x", 0)


def test_host_pipeline_takes_host_tensors_and_unchecked_arrays_stay_open():
    src = torch.zeros((16, 16), dtype=torch.uint8)
    arr = C.image_array([C.Image(src, torch.zeros_like(src), None)], None, "cpu")
    assert arr[0].width == 16 and arr[0].height == 16
    arr = C.image_array([C.Image(src)])  # no placement check requested
    assert arr[0].channels == 1


def test_float_shapes_must_match_x():
    x = torch.zeros((2, 8, 16))
    with pytest.raises(ValueError, match="shape of x"):
        C._f32(torch.zeros((1, 8, 16)), "gy", None, x)
    assert C._f32(torch.zeros((2, 8, 16)), "gy", None, x) == (2, 8, 16)
