"""Host-side checks of the allocation-free change-norm wrapper: every mismatch between the
tensors it is given (dtype, length, layout, mask type, output shape, device) is rejected in
Python before the library is called, so a wrong argument can never make the kernel read
past an array."""
import pytest
import torch

from paper_2111_09859_gb300 import wd


@pytest.fixture
def no_library(monkeypatch):
    def refuse(*a, **k):
        raise AssertionError("the library was called")

    monkeypatch.setattr(wd, "lib", refuse)


def f32(n):
    return torch.zeros(n, dtype=torch.float32)


@pytest.mark.parametrize("case", [
    "half", "dtype_mismatch", "length_mismatch", "empty", "mask_float", "mask_short",
    "out_float32", "out_long", "non_contiguous", "cpu_tensors",
])
def test_wrapper_rejects_before_any_call(no_library, case):
    new, old, mask, out = f32(16), f32(16), None, None
    if case == "half":
        new, old = new.half(), old.half()
    elif case == "dtype_mismatch":
        old = old.double()
    elif case == "length_mismatch":
        old = f32(15)
    elif case == "empty":
        new, old = f32(0), f32(0)
    elif case == "mask_float":
        mask = f32(16)
    elif case == "mask_short":
        mask = torch.zeros(8, dtype=torch.uint8)
    elif case == "out_float32":
        out = f32(2)
    elif case == "out_long":
        out = torch.zeros(3, dtype=torch.float64)
    elif case == "non_contiguous":
        new = f32(32)[::2]
    # "cpu_tensors": all checks pass except the device check
    with pytest.raises(ValueError) as ei:
        wd.change_norms_noalloc(new, old, mask, out=out)
    if case == "cpu_tensors":
        assert "CUDA device" in str(ei.value)
    else:
        assert "CUDA device" not in str(ei.value)
