"""The allocation-free change-norm entry point (wd_change_norms_noalloc) against the
solver's own change norms, which wd_steps reports after one pseudo step.

Callers that cannot allocate device memory (an application pool that has taken the device
memory, a real-time loop that must not call the allocator) use this entry point; its
scratch is a static device array shared by every call, so two calls in a row must both
give the same norms as the allocating path, and neither may allocate through torch.
Collected last so that a failure here never hides another test."""
import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wd():
    import torch

    assert torch.cuda.is_available()
    from paper_2111_09859_gb300 import build, wd as _wd

    build.build()
    return _wd


def wall_mask(spec):
    x, y = spec.xyz
    return ((x == 0) | (x == 1) | (y == 0) | (y == 1)).astype(np.uint8)


@pytest.mark.parametrize("prec,rtol", [(0, 1e-12), (2, 1e-6)])
def test_noalloc_norms_match_solver_norms_twice(wd, prec, rtol):
    import torch

    spec = W.square(41)
    g = wd.Grid(spec, prec, wd.E4)
    p = wd.default_params(wd.E4, equation=wd.HJ_LAD)
    x, y = spec.xyz
    exact = np.minimum.reduce([x, 1 - x, y, 1 - y])
    noise = 0.01 * W.random_field(spec, 17)
    phi0 = g.apply_bc(g.as_field(exact + noise))
    mask = torch.as_tensor(wall_mask(spec)).cuda()
    out = torch.empty(2, dtype=torch.float64, device="cuda")
    cur = phi0
    for call in range(2):
        after, st = g.steps(p, cur.clone(), 1)          # allocating path: solver's norms
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated()
        wd.change_norms_noalloc(after, cur, mask, scale=spec.L_ref, out=out)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated() == before
        rms, mx = out.cpu().tolist()
        assert rms == pytest.approx(st["res_l2"], rel=rtol, abs=1e-15), (call, rms, st)
        assert mx == pytest.approx(st["res_linf"], rel=rtol, abs=1e-15), (call, mx, st)
        cur = after


def test_noalloc_rejects_oversized_and_bad_input(wd):
    import ctypes
    import torch

    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    L = wd.lib()
    s = L.wd_change_norms_noalloc(ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(a.data_ptr()), None,
                                  (1 << 30) + 1, wd.FP64, 1.0, ctypes.c_void_p(out.data_ptr()), None)
    assert s == wd.ERR_INVALID_ARG
    assert b"maximum size" in L.wd_last_error()
    s = L.wd_change_norms_noalloc(None, ctypes.c_void_p(a.data_ptr()), None, 8, wd.FP64, 1.0,
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert s == wd.ERR_INVALID_ARG


@pytest.mark.gpu
def test_noalloc_wrapper_rejects_mismatched_tensors_on_the_gpu(wd):
    import torch

    a = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        wd.change_norms_noalloc(a, torch.zeros(8, dtype=torch.float32, device="cuda"))
    with pytest.raises(ValueError):
        wd.change_norms_noalloc(a, a.double())
    with pytest.raises(ValueError):
        wd.change_norms_noalloc(a, a, torch.zeros(16, dtype=torch.float32, device="cuda"))
