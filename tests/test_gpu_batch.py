"""wd_solve_batch through the C ABI: grids of different shapes solved side by side give bit for
bit what wd_solve gives each alone, and match the FP64 oracle at the FP32 bar (2e-4 L)."""
import ctypes as C

import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W
from tests.helpers import base_params, oracle_grid, oracle_kw, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wd():
    import torch

    assert torch.cuda.is_available()
    from paper_2111_09859_gb300 import build, wd as _wd

    build.build()
    return _wd


def _specs():
    return [W.ellipse(65, 128, 2.2),
            W.ellipse(129, 256, 1.4),
            W.cylinder(65, 128, 1.03 ** 4, r_wall=0.5),
            W.stack([W.cylinder(65, 128, 1.03 ** 4, r_wall=r) for r in (0.45, 0.6)])]


def test_batch_matches_single_solves_and_oracle(wd, oracle):
    import torch

    specs = _specs()
    prm = base_params(4, equation=1, tol_l2=1e-6)
    p = wd.default_params(wd.C6, equation=wd.HJ_LAD, tol_l2=1e-6)
    grids = [wd.Grid(sp, wd.FP32_METRIC64, wd.C6) for sp in specs]
    outs, stats, s = wd.solve_batch(grids, p)
    torch.cuda.synchronize()
    assert s == wd.OK, (s, stats)
    for g, sp, o, st in zip(grids, specs, outs, stats):
        assert st["converged"] and st["iters"] > 0
        alone = wd.Grid(sp, wd.FP32_METRIC64, wd.C6)
        ref, st1 = alone.solve(p)
        np.testing.assert_array_equal(to_np(o), to_np(ref))
        assert (st1["iters"], st1["poisson_iters"], st1["res_l2"]) == (st["iters"], st["poisson_iters"], st["res_l2"])
        alone.close()
    for k in (0, 2):   # the two smallest single grids against the FP64 oracle
        ref, ost = oracle_grid(oracle, specs[k], 4).solve(**oracle_kw(4, dict(prm, tol_l2=1e-12)))
        assert ost["converged"]
        assert float(np.abs(to_np(outs[k]) - ref).max()) <= 2e-4 * specs[k].L_ref
    for g in grids:
        g.close()


def test_batch_rejects_bad_input(wd):
    import torch

    sp = W.cylinder(65, 128, 1.03 ** 4)
    g = wd.Grid(sp, wd.FP32_METRIC64, wd.C6)
    phi = g.empty()
    p = wd.default_params(wd.C6)
    L = wd.lib()
    harr = (C.c_void_p * 2)(g._h, g._h)
    parr = (C.c_void_p * 2)(phi.data_ptr(), phi.data_ptr())
    st = (wd.Stats * 2)()
    assert L.wd_solve_batch(harr, 2, C.byref(p), parr, st) == wd.ERR_INVALID_ARG   # the same grid twice
    assert L.wd_solve_batch(harr, -1, C.byref(p), parr, st) == wd.ERR_INVALID_ARG
    assert L.wd_solve_batch(None, 1, C.byref(p), parr, st) == wd.ERR_INVALID_ARG
    assert L.wd_solve_batch(harr, 0, C.byref(p), parr, st) == wd.OK                 # empty batch
    torch.cuda.synchronize()
    g.close()
