"""Failure reports of a solve, with the faults made on the host: a NaN planted in the initial
field must end the solve with WD_ERR_DIVERGED and stats.diverged; a tolerance that max_iters
cannot reach must end it with WD_ERR_NOT_CONVERGED after exactly max_iters pseudo steps; and
the grid must solve normally afterwards.  No kernel is made to fault or wait.  Collected last
so that a failure here never hides another test."""
import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W
from tests.helpers import to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wd():
    import torch

    assert torch.cuda.is_available()
    from paper_2111_09859_gb300 import build, wd as _wd

    build.build()
    return _wd


@pytest.mark.parametrize("prec", [0, 1])
def test_divergence_and_non_convergence_are_reported(wd, prec):
    spec = W.square(17)
    g = wd.Grid(spec, prec, wd.E4)
    phi = g.as_field(np.full(spec.N, 0.3))
    phi[5 * 17 + 8] = float("nan")                       # an interior node
    p = wd.default_params(wd.E4, init=wd.INIT_GIVEN, tol_l2=1e-10)
    _, st = g.solve(p, phi, allow_fail=True)
    assert st["status"] == wd.ERR_DIVERGED and st["diverged"] == 1 and st["converged"] == 0

    p = wd.default_params(wd.E4, tol_l2=1e-14, max_iters=20)
    _, st = g.solve(p, allow_fail=True)
    assert st["status"] == wd.ERR_NOT_CONVERGED and st["converged"] == 0 and st["iters"] == 20
    assert st["diverged"] == 0 and np.isfinite(st["res_l2"])

    p = wd.default_params(wd.E4, tol_l2=1e-10 if prec == 0 else 1e-6)
    out, st = g.solve(p)
    assert st["status"] == wd.OK and st["converged"] == 1
    assert np.all(np.isfinite(to_np(out)))
