"""Edge cases and full-size checks on the GPU.

- The smallest grids the library accepts (8 nodes per direction) against the oracle.
- A grid whose nodes are all Dirichlet: the solve stops at once with zero change and no
  NaN.
- Invalid descriptors and arguments are errors, not faults.
- Full size:
  - the cylinder configuration (257 x 512, C6 + LAD + curvature, FP64) against the oracle,
    over pseudo steps;
  - the 256^3 duct solve, checked through properties that hold at any size: exact
    x-invariance, and the distance within the discretisation error of the exact one.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W
from tests.helpers import base_params, gpu_params, oracle_grid, oracle_kw, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wd():
    import torch

    assert torch.cuda.is_available()
    from paper_2111_09859_gb300 import build, wd as _wd

    build.build()
    return _wd


def scale(a):
    return max(1.0, float(np.abs(a).max()))


@pytest.mark.parametrize("gname,scheme,prec", [("square8", 1, 0), ("square8", 4, 0), ("duct8", 2, 0),
                                               ("cyl8x8", 4, 0), ("square8", 1, 1)])
def test_smallest_grids_against_oracle(wd, oracle, gname, scheme, prec):
    spec = {"square8": lambda: W.square(8), "duct8": lambda: W.duct(8, nx=8),
            "cyl8x8": lambda: W.cylinder(8, 8, 1.5)}[gname]()
    prm = base_params(scheme, equation=1)
    og = oracle_grid(oracle, spec, scheme)
    g = wd.Grid(spec, prec, scheme)
    phi0 = og.apply_bc(0.5 + 0.1 * W.random_field(spec, 3))
    ref, _ = og.hj_steps(phi0, 3, **oracle_kw(scheme, prm))
    out, _ = g.steps(gpu_params(wd, scheme, prm), g.as_field(phi0), 3, kind=0)
    tol = 1e-10 if prec == 0 else 1e-5
    np.testing.assert_allclose(to_np(out), ref, atol=tol * scale(ref), rtol=0)


def test_all_dirichlet_grid(wd):
    spec = W.square(16)
    spec.mask = np.ones(spec.N, np.uint8)
    spec.dval = np.linspace(-0.1, 0.1, spec.N)
    g = wd.Grid(spec, wd.FP64, wd.E4)
    phi, st = g.solve(wd.default_params(wd.E4, tol_l2=1e-10))
    assert st["converged"] == 1 and st["iters"] == 10 and st["res_l2"] == 0.0
    out = to_np(phi)
    assert np.all(np.isfinite(out))
    inner = np.zeros((16, 16), bool)
    inner[1:-1, 1:-1] = True            # the walls hold 0, every other node its value
    np.testing.assert_array_equal(out[inner.ravel()], spec.dval[inner.ravel()])


def _desc(wd, n, ndim=2):
    d = wd.GridDesc()
    d.ndim = ndim
    for k in range(3):
        d.n[k] = n[k]
        d.bc_lo[k] = d.bc_hi[k] = wd.BC_WALL
    d.precision = wd.FP32
    d.scheme = wd.E4
    d.L_ref = 1.0
    return d


@pytest.mark.parametrize("n,ndim", [((7, 16, 1), 2), ((16, 2049, 1), 2), ((16, 16, 0), 2), ((16, 16, 4), 3),
                                    ((2048, 2048, 600), 3)])
def test_invalid_descriptors_are_errors(wd, n, ndim):
    lib = wd.lib()
    d = _desc(wd, n, ndim)
    xyz = np.zeros(3 * max(1, n[0] * n[1] * max(1, n[2])) if n[0] * n[1] * max(1, n[2]) < 1e7 else 3)
    h = C.c_void_p()
    s = lib.wd_create_grid(C.byref(d), xyz.ctypes.data, None, None, None, C.byref(h))
    assert s == wd.ERR_INVALID_ARG and not h.value
    assert lib.wd_query_footprint(C.byref(d), None) == 0


def test_invalid_calls_are_errors(wd):
    import torch

    lib = wd.lib()
    sp = W.square(16)
    g = wd.Grid(sp, wd.FP64, wd.E4)
    p = wd.default_params(wd.E4)
    st = wd.Stats()
    assert lib.wd_solve(g._h, C.byref(p), None, C.byref(st)) == wd.ERR_INVALID_ARG
    bad = wd.default_params(wd.E4, alpha_f=0.6)
    phi = g.empty()
    assert lib.wd_solve(g._h, C.byref(bad), C.c_void_p(phi.data_ptr()), C.byref(st)) == wd.ERR_INVALID_ARG
    assert lib.wd_derivative(g._h, 5, C.c_void_p(phi.data_ptr()), C.c_void_p(phi.data_ptr())) == wd.ERR_INVALID_ARG
    assert lib.wd_recede(g._h, C.c_void_p(phi.data_ptr()), -1.0, -0.1, None, None) == wd.ERR_INVALID_ARG
    out = C.c_double()
    g3 = wd.Grid(W.duct(8, nx=8), wd.FP64, wd.E4)
    assert lib.wd_level_length(g3._h, C.c_void_p(g3.empty().data_ptr()), 0.0, C.byref(out)) == wd.ERR_INVALID_ARG
    torch.cuda.synchronize()
    # the grid is still usable after the errors
    _, st2 = g.solve(p)
    assert st2["converged"] == 1


def test_cylinder_full_size_steps_against_oracle(wd, oracle):
    """The cylinder configuration at its full size, FP64: four HJ pseudo steps (C6 + LAD +
    curvature, alpha_f 0.495) from a perturbed exact field, and ten Poisson steps."""
    spec = W.cylinder(257, 512, 1.03)
    prm = base_params(4, equation=1, curvature=1, alpha_f=0.495)
    og = oracle_grid(oracle, spec, 4)
    g = wd.Grid(spec, wd.FP64, wd.C6)
    r = np.hypot(*spec.xyz) - 0.5
    phi0 = og.apply_bc(r + 0.01 * np.minimum(r, 1.0) * W.random_field(spec, 11))
    ref, ost = og.hj_steps(phi0, 4, **oracle_kw(4, prm))
    out, st = g.steps(gpu_params(wd, 4, prm), g.as_field(phi0), 4, kind=0)
    np.testing.assert_allclose(to_np(out), ref, atol=1e-10 * scale(ref), rtol=0)
    assert abs(st["res_l2"] - ost["res_l2"]) <= 1e-8 * ost["res_l2"]
    refp, _ = og.poisson_steps(np.zeros(spec.N), 10, **oracle_kw(4, prm))
    outp, _ = g.steps(gpu_params(wd, 4, prm), g.as_field(np.zeros(spec.N)), 10, kind=1)
    np.testing.assert_allclose(to_np(outp), refp, atol=1e-10 * scale(refp), rtol=0)


def test_duct_full_size_properties(wd):
    """256^3 duct, E6 + LAD, FP32 solve: the field is exactly independent of x (periodic
    direction, x-independent data), and within 1.5 h of min(y, 1-y, z, 1-z) everywhere (the
    LAD-smoothed kinks on the duct's diagonal planes), 0.1 h in RMS."""
    import torch

    spec = W.duct(256)
    g = wd.Grid(spec, wd.FP32_METRIC64, wd.E6)
    p = wd.default_params(wd.E6, equation=wd.HJ_LAD, tol_l2=1e-6, max_iters=5000)
    phi, st = g.solve(p)
    torch.cuda.synchronize()
    assert st["converged"] == 1
    P = phi.view(256, 256, 256)
    assert float((P - P[:, :, :1]).abs().max()) == 0.0
    x, y, z = spec.xyz
    ex = np.minimum.reduce([y, 1 - y, z, 1 - z])
    err = np.abs(phi.double().cpu().numpy() - ex)
    h = 1.0 / 255
    assert err.max() <= 1.5 * h and np.sqrt((err ** 2).mean()) <= 0.1 * h
    g.close()

