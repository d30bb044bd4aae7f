"""Host logic of the ctypes binding (no GPU): the grid descriptor and arrays built from a
GridSpec, and the library's footprint query for the descriptors the workloads produce."""
import ctypes as C

import numpy as np

from paper_2111_09859_gb300 import wd, workloads as W


def test_descriptor_of_an_ogrid():
    sp = W.cylinder(33, 64, 1.1)
    d, xyz, mask, dval, n = wd._grid_inputs(sp, wd.FP32_METRIC64, wd.C6)
    assert d.ndim == 2 and list(d.n) == [64, 33, 1] and n == [64, 33, 1]
    assert (d.bc_lo[0], d.bc_hi[0]) == (wd.BC_PERIODIC, wd.BC_PERIODIC)
    assert (d.bc_lo[1], d.bc_hi[1]) == (wd.BC_WALL, wd.BC_FARFIELD)
    assert (d.bc_lo[2], d.bc_hi[2]) == (wd.BC_WALL, wd.BC_WALL)   # unused third direction
    assert d.precision == wd.FP32_METRIC64 and d.scheme == wd.C6 and d.L_ref == sp.L_ref
    assert xyz.shape == (2, sp.N) and xyz.dtype == np.float64 and xyz.flags.c_contiguous
    assert mask is None and dval is None


def test_descriptor_of_a_stack_and_of_the_star():
    members = [W.cylinder(33, 64, 1.1, r_wall=r) for r in (0.5, 0.4, 0.6)]
    d, xyz, _, _, n = wd._grid_inputs(W.stack(members), wd.FP64, wd.E4)
    assert list(d.n) == [64, 33, 3] and xyz.shape == (2, 3 * 64 * 33)
    np.testing.assert_array_equal(xyz[:, 64 * 33:2 * 64 * 33], members[1].xyz)
    star = W.star(65)
    d, xyz, mask, dval, n = wd._grid_inputs(star, wd.FP32, wd.UW)
    assert d.scheme == wd.UW and all(d.bc_lo[k] == wd.BC_NEUMANN for k in range(2))
    assert mask.dtype == np.uint8 and mask.shape == (star.N,) and mask.any()
    assert dval.dtype == np.float64 and np.all(dval[mask == 1] <= 0.0)


def test_footprint_of_the_workloads():
    """The footprint grows with the nodes and the state precision; a stack of k grids holds
    k times the per-node arrays of one."""
    L = wd.lib()

    def fp(spec, prec, sch):
        d, *_ = wd._grid_inputs(spec, prec, sch)
        return L.wd_query_footprint(C.byref(d), None)

    one = W.cylinder(65, 128, 1.1)
    a64, a32 = fp(one, wd.FP64, wd.C6), fp(one, wd.FP32_METRIC64, wd.C6)
    assert a64 > a32 > 0
    three = fp(W.stack([one, one, one]), wd.FP32_METRIC64, wd.C6)
    assert 2.5 * a32 < three < 3.0 * a32 + (1 << 20)
    assert fp(W.duct(16, nx=8), wd.FP32_METRIC64, wd.E6) > 0
