"""Host logic (no GPU): the grid descriptor and arrays the ctypes binding builds from a
GridSpec, the library's footprint query for the workloads' descriptors, and the index
argument behind the level-set stage kernel's folded face conditions."""
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


def _faces_by_copies(V, periodic):
    """Zero-gradient faces as the oracle applies them: direction by direction (0, 1, 2 =
    the last, middle and first numpy axes), each non-periodic face node takes its inner
    neighbour's current value."""
    A = V.copy()
    nd = A.ndim
    for d in range(nd):
        if periodic[d]:
            continue
        ax = nd - 1 - d
        lo = [slice(None)] * nd
        lo1 = [slice(None)] * nd
        lo[ax], lo1[ax] = 0, 1
        A[tuple(lo)] = A[tuple(lo1)]
        hi = [slice(None)] * nd
        hi1 = [slice(None)] * nd
        hi[ax], hi1[ax] = -1, -2
        A[tuple(hi)] = A[tuple(hi1)]
    return A


def _faces_by_clamping(V, periodic):
    """The level-set stage kernel's form: every node takes the value of the node whose
    non-periodic coordinates are clamped to [1, n - 2]."""
    nd = V.ndim
    idx = []
    for ax in range(nd):
        d = nd - 1 - ax
        n = V.shape[ax]
        i = np.arange(n)
        idx.append(i if periodic[d] else np.clip(i, 1, n - 2))
    return V[np.ix_(*idx)]


def test_level_set_faces_fold_into_the_stage():
    """The level-set stage kernel stores at each face node the stage value of its clamped
    interior node instead of running face-copy launches; the two agree for every grid shape,
    corners and edges included."""
    rng = np.random.default_rng(9)
    for shape, periodic in (((9, 8), (False, False)), ((9, 8), (True, False)),
                            ((6, 7, 8), (False, False, False)), ((6, 7, 8), (True, False, False)),
                            ((6, 7, 8), (False, True, False))):
        V = rng.standard_normal(shape)
        np.testing.assert_array_equal(_faces_by_clamping(V, periodic), _faces_by_copies(V, periodic))
