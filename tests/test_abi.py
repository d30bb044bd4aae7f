"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every function
that include/wd.h declares; the Python binding declares exactly those functions.  Only
host-only entry points are called here (no device work without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "wd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wd_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libwd():
    from paper_2111_09859_gb300 import build, wd

    build.build()
    return wd


def test_every_declared_symbol_is_exported(libwd):
    import ctypes

    L = ctypes.CDLL(libwd.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 17
    for n in names:
        assert hasattr(L, n), n


def test_binding_mirrors_header(libwd):
    assert sorted(libwd.SIGNATURES) == declared_functions()


def test_host_only_entry_points(libwd):
    import ctypes

    L = libwd.lib()
    assert L.wd_status_string(0) == b"ok"
    assert L.wd_status_string(5) == b"diverged"
    p = libwd.default_params(libwd.C6)
    assert p.equation == libwd.HJ_LAD and abs(p.cfl - 0.6) < 1e-15 and p.filter == 1
    p = libwd.default_params(libwd.E4)
    assert abs(p.cfl - 0.8) < 1e-15 and abs(p.alpha_f - 0.49) < 1e-15
    from paper_2111_09859_gb300 import workloads as W

    b64 = libwd.footprint(W.cylinder(), libwd.FP64, libwd.C6)
    b32 = libwd.footprint(W.cylinder(), libwd.FP32, libwd.C6)
    assert b64 > b32 > 512 * 257 * 4 * 10
    # the baseline upwind scheme holds one more state-size field (its advection term)
    assert libwd.footprint(W.cylinder(), libwd.FP64, libwd.UW) - b64 == 512 * 257 * 8
    d = libwd.GridDesc()
    d.ndim = 2
    d.n[0], d.n[1], d.n[2] = 4, 16, 1      # too few nodes: rejected, footprint 0
    d.L_ref = 1.0
    assert L.wd_query_footprint(ctypes.byref(d), None) == 0
