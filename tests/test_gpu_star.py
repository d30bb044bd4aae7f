"""Unsteady star grain on the GPU (Sec. 5.5): the receding-surface update and the
level-set length against the oracle's, and the receding chain (initial solve, then warm
re-solves after each recession) against the oracle's chain, in FP64 directly and in FP32
through the request loop on caller-owned grids."""
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


def gpu_star_params(wd, **kw):
    base = dict(equation=wd.HJ_LAD, eps=0.15, alpha_f=0.49, cfl=0.8, tol_l2=1e-10, lad_exp=4.0,
                max_iters=20000, poisson_max_iters=100, check_every=10)
    base.update(kw)
    return wd.default_params(wd.E4, **base)


def oracle_star_params(**kw):
    p = dict(scheme=1, equation=1, eps=0.15, alpha_f=0.49, cfl=0.8, tol_l2=1e-10,
             max_iters=20000, poisson_max_iters=100, check_every=10, init=1, C_lad=0.1,
             lad_exp=4.0, filter=1, curvature=0, eps0=1e-8)
    p.update(kw)
    return p


@pytest.mark.parametrize("prec", [0, 1])
def test_recede_matches_oracle(wd, oracle, prec):
    sp = W.star(129)
    g = wd.Grid(sp, prec, wd.E4)
    phi = sp.meta["signed_distance"] + 0.004 * W.random_field(sp, 3)
    t = g.as_field(phi)
    ph = to_np(t)                            # the field as the GPU holds it
    m, d = g.recede(t, 0.002, -3 * sp.meta["h"])
    onew, om, od = oracle.recede(ph, 0.002, -3 * sp.meta["h"])
    tol = 0.0 if prec == 0 else 1e-7
    np.testing.assert_allclose(to_np(t), onew, atol=tol, rtol=0)
    # the mask is decided on the shifted value in the grid's own precision
    np.testing.assert_array_equal(m.cpu().numpy(), (to_np(t) <= 0).astype(np.uint8))
    if prec == 0:
        np.testing.assert_array_equal(m.cpu().numpy(), om)
    np.testing.assert_allclose(to_np(d), np.where(m.cpu().numpy() == 1, np.maximum(to_np(t), -3 * sp.meta["h"]), 0.0),
                               atol=0, rtol=0)
    np.testing.assert_allclose(to_np(d), od, atol=tol, rtol=0)


def test_level_length_matches_oracle(wd, oracle):
    for sp in (W.star(257), W.cylinder(65, 128, 1.1)):
        g = wd.Grid(sp, wd.FP64, wd.E4)
        if sp.name == "star":
            phi = sp.meta["signed_distance"]
            levels = (0.0, 0.01, 0.02)
        else:
            phi = np.hypot(*sp.xyz) - 0.5
            levels = (0.25, 1.0, 3.0)
        for lv in levels:
            L = g.level_length(g.as_field(phi), lv)
            per = tuple(b == W.PERIODIC for b in sp.bc_lo)
            Lo = oracle.level_length(sp.xyz[0], sp.xyz[1], phi, sp.shape, lv, per, sp.period)
            assert abs(L - Lo) <= 1e-12 * Lo
        if sp.name == "cylinder":
            # circle r = 1.5 through 128 rays: the 128 chords of the inscribed polygon
            chords = 2 * 128 * 1.5 * np.sin(np.pi / 128)
            assert abs(g.level_length(g.as_field(phi), 1.0) - chords) < 1e-12


def test_star_chain_fp64_matches_oracle(wd, oracle):
    sp = W.star(129)
    h = sp.meta["h"]
    og = oracle.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=1, mask=sp.mask, dval=sp.dval)
    g = wd.Grid(sp, wd.FP64, wd.E4)
    ophi, _ = og.solve(**oracle_star_params())
    phi, st = g.solve(gpu_star_params(wd))
    assert st["converged"]
    np.testing.assert_allclose(to_np(phi), ophi, atol=1e-6, rtol=0)
    s = 0.01
    for k in range(2):
        ophi, om, od = oracle.recede(ophi, s, -3 * h)
        og.set_dirichlet(om, od)
        ophi, _ = og.solve(phi=ophi, **oracle_star_params(init=2))
        m, d = g.recede(phi, s, -3 * h)
        phi, st = g.step_unsteady(gpu_star_params(wd), phi, m, d)
        assert st["converged"] and st["poisson_iters"] == 0
        np.testing.assert_allclose(to_np(phi), ophi, atol=1e-6, rtol=0)


def test_star_chain_fp32_through_server_matches_oracle_chain(wd, oracle):
    """FP32 chain on a session grid served by the request loop, with the benchmark's filter
    coefficient (alpha_f 0.45), against the FP64 oracle's chain on the same grid (2e-4 L per
    step), and the perimeter of each step's zero level against the fillet offset's closed
    form P0 + 2 pi s."""
    import torch

    sp = W.star(257)
    h = sp.meta["h"]
    og = oracle.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=1, mask=sp.mask, dval=sp.dval)
    ophi, ost = og.solve(**oracle_star_params(alpha_f=0.45))
    assert ost["converged"]
    g32 = wd.Grid(sp, wd.FP32_METRIC64, wd.E4)
    p32 = gpu_star_params(wd, tol_l2=1e-7, alpha_f=0.45)
    srv = wd.Server()
    try:
        phi32 = g32.empty()
        t = srv.submit_grid(g32, p32, phi32)
        s_, st, _ = srv.wait(t, 300)
        assert st["converged"]
        torch.cuda.synchronize()
        err = [float(np.abs(to_np(phi32) - ophi).max())]
        assert err[0] <= 2e-4
        s = 0.002
        P0 = sp.meta["geom"]["perimeter"]
        for k in range(1, 4):
            ophi, om, od = oracle.recede(ophi, s, -3 * h)
            og.set_dirichlet(om, od)
            ophi, ost = og.solve(phi=ophi, **oracle_star_params(init=2, alpha_f=0.45))
            assert ost["converged"]
            m32, d32 = g32.recede(phi32, s, -3 * h)
            t = srv.submit_grid(g32, p32, phi32, warm=True, mask=m32, dval=d32)
            s_, st, lat = srv.wait(t, 300)
            assert st["converged"] and st["poisson_iters"] == 0
            torch.cuda.synchronize()
            err.append(float(np.abs(to_np(phi32) - ophi).max()))
            assert err[-1] <= 2e-4, err
            L = g32.level_length(phi32, 0.0)
            assert abs(L - (P0 + 2 * np.pi * k * s)) <= 1e-2
        print("FP32 star chain: max |d - d_oracle| per step:", ["%.2e" % e for e in err])
    finally:
        srv.close()
