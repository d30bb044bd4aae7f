"""Pins of the oracle's baseline upwind scheme (Sec. 3.2.1, Eqs. UW1-UW5) and of its
level-set march (Sec. 5.5), against closed forms that do not come from the oracle:

- the upwind slope squared is Godunov's numerical Hamiltonian of |grad phi| for a front
  moving towards increasing phi, max(B+, F-)^2 (Rouy & Tourin; Osher & Sethian);
- on an affine (sheared) grid a linear phi has B = F = grad(phi) . dx/dxi_l exactly, so the
  advection term equals |grad phi|^2 and the level-set |grad phi| equals |a|;
- in a channel the converged upwind Eikonal solution is the exact distance at the nodes;
  on the square its error falls at first order;
- a planar front moves at speed F exactly, outside the inflow boundary's domain of
  influence; an expanding circle's perimeter tends to 2 pi (a + F t) at first order, and
  F < 0 shrinks it.
"""
import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W
from tests.helpers import base_params, oracle_grid, oracle_kw

def test_upwind_slope_is_godunov(oracle):
    rng = np.random.default_rng(5)
    vals = np.concatenate([rng.normal(size=400), [0.0, -0.0, 1.0, -1.0, 0.5, -0.5]])
    for B in vals[::7]:
        for F in vals:
            s = oracle.upwind_slope(B, F)
            god = max(max(B, 0.0), max(-F, 0.0))
            assert s * s == god * god, (B, F, s)
            assert s in (B, F, 0.0)


def _affine_grid(oracle, n, shear, scheme):
    i, j = np.meshgrid(np.arange(n), np.arange(n))
    x = (i + shear * j) / (n - 1)
    y = (0.4 * i + j) / (n - 1)
    return oracle.Grid((n, n), np.stack([x.ravel(), y.ravel()]), (oracle.BC_FARFIELD,) * 2,
                       (oracle.BC_FARFIELD,) * 2, scheme=scheme), x.ravel(), y.ravel()


@pytest.mark.parametrize("a", [(0.7, 0.2), (-0.3, 0.9), (0.5, -0.8), (-0.6, -0.4)])
def test_advection_of_linear_field_on_sheared_grid(oracle, a):
    n = 12
    og, x, y = _affine_grid(oracle, n, 0.3, oracle.UW)
    phi = a[0] * x + a[1] * y + 0.1
    adv = og.upwind_advection(phi)
    inner = np.zeros((n, n), bool)
    inner[1:-1, 1:-1] = True
    np.testing.assert_allclose(adv[inner.ravel()], a[0] ** 2 + a[1] ** 2, rtol=1e-12)
    for F in (0.3, -0.3):
        gm = og.levelset_gradmag(phi, F)
        np.testing.assert_allclose(gm[inner.ravel()], np.hypot(*a), rtol=1e-12)


def test_upwind_terms_of_a_linear_field_on_an_affine_3d_grid(oracle):
    """3-D affine map x = M (i, j, k) + c: every one-sided difference of a linear field is
    exact, so the advection term is |a|^2 and the level-set |grad phi| is |a| at the interior
    nodes, for fronts along any direction (all nine metric terms enter)."""
    M = np.array([[0.9, 0.2, -0.1], [0.05, 1.1, 0.3], [0.15, -0.2, 0.8]]) * 0.1
    n = (9, 10, 11)
    K, J, I = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = np.stack([I.reshape(-1), J.reshape(-1), K.reshape(-1)]).astype(float)
    xyz = M @ idx + np.array([[0.3], [-0.2], [1.0]])
    g = oracle.Grid(n, xyz, (oracle.BC_FARFIELD,) * 3, (oracle.BC_FARFIELD,) * 3, scheme=oracle.UW)
    inner = ((I > 0) & (I < n[0] - 1) & (J > 0) & (J < n[1] - 1) & (K > 0) & (K < n[2] - 1)).reshape(-1)
    for a in ((0.6, 0.3, -0.5), (-0.2, -0.7, 0.4)):
        phi = np.asarray(a) @ xyz + 0.2
        adv = g.upwind_advection(phi)
        np.testing.assert_allclose(adv[inner], np.dot(a, a), rtol=1e-11)
        for F in (0.3, -0.3):
            np.testing.assert_allclose(g.levelset_gradmag(phi, F)[inner], np.linalg.norm(a), rtol=1e-11)


def test_advection_of_monotone_field_is_first_order_upwind(oracle):
    """Uniform Cartesian grid, phi increasing along both directions: the term is
    sum_l (B_l / h_l)^2 with the backward differences; decreasing: the forward ones."""
    nx, ny = 14, 11
    hx, hy = 1.0 / (nx - 1), 0.5 / (ny - 1)
    X, Y = np.meshgrid(np.arange(nx) * hx, np.arange(ny) * hy)
    og = oracle.Grid((nx, ny), np.stack([X.ravel(), Y.ravel()]), (oracle.BC_WALL,) * 2,
                     (oracle.BC_WALL,) * 2, scheme=oracle.UW)
    rng = np.random.default_rng(2)
    for sgn in (1.0, -1.0):
        phi = sgn * np.cumsum(np.cumsum(rng.uniform(0.1, 1.0, (ny, nx)), 0), 1) * hx * hy
        adv = og.upwind_advection(phi.ravel()).reshape(ny, nx)
        if sgn > 0:
            d0 = (phi[1:-1, 1:-1] - phi[1:-1, :-2]) / hx
            d1 = (phi[1:-1, 1:-1] - phi[:-2, 1:-1]) / hy
        else:
            d0 = (phi[1:-1, 2:] - phi[1:-1, 1:-1]) / hx
            d1 = (phi[2:, 1:-1] - phi[1:-1, 1:-1]) / hy
        np.testing.assert_allclose(adv[1:-1, 1:-1], d0 ** 2 + d1 ** 2, rtol=1e-12)


def test_uw_eikonal_channel_is_exact(oracle):
    sp = W.channel(16, 33)
    og = oracle_grid(oracle, sp, oracle.UW)
    prm = base_params(oracle.UW, equation=2, filter=0, tol_l2=1e-13)
    phi, st = og.solve(**oracle_kw(oracle.UW, prm))
    assert st["converged"]
    y = sp.xyz[1]
    np.testing.assert_allclose(phi, np.minimum(y, 1.0 - y), atol=1e-12, rtol=0)


def test_uw_eikonal_square_first_order(oracle):
    errs = []
    for n in (33, 65):
        sp = W.square(n)
        x, y = sp.xyz
        og = oracle_grid(oracle, sp, oracle.UW)
        prm = base_params(oracle.UW, equation=2, filter=0, tol_l2=1e-11)
        phi, st = og.solve(**oracle_kw(oracle.UW, prm))
        assert st["converged"]
        err = np.abs(phi - np.minimum.reduce([x, 1 - x, y, 1 - y])).max()
        assert err < 0.75 / (n - 1)
        errs.append(err)
    assert 1.7 < errs[0] / errs[1] < 2.3


def test_uw_hj_with_zero_eps_is_the_eikonal(oracle):
    sp = W.square(17)
    og = oracle_grid(oracle, sp, oracle.UW)
    phi0 = og.apply_bc(0.3 + 0.05 * W.random_field(sp, 4))
    a, _ = og.hj_steps(phi0, 5, **oracle_kw(oracle.UW, base_params(oracle.UW, equation=0, eps=0.0, filter=0)))
    b, _ = og.hj_steps(phi0, 5, **oracle_kw(oracle.UW, base_params(oracle.UW, equation=2, filter=0)))
    np.testing.assert_array_equal(a, b)


def _box(oracle, n, lo, hi):
    xs = np.linspace(lo, hi, n)
    X, Y = np.meshgrid(xs, xs)
    og = oracle.Grid((n, n), np.stack([X.ravel(), Y.ravel()]), (oracle.BC_NEUMANN,) * 2,
                     (oracle.BC_NEUMANN,) * 2, scheme=oracle.E2)
    return og, X.ravel(), Y.ravel(), (hi - lo) / (n - 1)


def test_levelset_planar_front_speed(oracle):
    n, F, T = 65, 0.3, 0.5
    og, X, Y, h = _box(oracle, n, 0.0, 1.0)
    p0 = Y - 0.3
    ns = int(np.ceil(T / (0.5 * h / F)))
    p = og.levelset_steps(p0, F, T / ns, ns)
    far = (Y >= F * T + 0.5) & (Y < 1.0 - 0.5 * h)     # beyond the inflow disturbance
    np.testing.assert_allclose(p[far], (p0 - F * T)[far], atol=1e-13, rtol=0)
    # the last row holds its neighbour's value (zero normal gradient)
    top = Y > 1.0 - 0.5 * h
    np.testing.assert_array_equal(p[top], p[np.nonzero(top)[0] - n])


def test_levelset_circle_perimeter_first_order(oracle):
    a, F, T = 0.3, 0.3, 1.0
    errs = []
    for n in (65, 129):
        og, X, Y, h = _box(oracle, n, -1.0, 1.0)
        ns = int(np.ceil(T / (0.5 * h / F)))
        p = og.levelset_steps(np.hypot(X, Y) - a, F, T / ns, ns)
        L = oracle.level_length(X, Y, p, (n, n), 0.0)
        errs.append(abs(L / (2 * np.pi * (a + F * T)) - 1.0))
    assert errs[0] < 0.012 and 1.6 < errs[0] / errs[1] < 2.4


def test_levelset_negative_speed_shrinks(oracle):
    a, F, T, n = 0.6, -0.3, 1.0, 129
    og, X, Y, h = _box(oracle, n, -1.0, 1.0)
    ns = int(np.ceil(T / (0.5 * h / abs(F))))
    p = og.levelset_steps(np.hypot(X, Y) - a, F, T / ns, ns)
    L = oracle.level_length(X, Y, p, (n, n), 0.0)
    assert abs(L / (2 * np.pi * (a + F * T)) - 1.0) < 0.01
