"""Whole-solve pins of the oracle: closed-form distances (flat plate, channel, square,
circle), brute-force nearest-wall distances, symmetry and x-invariance, independence from
the initial guess, |grad d| = 1 away from the medial axis, and the paper's qualitative
claims (tests/golden/paper_claims.json) on the synthetic channel."""
import json
import os

import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")))


def grid_of(O, sp, scheme):
    return O.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=scheme, period=sp.period,
                  mask=sp.mask, dval=sp.dval)


def brute_force_box(x, y, nwall=4001):
    """Nearest distance to densely sampled points on the four sides of the unit square."""
    s = np.linspace(0.0, 1.0, nwall)
    z = np.zeros_like(s)
    o = np.ones_like(s)
    wx = np.concatenate([s, s, z, o])
    wy = np.concatenate([z, o, s, s])
    d = np.full(x.shape, np.inf)
    for k in range(0, len(wx), 1000):
        d = np.minimum(d, np.sqrt((x[:, None] - wx[None, k:k + 1000]) ** 2
                                  + (y[:, None] - wy[None, k:k + 1000]) ** 2).min(1))
    return d


@pytest.mark.parametrize("scheme", [1, 4])
def test_plate_solve_reaches_exact_linear_distance(oracle, scheme):
    sp = W.plate(8, 33, height=2.0)
    g = grid_of(oracle, sp, scheme)
    phi, st = g.solve(equation=1, scheme=scheme, cfl=0.8 if scheme < 3 else 0.6,
                      tol_l2=1e-12, max_iters=20000, poisson_max_iters=100, poisson_tol=0)
    assert st["converged"]
    np.testing.assert_allclose(phi, sp.xyz[1], atol=1e-9)


def test_square_against_brute_force_and_symmetry(oracle):
    sp = W.square(33)
    g = grid_of(oracle, sp, 1)
    phi, st = g.solve(equation=1, tol_l2=1e-12, max_iters=20000)
    assert st["converged"]
    x, y = sp.xyz
    bf = brute_force_box(x, y)
    np.testing.assert_allclose(bf, np.minimum.reduce([x, 1 - x, y, 1 - y]), atol=1e-12)
    e = phi - bf
    assert np.abs(e).max() < 0.05 and np.sqrt((e ** 2).mean()) < 5e-3
    P = phi.reshape(33, 33)
    # symmetric stencils on a symmetric problem: the D4 symmetry holds to round-off
    np.testing.assert_allclose(P, P.T, atol=1e-10)
    np.testing.assert_allclose(P, P[::-1, :], atol=1e-10)
    np.testing.assert_allclose(P, P[:, ::-1], atol=1e-10)


def test_square_refinement_lad_error_decreases(oracle):
    rms = []
    for n in (17, 33, 65):
        sp = W.square(n)
        g = grid_of(oracle, sp, 1)
        phi, st = g.solve(equation=1, tol_l2=1e-11, max_iters=20000)
        assert st["converged"]
        x, y = sp.xyz
        rms.append(np.sqrt(((phi - np.minimum.reduce([x, 1 - x, y, 1 - y])) ** 2).mean()))
    assert rms[1] < 0.7 * rms[0] and rms[2] < 0.7 * rms[1], rms


def test_initial_guess_independence(oracle):
    """The converged discrete state does not depend on the initial guess (zero, Poisson
    or exact plus noise)."""
    sp = W.square(25)
    g = grid_of(oracle, sp, 1)
    x, y = sp.xyz
    kw = dict(equation=1, tol_l2=1e-13, max_iters=40000)
    a, _ = g.solve(init=0, **kw)
    b, _ = g.solve(init=1, poisson_max_iters=300, poisson_tol=0, **kw)
    noisy = np.minimum.reduce([x, 1 - x, y, 1 - y]) + 0.01 * np.random.default_rng(7).standard_normal(sp.N)
    c, _ = g.solve(noisy, init=2, **kw)
    np.testing.assert_allclose(a, b, atol=1e-9)
    np.testing.assert_allclose(a, c, atol=1e-9)


def test_gradient_magnitude_one_away_from_medial_axis(oracle):
    sp = W.square(65)
    g = grid_of(oracle, sp, 1)
    phi, _ = g.solve(equation=1, tol_l2=1e-11, max_iters=20000)
    x, y = sp.xyz
    P = phi.reshape(65, 65)
    gy, gx = np.gradient(P, 1 / 64, 1 / 64)
    gm = np.hypot(gx, gy).reshape(-1)
    d = np.minimum.reduce([x, 1 - x, y, 1 - y])
    # distance to the medial axis (diagonals of the square)
    dm = np.minimum(np.abs(x - y), np.abs(x + y - 1)) / np.sqrt(2)
    sel = (dm > 0.1) & (d > 0.05)
    assert np.abs(gm[sel] - 1).max() < 0.02


def test_duct_x_invariance(oracle):
    sp = W.duct(17, nx=8)
    g = grid_of(oracle, sp, 2)
    phi, st = g.solve(equation=1, scheme=2, tol_l2=1e-11, max_iters=20000)
    assert st["converged"]
    P = phi.reshape(17, 17, 8)
    np.testing.assert_allclose(P, np.repeat(P[:, :, :1], 8, axis=2), atol=1e-12)
    x, y, z = sp.xyz
    ex = np.minimum.reduce([y, 1 - y, z, 1 - z])
    assert np.abs(phi - ex).max() < 0.06


def test_cylinder_lad_curvature_beats_plain(oracle):
    """O-grid around a circle, exact d = r - 1/2: LAD with the curvature correction is
    more accurate than LAD alone, which is far more accurate than standard HJ."""
    sp = W.cylinder(33, 64, 1.03 ** 8)
    g = grid_of(oracle, sp, 4)
    ex = np.hypot(*sp.xyz) - 0.5
    errs = {}
    for name, eq, cv in (("std", 0, 0), ("lad", 1, 0), ("lad+curv", 1, 1)):
        phi, st = g.solve(equation=eq, curvature=cv, scheme=4, cfl=0.6, alpha_f=0.495,
                          tol_l2=1e-10, max_iters=20000, poisson_max_iters=100, poisson_tol=0)
        assert st["converged"], name
        errs[name] = np.abs(phi - ex).max()
    assert errs["lad+curv"] < errs["lad"] < 0.05 * errs["std"], errs


def test_paper_claims_on_channel(oracle):
    claim = GOLD["lad_vs_standard_l2"]
    nj = claim["grid_nodes_across_checked"]
    sp = W.channel(8, nj)
    y = sp.xyz[1]
    ex = np.minimum(y, 1 - y)
    h = 1.0 / (nj - 1)
    g = grid_of(oracle, sp, 1)
    res = {}
    for eq in (0, 1):
        phi, st = g.solve(equation=eq, tol_l2=1e-12, max_iters=40000, poisson_max_iters=100,
                          poisson_tol=0)
        assert st["converged"]
        res[eq] = phi
    l2 = {eq: np.sqrt((1.0 / 8) * h * ((res[eq] - ex) ** 2).sum()) for eq in res}   # Eq. 24
    assert l2[0] / l2[1] > claim["ratio_min_checked"], l2
    sc = GOLD["standard_hj_error_scatter"]
    act = ex > 0
    pct = (ex[act] - res[0][act]) / ex[act] * 100
    lo, hi = sc["pct_range_checked"]
    assert pct.min() > lo and pct.max() < hi and pct.mean() > 0


def test_lad_constant_sensitivity(oracle):
    """Changing C by 10% changes the LAD error by a few percent: 3-5% in this reading, where
    the paper reports under 1% (a stated deviation, tests/golden/paper_claims.json), and far
    less than the 10% change of C itself."""
    claim = GOLD["lad_c_sensitivity"]
    sp = W.channel(8, 65)
    y = sp.xyz[1]
    ex = np.minimum(y, 1 - y)
    g = grid_of(oracle, sp, 1)
    e = []
    for C in (0.09, 0.10, 0.11):
        phi, _ = g.solve(equation=1, C_lad=C, tol_l2=1e-12, poisson_max_iters=100, poisson_tol=0)
        e.append(np.sqrt(((phi - ex) ** 2).mean()))
    for k in (0, 2):
        assert abs(e[k] - e[1]) / e[1] < claim["rel_change_max_checked"], e
    assert e[0] < e[1] < e[2]   # more diffusivity, more smoothing of the kink


def sampled_ellipse_distance(sp, n=16384):
    """Distance from every node to the nearest of n points sampled uniformly in the
    parameter on the ellipse (sampling error below half the largest chord)."""
    a, b = sp.meta["a"], sp.meta["b"]
    t = 2 * np.pi * np.arange(n) / n
    wx, wy = a * np.cos(t), b * np.sin(t)
    x, y = sp.xyz
    d = np.full(x.shape, np.inf)
    for k in range(0, n, 2048):
        d = np.minimum(d, np.hypot(x[:, None] - wx[None, k:k + 2048], y[:, None] - wy[None, k:k + 2048]).min(1))
    return d


@pytest.mark.parametrize("aspect", [1.16, 3.46])
def test_ellipse_against_sampled_distance(oracle, aspect):
    """Ellipse O-grids (axis ratio up to 3.46, skewed cells near the tips) converge and
    match the brute-force distance to 16384 sampled wall points within the 65x128
    discretisation error."""
    sp = W.ellipse(65, 128, aspect)
    g = grid_of(oracle, sp, 4)
    phi, st = g.solve(equation=1, scheme=4, cfl=0.6, tol_l2=1e-6, max_iters=2000,
                      poisson_max_iters=100, alpha_f=0.49)
    assert st["converged"] and not st["diverged"]
    err = np.abs(phi - sampled_ellipse_distance(sp))
    assert err.max() <= 1.5e-2
    assert np.sqrt((err ** 2).mean()) <= 5e-3


@pytest.mark.parametrize("scheme", [0, 1, 4])
def test_eikonal_channel_errors_where_fronts_meet(oracle, scheme):
    """Eikonal with central schemes (Gamma = 0, filtered): the error peaks on the channel's
    centre line, where the fronts from both walls meet, and HJ-LAD's global L2 error is below
    the Eikonal one for the same scheme (tests/golden/paper_claims.json, eikonal_channel)."""
    claim = GOLD["eikonal_channel"]
    sp = W.channel(16, 65)
    ex = np.minimum(sp.xyz[1], 1 - sp.xyz[1])
    err = {}
    for eq in (2, 1):
        g = grid_of(oracle, sp, scheme)
        phi, st = g.solve(equation=eq, scheme=scheme, cfl=0.8 if scheme < 3 else 0.6, tol_l2=1e-10,
                          max_iters=20000, poisson_max_iters=100, alpha_f=0.49)
        assert st["converged"]
        err[eq] = np.abs(phi - ex).reshape(65, 16)
    j = np.unravel_index(np.argmax(err[2]), err[2].shape)[0]
    assert abs(j - 32) <= claim["centre_tolerance_nodes"]
    l2 = {eq: np.sqrt((e ** 2).mean()) for eq, e in err.items()}
    assert l2[1] < l2[2]
