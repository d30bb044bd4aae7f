"""Pins of the oracle's operators against mathematics that does not come from the oracle:
polynomial exactness and order of accuracy of the central derivatives (Sec. 3.2.2,
Eq. 16), the filter's defining conditions and transfer function (Sec. 3.4, Eq. 21),
dense linear algebra for the tridiagonal solvers, and analytic grid metrics (Sec. 3.1)."""
import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W

SCHEMES = {"E2": 0, "E4": 1, "E6": 2, "C4": 3, "C6": 4}
ORDER = {"E2": 2, "E4": 4, "E6": 6, "C4": 4, "C6": 6}


def line_grid(O, n, periodic, scheme=1):
    """2-D grid whose direction 1 lines have n nodes (direction 0 has 8 nodes)."""
    if periodic:
        sp = W.channel(8, n)          # dir 0 periodic; use dir 0 lines for periodic tests
        sp = W.GridSpec("t", (n, 8), W._cartesian(np.arange(n) / n, np.arange(8) / 7.0),
                        (W.PERIODIC, W.WALL), (W.PERIODIC, W.WALL),
                        period=((1.0, 0, 0), (0, 0, 0), (0, 0, 0)))
        return O.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=scheme, period=sp.period), 0
    sp = W.square(8)
    sp = W.GridSpec("t", (8, n), W._cartesian(np.arange(8) / 7.0, np.arange(n) / (n - 1.0)),
                    (W.WALL, W.WALL), (W.WALL, W.WALL))
    return O.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=scheme), 1


def field_along(n, dir, vals):
    """Field on the (n0, n1) grid that varies only along `dir` with the given line values."""
    if dir == 1:
        return np.repeat(vals[:, None], 8, axis=1).reshape(-1)
    return np.repeat(vals[None, :], 8, axis=0).reshape(-1)


def take_line(f, n, dir):
    if dir == 1:
        return f.reshape(n, 8)[:, 3]
    return f.reshape(8, n)[3]


# ------------------------------------------------------------------------------------
# derivatives
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(SCHEMES))
def test_deriv_exact_on_quadratics_everywhere(oracle, name):
    """Every row (boundary rows included) is at least 2nd order: exact on quadratics."""
    n = 24
    g, d = line_grid(oracle, n, False)
    t = np.arange(n, dtype=float)
    for c0, c1, c2 in [(1.0, 0.0, 0.0), (0.3, -1.7, 0.0), (2.0, 0.5, -0.25)]:
        f = c0 + c1 * t + c2 * t * t
        df = take_line(g.deriv(field_along(n, d, f), d, SCHEMES[name]), n, d)
        np.testing.assert_allclose(df, c1 + 2 * c2 * t, atol=1e-12, rtol=0)


@pytest.mark.parametrize("name", list(SCHEMES))
def test_deriv_interior_polynomial_order(oracle, name):
    """Far from the ends a scheme of order p differentiates degree-p polynomials exactly
    (compact schemes: the boundary rows' influence decays geometrically inwards)."""
    n = 96
    g, d = line_grid(oracle, n, False)
    t = np.arange(n, dtype=float)
    s = (t - n / 2) / 10.0
    p = ORDER[name]
    f = s ** p
    exact = p * s ** (p - 1) / 10.0
    df = take_line(g.deriv(field_along(n, d, f), d, SCHEMES[name]), n, d)
    mid = slice(40, 56)
    np.testing.assert_allclose(df[mid], exact[mid], atol=1e-9 * np.abs(f).max(), rtol=0)
    # and degree p+1 is NOT exact (the order is not higher than claimed)
    f2 = s ** (p + 1)
    df2 = take_line(g.deriv(field_along(n, d, f2), d, SCHEMES[name]), n, d)
    assert np.abs(df2[mid] - (p + 1) * s[mid] ** p / 10.0).max() > 1e-9


def test_deriv_boundary_rows(oracle):
    """Node 0 is a one-sided 4th-order row (exact on quartics at the end node); node 1 is
    the centred 2nd-order row (f_2 - f_0)/2 for every scheme."""
    n = 24
    t = np.arange(n, dtype=float)
    for name, sch in SCHEMES.items():
        g, d = line_grid(oracle, n, False, sch)
        f = (t / 5.0) ** 4
        df = take_line(g.deriv(field_along(n, d, f), d, sch), n, d)
        assert abs(df[0] - 0.0) < 1e-12, name
        # right end, mirrored: exact for a quartic in (n-1-t)
        f2 = ((n - 1 - t) / 5.0) ** 4
        df2 = take_line(g.deriv(field_along(n, d, f2), d, sch), n, d)
        assert abs(df2[-1]) < 1e-12, name
        r = np.random.default_rng(3).standard_normal(n)
        dr = take_line(g.deriv(field_along(n, d, r), d, sch), n, d)
        assert abs(dr[1] - 0.5 * (r[2] - r[0])) < 1e-12, name
        assert abs(dr[n - 2] - 0.5 * (r[n - 1] - r[n - 3])) < 1e-12, name


def modified_wavenumber(name, w):
    """Fourier symbol of Eq. 16: (a sin w + b/2 sin 2w) / (1 + 2 alpha cos w)."""
    if name == "E6":
        return 1.5 * np.sin(w) - 0.3 * np.sin(2 * w) + np.sin(3 * w) / 30.0
    al, a, b = {"E2": (0, 1, 0), "E4": (0, 4 / 3, -1 / 3), "C4": (0.25, 1.5, 0),
                "C6": (1 / 3, 14 / 9, 1 / 9)}[name]
    return (a * np.sin(w) + 0.5 * b * np.sin(2 * w)) / (1 + 2 * al * np.cos(w))


@pytest.mark.parametrize("name", list(SCHEMES))
def test_deriv_periodic_symbol(oracle, name):
    n = 40
    g, d = line_grid(oracle, n, True)
    t = np.arange(n, dtype=float)
    for k in (1, 3, 7, 13, 19):
        w = 2 * np.pi * k / n
        f = np.sin(w * t + 0.4)
        df = take_line(g.deriv(field_along(n, d, f), d, SCHEMES[name]), n, d)
        np.testing.assert_allclose(df, modified_wavenumber(name, w) * np.cos(w * t + 0.4),
                                   atol=1e-12, rtol=0)
    # the symbol is consistent to the scheme's order: k(w) - w = O(w^(p+1))
    p = ORDER[name]
    e1 = abs(modified_wavenumber(name, 0.1) - 0.1)
    e2 = abs(modified_wavenumber(name, 0.05) - 0.05)
    assert 0.8 * 2 ** (p + 1) < e1 / e2 < 1.2 * 2 ** (p + 1)


# ------------------------------------------------------------------------------------
# tridiagonal solvers
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("cyclic", [False, True])
def test_tridiag_matches_dense_solve(oracle, cyclic):
    rng = np.random.default_rng(11)
    for n in (5, 8, 33, 257):
        a, c = rng.uniform(-0.45, 0.45, n), rng.uniform(-0.45, 0.45, n)
        b = 1.0 + rng.uniform(0.0, 0.5, n)
        d = rng.standard_normal(n)
        A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
        if cyclic:
            A[0, n - 1] = a[0]
            A[n - 1, 0] = c[n - 1]
        x = oracle.tridiag(a, b, c, d, cyclic)
        np.testing.assert_allclose(x, np.linalg.solve(A, d), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------------------------
# filter
# ------------------------------------------------------------------------------------

@pytest.mark.parametrize("hw", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("al", [0.0, 0.3, 0.48, 0.49, 0.495])
def test_filter_coefficients_solve_their_defining_conditions(oracle, hw, al):
    """Order-2N filter: T(0) = 1, T(pi) = 0 and T(w) = 1 + O(w^{2N}), i.e.
    sum a_n = 1 + 2 al, sum (-1)^n a_n = 0, sum a_n n^{2k} = 2 al (k = 1..N-1).
    Solving this system with numpy must give the oracle's table."""
    N = hw
    M = np.zeros((N + 1, N + 1))
    r = np.zeros(N + 1)
    M[0] = 1.0
    r[0] = 1 + 2 * al
    M[1] = [(-1.0) ** n for n in range(N + 1)]
    r[1] = 0.0
    for k in range(1, N):
        M[k + 1] = [float(n) ** (2 * k) for n in range(N + 1)]
        r[k + 1] = 2 * al
    np.testing.assert_allclose(oracle.filter_coeffs(hw, al), np.linalg.solve(M, r),
                               rtol=1e-12, atol=1e-14)


def test_filter_transfer_function_periodic(oracle):
    n = 40
    g, d = line_grid(oracle, n, True)
    t = np.arange(n, dtype=float)
    for al in (0.48, 0.49, 0.495):
        a = oracle.filter_coeffs(5, al)
        for k in (0, 2, 9, 15, 20):
            w = 2 * np.pi * k / n
            T = sum(a[m] * np.cos(m * w) for m in range(6)) / (1 + 2 * al * np.cos(w))
            f = np.cos(w * t + 0.3)
            out = take_line(g.filter(field_along(n, d, f), d, al), n, d)
            np.testing.assert_allclose(out, T * f, atol=1e-12, rtol=0)
    # the odd-even mode is removed exactly
    f = (-1.0) ** t
    out = take_line(g.filter(field_along(n, d, f), d, 0.49), n, d)
    assert np.abs(out).max() < 1e-12


def test_filter_nonperiodic_ends(oracle):
    n = 30
    g, d = line_grid(oracle, n, False)
    t = np.arange(n, dtype=float)
    rng = np.random.default_rng(5)
    f = rng.standard_normal(n)
    out = take_line(g.filter(field_along(n, d, f), d, 0.49), n, d)
    assert out[0] == f[0] and out[-1] == f[-1]           # end nodes are not filtered
    lin = 0.7 - 0.2 * t
    outl = take_line(g.filter(field_along(n, d, lin), d, 0.49), n, d)
    np.testing.assert_allclose(outl, lin, atol=1e-12)   # every member preserves lines
    cub = ((t - 15) / 10.0) ** 3
    outc = take_line(g.filter(field_along(n, d, cub), d, 0.49), n, d)
    # order 4 and up preserve cubics up to the coupling with row 1, which decays inwards
    assert np.abs(outc[10:20] - cub[10:20]).max() < 0.2 * np.abs(outc[1:3] - cub[1:3]).max() + 1e-12
    # the odd-even mode is removed away from the ends; what is left is the unfiltered end
    # node's influence, which decays geometrically inwards
    n2 = 80
    g2, d2 = line_grid(oracle, n2, False)
    osc = (-1.0) ** np.arange(n2)
    outo = np.abs(take_line(g2.filter(field_along(n2, d2, osc), d2, 0.49), n2, d2))
    assert outo[35:45].max() < 0.01
    assert (np.diff(outo[5:40]) < 0).all()


# ------------------------------------------------------------------------------------
# metrics
# ------------------------------------------------------------------------------------

def test_metrics_uniform_and_affine(oracle):
    sp = W.square(17)
    g = oracle.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=1)
    xi, J, dx = g.metrics()
    np.testing.assert_allclose(xi[0, 0], 16.0, rtol=1e-12)
    np.testing.assert_allclose(xi[1, 1], 16.0, rtol=1e-12)
    assert np.abs(xi[0, 1]).max() < 1e-10 and np.abs(xi[1, 0]).max() < 1e-10
    np.testing.assert_allclose(J, 1 / 256.0, rtol=1e-12)
    np.testing.assert_allclose(dx[:2], 1 / 16.0, rtol=1e-12)
    # 3-D affine map x = M xi + c: the metrics are M^-1 exactly, for every scheme
    M = np.array([[0.9, 0.2, -0.1], [0.05, 1.1, 0.3], [0.15, -0.2, 0.8]]) * 0.1
    n = (9, 10, 11)
    K, Jj, I = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = np.stack([I.reshape(-1), Jj.reshape(-1), K.reshape(-1)]).astype(float)
    xyz = M @ idx + np.array([[0.3], [-0.2], [1.0]])
    Minv = np.linalg.inv(M)
    for sch in SCHEMES.values():
        g3 = oracle.Grid(n, xyz, (0, 0, 0), (0, 0, 0), scheme=sch)
        xi3, J3, dx3 = g3.metrics()
        for l in range(3):
            for m in range(3):
                np.testing.assert_allclose(xi3[l, m], Minv[l, m], atol=1e-11)
        np.testing.assert_allclose(J3, np.linalg.det(M), rtol=1e-11)
        np.testing.assert_allclose(dx3[1], np.linalg.norm(M[:, 1]), rtol=1e-11)


def test_metrics_periodic_shift(oracle):
    """A periodic direction whose coordinate jumps by the period (duct x) still gets
    constant metrics."""
    sp = W.duct(12, nx=8)
    g = oracle.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=2, period=sp.period)
    xi, J, dx = g.metrics()
    np.testing.assert_allclose(xi[0, 0], 12.0, rtol=1e-12)
    np.testing.assert_allclose(xi[1, 1], 11.0, rtol=1e-12)
    np.testing.assert_allclose(xi[2, 2], 11.0, rtol=1e-12)


def _polar_metric_error(O, sch, nr, nt):
    q = 1.03 ** (256.0 / (nr - 1))
    sp = W.cylinder(nr, nt, q)
    g = O.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=sch, period=sp.period)
    xi, J, dx = g.metrics()
    j = np.arange(nr, dtype=float)
    dr0 = 9.5 * (q - 1) / (q ** (nr - 1) - 1)
    r = 0.5 + dr0 * (q ** j - 1) / (q - 1)
    drdj = dr0 * q ** j * np.log(q) / (q - 1)
    th = -2 * np.pi * np.arange(nt) / nt
    R, TH = np.meshgrid(r, th, indexing="ij")
    DR = np.meshgrid(drdj, th, indexing="ij")[0]
    dthdi = -2 * np.pi / nt
    # d(xi)/dx = -sin(th) / (r dth/di), d(xi)/dy = cos(th) / (r dth/di),
    # d(eta)/dx = cos(th) / r'(j),      d(eta)/dy = sin(th) / r'(j)
    ex = [[-np.sin(TH) / (R * dthdi), np.cos(TH) / (R * dthdi)],
          [np.cos(TH) / DR, np.sin(TH) / DR]]
    worst = 0.0
    for l in range(2):
        scale = np.abs(ex[l][0]) + np.abs(ex[l][1])
        for m in range(2):
            err = np.abs(xi[l, m].reshape(nr, nt) - ex[l][m]) / scale
            worst = max(worst, err.max())
    return worst, J


@pytest.mark.parametrize("sch", [1, 4])
def test_metrics_polar_ogrid_analytic(oracle, sch):
    """O-grid x = r(j) cos(th_i), y = r(j) sin(th_i), th_i = -2 pi i / nt, r geometric:
    the metrics converge to the analytic polar metrics at (at least) the 2nd order that
    the node-1 boundary row allows, and the Jacobian is positive."""
    errs = []
    for nr, nt in ((33, 64), (65, 128), (129, 256)):
        e, J = _polar_metric_error(oracle, sch, nr, nt)
        assert (J > 0).all()
        errs.append(e)
    assert errs[2] < 1e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
