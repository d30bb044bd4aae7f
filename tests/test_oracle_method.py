"""Pins of the oracle's method steps against closed forms: the HJ residual assembly
(Eqs. 5-7, 9, 25), the Spalding auxiliary equation (Eq. 4), the Poisson pseudo-time
equation (Eq. 19), boundary conditions (Eqs. 22-23), the exact discrete fixed point
d = y of a flat wall, and the convergence norms (Eq. 20)."""
import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W


def grid_of(O, sp, scheme):
    return O.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=scheme, period=sp.period,
                  mask=sp.mask, dval=sp.dval)


def box(n0=12, n1=14, h0=0.1, h1=0.08):
    x = np.arange(n0) * h0
    y = np.arange(n1) * h1
    return W.GridSpec("box", (n0, n1), W._cartesian(x, y), (W.WALL, W.WALL), (W.WALL, W.WALL))


@pytest.mark.parametrize("scheme", [1, 2, 4])
@pytest.mark.parametrize("equation", [0, 1, 2])
def test_rhs_closed_form_quadratic(oracle, scheme, equation):
    """phi = a + b x + c y + p x^2 + q x y + s y^2: every derivative is exact, so
    U = (b + 2 p x + q y, c + q x + 2 s y), lap = 2 p + 2 s, fourth differences vanish and
    R = 1 + Gamma lap - |U|^2 with Gamma = eps max(phi, 0) (standard), 0 (LAD), 0 (Eikonal)."""
    sp = box()
    g = grid_of(oracle, sp, scheme)
    x, y = sp.xyz
    a, b, c, p, q, s = 0.3, 0.7, -0.4, 0.2, -0.15, 0.35
    phi = a + b * x + c * y + p * x * x + q * x * y + s * y * y
    R, dt = g.rhs_hj(phi, equation=equation, scheme=scheme, eps=0.2)
    Ux, Uy = b + 2 * p * x + q * y, c + q * x + 2 * s * y
    G2 = Ux ** 2 + Uy ** 2
    gam = 0.2 * np.maximum(phi, 0) if equation == 0 else 0.0
    np.testing.assert_allclose(R, 1 + gam * (2 * p + 2 * s) - G2, atol=1e-11)


@pytest.mark.parametrize("scheme", [1, 4])
def test_rhs_linear_field_on_sheared_grid(oracle, scheme):
    """On an affine, non-orthogonal grid the metrics are exact constants and a linear field
    phi = a.x + c has U = a exactly at every node (Sec. 3.1 chain rule with all four metric
    terms), lap = 0 and R = 1 - |a|^2."""
    n = 12
    i, j = np.meshgrid(np.arange(n), np.arange(n))
    x = (i + 0.3 * j) / (n - 1)
    y = (0.4 * i + j) / (n - 1)
    g = oracle.Grid((n, n), np.stack([x.ravel(), y.ravel()]), (oracle.BC_FARFIELD,) * 2,
                    (oracle.BC_FARFIELD,) * 2, scheme=scheme)
    for a in ((0.7, 0.2), (-0.3, 0.9)):
        phi = a[0] * x.ravel() + a[1] * y.ravel() + 0.1
        for eq in (0, 2):
            R, _ = g.rhs_hj(phi, equation=eq, scheme=scheme, eps=0.2)
            np.testing.assert_allclose(R, 1 - a[0] ** 2 - a[1] ** 2, rtol=0, atol=1e-12)


@pytest.mark.parametrize("scheme", [1, 4])
def test_rhs_curvature_closed_form(oracle, scheme):
    """With the Nakanishi correction (Eq. 25) and phi = c0 + b x + c y (straight fronts),
    |U| = sqrt(b^2+c^2), n is constant so kappa = 0, lap = 0 and R = 1 - |U|^2."""
    sp = box()
    g = grid_of(oracle, sp, scheme)
    x, y = sp.xyz
    phi = 0.2 + 0.6 * x - 0.9 * y
    R, _ = g.rhs_hj(phi, equation=0, scheme=scheme, curvature=1)
    np.testing.assert_allclose(R, 1 - (0.36 + 0.81), atol=1e-11)


def test_rhs_circle_curvature_sign(oracle):
    """Distance to a circle, phi = r - 1/2, on the O-grid: lap(phi) = 1/r and kappa = 1/r.
    Because the metrics come from the same discrete operators, the discrete chain rule
    reproduces |U| = 1 and lap = 1/r to round-off on this grid, so standard HJ gives
    R = eps phi / r exactly, and the curvature-corrected residual (Eq. 25) is zero up to
    the eps0 regularisation of n."""
    for nr, nt in ((33, 64), (65, 128)):
        sp = W.cylinder(nr, nt, 1.03 ** (256.0 / (nr - 1)))
        g = grid_of(oracle, sp, 4)
        r = np.hypot(*sp.xyz)
        phi = r - 0.5
        R0, _ = g.rhs_hj(phi, equation=0, scheme=4, eps=0.2)
        R1, _ = g.rhs_hj(phi, equation=0, scheme=4, eps=0.2, curvature=1, eps0=1e-8)
        np.testing.assert_allclose(R0, 0.2 * phi / r, atol=1e-10)
        assert np.abs(R1).max() < 1e-7
        # the correction acts only on convex fronts: flipping the sign of phi (a concave
        # front, kappa < 0) leaves MAX(0, |U| kappa) = 0 and the plain Laplacian in place
        R2, _ = g.rhs_hj(0.5 - r, equation=0, scheme=4, eps=0.2, curvature=1, eps0=1e-8)
        R3, _ = g.rhs_hj(0.5 - r, equation=0, scheme=4, eps=0.2, curvature=0)
        v = 0.0
        np.testing.assert_allclose(R2, R3 + v, atol=1e-10)


def test_lad_vanishes_on_linear_and_sees_a_kink(oracle):
    """The LAD diffusivity (Eq. 7) is built from fourth differences: zero on a linear
    field, positive near a kink, and capped by eps*phi."""
    sp = W.channel(16, 33)
    g = grid_of(oracle, sp, 1)
    x, y = sp.xyz
    lin = 0.1 + 0.5 * y
    R_lad, _ = g.rhs_hj(lin, equation=1, eps=0.2)
    R_eik, _ = g.rhs_hj(lin, equation=2)
    np.testing.assert_allclose(R_lad, R_eik, atol=1e-12)
    kink = np.minimum(y, 1 - y)
    R_lad, dt_lad = g.rhs_hj(kink, equation=1, eps=0.2)
    R_eik, dt_eik = g.rhs_hj(kink, equation=2)
    R_std, _ = g.rhs_hj(kink, equation=0, eps=0.2)
    mid = np.abs(y - 0.5) < 1e-9
    far = np.abs(y - 0.5) > 0.3
    # at the ridge LAD = min(eps phi, C|...|) = eps phi, so it equals standard HJ there
    np.testing.assert_allclose(R_lad[mid], R_std[mid], atol=1e-12)
    # far from the ridge (and walls) the field is linear: no diffusion
    assert np.abs(R_lad - R_eik)[far].max() < 1e-12
    assert (dt_lad[mid] < dt_eik[mid]).all()


@pytest.mark.parametrize("lad_exp", [3.0, 4.0])
@pytest.mark.parametrize("c", [0.2, -0.2])
def test_lad_closed_form_on_a_quartic(oracle, lad_exp, c):
    """phi = a + b y + c y^4 on the channel (uniform h in y): the five-point fourth difference
    of y^4 is 24 h^4 at every node, so the LAD term of Eq. 7 is C |(1/h)^4 h^exp 24 c h^4| =
    24 C |c| h^exp at every node (either sign of c), and the Gaussian keeps a constant.  Below
    the cap eps phi, R = 1 + Gamma lap - |U|^2 with lap = 12 c y^2 and U = b + 4 c y^3 (exact away from the
    walls, where only centred rows are used)."""
    sp = W.channel(16, 33)
    g = grid_of(oracle, sp, 1)
    y = sp.xyz[1]
    h = 1.0 / 32
    a, b, C = 0.3, 0.5, 0.1
    phi = a + b * y + c * y ** 4
    R, _ = g.rhs_hj(phi, equation=1, scheme=1, eps=0.2, C_lad=C, lad_exp=lad_exp)
    gam = 24 * C * abs(c) * h ** lad_exp
    assert gam < (0.2 * phi).min()
    ref = 1 + gam * 12 * c * y ** 2 - (b + 4 * c * y ** 3) ** 2
    inner = (y > 4.5 * h) & (y < 1 - 4.5 * h)
    np.testing.assert_allclose(R[inner], ref[inner], rtol=0, atol=1e-12)
    assert np.abs(gam * 12 * c * y[inner] ** 2).max() > 1e3 * 1e-12   # the term is resolved


def test_lad_gaussian_removes_the_nyquist_mode(oracle):
    """The quartic of the previous pin plus d (-1)^i along the periodic direction x: the
    central derivatives of (-1)^i vanish, so U and lap keep their closed forms, while the
    raw LAD field gains an alternating part C s_x 16 d (-1)^i (below the constant part, so
    the absolute value does not fold it).  The Gaussian smoothing must remove it (its
    transfer function is 1 at zero and 0 at the Nyquist wavenumber), leaving Gamma constant
    and R as for the quartic alone."""
    sp = W.channel(16, 33)
    g = grid_of(oracle, sp, 1)
    x, y = sp.xyz
    i = np.rint(x * 16).astype(int)
    h, hx = 1.0 / 32, 1.0 / 16
    a, b, c, C, d = 0.3, 0.5, 0.2, 0.1, 2e-7
    phi = a + b * y + c * y ** 4 + d * (-1.0) ** i
    R, _ = g.rhs_hj(phi, equation=1, scheme=1, eps=0.2, C_lad=C, lad_exp=3.0)
    gam = 24 * C * c * h ** 3
    assert 16 * d * hx ** -1 < 24 * c * h ** 3       # the raw field keeps its sign
    ref = 1 + gam * 12 * c * y ** 2 - (b + 4 * c * y ** 3) ** 2
    inner = (y > 4.5 * h) & (y < 1 - 4.5 * h)
    np.testing.assert_allclose(R[inner], ref[inner], rtol=0, atol=1e-13)


def test_rhs_curvature_velocity_term(oracle):
    """Eq. 25 with phi = c y^2 on the channel (y > 0): n = U / (|U| + eps0) is 1 up to
    eps0, so kappa ~ eps0 / y^2 and the correction MAX(0, |U| kappa) ~ eps0 / y vanish, lap =
    2c exactly, and R = 1 + (eps phi + 0.001 (1 - |U|)^2) 2c - |U|^2 with |U| = 2 c y."""
    sp = W.channel(16, 33)
    g = grid_of(oracle, sp, 1)
    y = sp.xyz[1]
    h, c = 1.0 / 32, 0.3
    phi = c * y ** 2
    R, _ = g.rhs_hj(phi, equation=0, scheme=1, eps=0.2, curvature=1, eps0=1e-8)
    G = 2 * c * y
    ref = 1 + (0.2 * phi + 0.001 * (1 - G) ** 2) * 2 * c - G ** 2
    inner = (y > 0.25) & (y < 1 - 5.5 * h)
    np.testing.assert_allclose(R[inner], ref[inner], rtol=0, atol=1e-7)
    assert (0.001 * (1 - G[inner]) ** 2 * 2 * c).min() > 1e3 * 1e-7    # the term is resolved


def test_local_time_step_special_case(oracle):
    """phi = 0 (zero gradient, zero diffusivity): dt = cfl / sum_l |grad xi_l|, i.e.
    cfl / (1/h0 + 1/h1) on a Cartesian grid."""
    sp = box(h0=0.1, h1=0.05)
    g = grid_of(oracle, sp, 1)
    _, dt = g.rhs_hj(np.zeros(sp.N), equation=0, cfl=0.7)
    np.testing.assert_allclose(dt, 0.7 / (10.0 + 20.0), rtol=1e-12)
    _, dtp = g.rhs_poisson(np.zeros(sp.N), cfl=0.7)
    np.testing.assert_allclose(dtp, 0.7 / (100.0 + 400.0), rtol=1e-12)


def test_local_time_step_sheared_grid(oracle):
    """On the affine grid x = (i + 0.3 j) h, y = (0.4 i + j) h the contravariant metrics are
    the rows of the analytic inverse of [[1, 0.3], [0.4, 1]] / h, so the local step of
    standard HJ on phi = a.x + c is cfl / (sigma_1 max(1, |a|) + eps phi sigma_2) with
    sigma_1 = sum_l |grad xi_l| and sigma_2 = sum_l sum_k |grad xi_l . grad xi_k| (the
    Gershgorin reading of the diffusive bound) from those exact metrics."""
    n = 12
    h = 1.0 / (n - 1)
    i, j = np.meshgrid(np.arange(n), np.arange(n))
    x = (i + 0.3 * j) * h
    y = (0.4 * i + j) * h
    g = oracle.Grid((n, n), np.stack([x.ravel(), y.ravel()]), (oracle.BC_FARFIELD,) * 2,
                    (oracle.BC_FARFIELD,) * 2, scheme=1)
    G = np.linalg.inv(np.array([[1.0, 0.3], [0.4, 1.0]]) * h)     # G[l] = grad xi_l
    s1 = np.linalg.norm(G, axis=1).sum()
    s2 = np.abs(G @ G.T).sum()
    a = (0.7, 0.2)
    phi = a[0] * x.ravel() + a[1] * y.ravel() + 0.4
    _, dt = g.rhs_hj(phi, equation=0, scheme=1, eps=0.2, cfl=0.8)
    ref = 0.8 / (s1 * max(1.0, np.hypot(*a)) + 0.2 * phi * s2)
    np.testing.assert_allclose(dt, ref, rtol=1e-12)


@pytest.mark.parametrize("scheme", [1, 4])
def test_spalding_channel_exact(oracle, scheme):
    """Channel of unit height: phi' = y (1 - y) / 2 solves lap = -1 with phi' = 0 at both
    walls; Eq. 4 with the minus root returns min(y, 1 - y) exactly (the plus root would
    give the distance to the far wall)."""
    sp = W.channel(16, 41)
    g = grid_of(oracle, sp, scheme)
    y = sp.xyz[1]
    d = g.spalding(y * (1 - y) / 2, scheme=scheme)
    np.testing.assert_allclose(d, np.minimum(y, 1 - y), atol=1e-12)


def test_poisson_fixed_point_and_convergence(oracle):
    """Without the filter, phi' = y (1 - y) / 2 is an exact steady state of the Poisson
    pseudo-time equation (Eq. 19) on the channel (D(D) is exact on quadratics); from
    phi' = 0 the iteration approaches it monotonically."""
    sp = W.channel(8, 21)
    g = grid_of(oracle, sp, 1)
    y = sp.xyz[1]
    ex = y * (1 - y) / 2
    out, _ = g.poisson_steps(ex, 20, filter=0, cfl=0.8)
    np.testing.assert_allclose(out, ex, atol=1e-14)
    R, _ = g.rhs_poisson(ex)
    assert np.abs(R).max() < 1e-12
    p = np.zeros(sp.N)
    res = []
    for _ in range(5):
        p, st = g.poisson_steps(p, 200, filter=1, cfl=0.8)
        res.append(st["res_l2"])
    assert all(b < 0.1 * a for a, b in zip(res, res[1:]))     # geometric convergence
    # the filtered fixed point sits close to the quadratic (the order-2 filter rows next
    # to the walls do not preserve quadratics, so it is not exactly on it)
    assert np.abs(p - ex).max() < 1e-4


def test_poisson_far_field_is_neumann(oracle):
    """The auxiliary Poisson problem takes d(phi')/dn = 0 on far-field faces (Sec. 3.5):
    after Poisson steps on the plate (wall y = 0, far field y = 1, stretched so that the
    HJ extrapolation would give another value) every far-field node holds its inner
    neighbour's value."""
    sp = W.plate(8, 33, 1.0, stretch=1.05)
    g = grid_of(oracle, sp, 1)
    p, st = g.poisson_steps(np.zeros(sp.N), 50, filter=0, cfl=0.8)
    P = p.reshape(33, 8)
    assert np.abs(P[-2] - P[-3]).min() > 1e-6        # an extrapolation would differ
    np.testing.assert_array_equal(P[-1], P[-2])


@pytest.mark.parametrize("scheme", [1, 2, 4])
@pytest.mark.parametrize("equation,curv", [(0, 0), (1, 0), (1, 1)])
def test_flat_wall_linear_fixed_point(oracle, scheme, equation, curv):
    """Flat plate (wall y = 0, far field y = H, periodic x): d = y is an exact discrete
    fixed point.  Every derivative is exact on linear fields (also through the metrics of
    a geometrically stretched grid), LAD and the curvature term vanish, and the far-field
    extrapolation uses the actual spacing ratio; the filter works in index space, so it
    preserves y only where y is linear in the index (uniform spacing).  Ten full pseudo
    steps must return y to round-off in both settings."""
    sp = W.plate(8, 33, height=2.0, stretch=1.08)
    g = grid_of(oracle, sp, scheme)
    y = sp.xyz[1]
    out, st = g.hj_steps(y, 10, equation=equation, curvature=curv, scheme=scheme, cfl=0.5,
                         filter=0)
    np.testing.assert_allclose(out, y, atol=1e-12)
    assert st["res_l2"] < 1e-13
    sp = W.plate(8, 33, height=2.0)
    g = grid_of(oracle, sp, scheme)
    y = sp.xyz[1]
    out, st = g.hj_steps(y, 10, equation=equation, curvature=curv, scheme=scheme, cfl=0.5,
                         filter=1)
    np.testing.assert_allclose(out, y, atol=1e-12)
    assert st["res_l2"] < 1e-13


def test_bc_far_field_and_dirichlet(oracle):
    sp = W.plate(8, 20, height=1.0, stretch=1.1)
    g = grid_of(oracle, sp, 1)
    y = sp.xyz[1]
    junk = y.copy()
    top = np.arange(sp.N) // 8 == 19
    bot = np.arange(sp.N) // 8 == 0
    junk[top] = 123.0
    junk[bot] = -7.0
    out = g.apply_bc(junk)
    np.testing.assert_allclose(out, y, atol=1e-13)     # linear extrapolation on spacing
    # extra Dirichlet nodes with values (immersed wall)
    mask = np.zeros(sp.N, np.uint8)
    mask[50] = 1
    dv = np.zeros(sp.N)
    dv[50] = -0.25
    g.set_dirichlet(mask, dv)
    out = g.apply_bc(y)
    assert out[50] == -0.25 and out[51] == y[51]


def test_step_norms_match_numpy(oracle):
    """res_l2 is the RMS of the last step's change over non-Dirichlet nodes / L_ref,
    res_linf its max (Eq. 20)."""
    sp = W.square(17)
    g = grid_of(oracle, sp, 1)
    x, y = sp.xyz
    rng = np.random.default_rng(2)
    phi = g.apply_bc(np.minimum.reduce([x, 1 - x, y, 1 - y]) + 0.01 * rng.standard_normal(sp.N))
    p1, _ = g.hj_steps(phi, 1, equation=1)
    p2, st = g.hj_steps(p1, 1, equation=1)
    act = ~((x == 0) | (x == 1) | (y == 0) | (y == 1))
    d = (p2 - p1)[act]
    assert abs(st["res_l2"] - np.sqrt((d ** 2).mean())) < 1e-15
    assert abs(st["res_linf"] - np.abs(d).max()) < 1e-15
