"""Pins of the oracle's two RK4 integrators against the closed form of classical RK4 on a
linear autonomous system y' = A y + b with step h:

    y_1 = y_0 + h T(hA) (A y_0 + b),   T(z) = 1 + z/2 + z^2/6 + z^3/24,

the degree-3 Taylor polynomial of (exp(z) - 1) / z (1 + z T(z) is the RK4 stability
polynomial).  It is not the stage recursion: a wrong stage weight, a wrong stage abscissa or a stage built from
the wrong predecessor changes the polynomial.

- Pseudo steps (Sec. 3.3): the Poisson pseudo-time equation (Eq. 19) on a doubly periodic
  uniform grid has R = 1 + L phi with L linear, no boundary nodes and a constant local
  step, so one oracle step is the closed form with A = L (L assembled here column by column
  from the oracle's own right-hand side; the pin is on the time integration).
- Level-set steps (Sec. 5.5): for a field increasing along x only, every upwind slope is
  the backward difference, so d(phi)/dt = -F (phi_i - phi_{i-1}) / h is linear; away from
  the inflow face (further than the 4 nodes one step can reach) a step is the closed form
  with A = -(F/h)(I - S), S the backward shift.
"""
import numpy as np


def _taylor_step(A, y0, b, h):
    n = len(y0)
    z = h * A
    T = np.eye(n) + z / 2 + z @ z / 6 + z @ z @ z / 24
    return y0 + h * T @ (A @ y0 + b)


def test_pseudo_step_is_classical_rk4(oracle):
    O = oracle
    n = 8
    xs = np.arange(n) / n
    X, Y = np.meshgrid(xs, xs)
    per = ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 0.0))
    g = O.Grid((n, n), np.stack([X.ravel(), Y.ravel()]), (O.BC_PERIODIC,) * 2, (O.BC_PERIODIC,) * 2,
               scheme=O.E4, period=per)
    kw = dict(scheme=O.E4, filter=0, cfl=0.7)
    N = n * n
    R0, dt = g.rhs_poisson(np.zeros(N), **kw)
    assert np.allclose(R0, 1.0) and np.ptp(dt) < 1e-15
    L = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        L[:, j] = g.rhs_poisson(e, **kw)[0] - R0
    rng = np.random.default_rng(3)
    y0 = rng.standard_normal(N)
    y1, _ = g.poisson_steps(y0, 1, **kw)
    np.testing.assert_allclose(y1, _taylor_step(L, y0, np.ones(N), dt[0]), rtol=0, atol=1e-13)


def test_levelset_step_is_classical_rk4(oracle):
    O = oracle
    nx, ny, F = 40, 9, 0.3
    h = 1.0 / (nx - 1)
    X, Y = np.meshgrid(np.arange(nx) * h, np.arange(ny) * 0.1)
    g = O.Grid((nx, ny), np.stack([X.ravel(), Y.ravel()]), (O.BC_NEUMANN,) * 2, (O.BC_NEUMANN,) * 2,
               scheme=O.E2)
    rng = np.random.default_rng(4)
    row = np.cumsum(rng.uniform(0.2, 1.0, nx)) * h            # increasing along x
    phi0 = np.tile(row, ny)
    dt = 0.45 * h / F
    out = g.levelset_steps(phi0, F, dt, 1).reshape(ny, nx)
    S = np.eye(nx, k=-1)                                       # (S y)_i = y_{i-1}
    A = -(F / h) * (np.eye(nx) - S)
    ref = _taylor_step(A, row, np.zeros(nx), dt)
    for j in range(1, ny - 1):
        np.testing.assert_allclose(out[j, 5:nx - 1], ref[5:nx - 1], rtol=0, atol=1e-14)
