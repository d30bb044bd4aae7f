"""Seeded synthetic grids that stand in for the paper's canonical cases.

This module only builds INPUTS (node coordinates, boundary kinds, Dirichlet masks) with
numpy.  It holds none of the wall-distance method's arithmetic, imports neither the CUDA
binding nor the oracle, and is the one module both sides share.

The paper's case table survives only as an image placeholder, so every grid below is a
synthetic stand-in with the shape the paper's canonical cases suggest (Sec. 4): a 2D box
with four walls, an O-grid around a circular cylinder, a periodic square duct, O-grids
around ellipses, and a star-shaped propellant port on a Cartesian box (Sec. 5.5).

Index convention: node (i, j, k) with i fastest; coordinates are returned with shape
(ndim, N), N = ni * nj * nk.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

WALL, FARFIELD, NEUMANN, PERIODIC = 0, 1, 2, 3


@dataclass
class GridSpec:
    name: str
    shape: tuple            # (ni, nj) or (ni, nj, nk)
    xyz: np.ndarray         # (ndim, N) float64
    bc_lo: tuple
    bc_hi: tuple
    period: tuple = ((0.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0))
    L_ref: float = 1.0
    uniform_h: tuple | None = None   # spacing per direction when the grid is Cartesian
    mask: np.ndarray | None = None   # (N,) uint8, 1 = Dirichlet node
    dval: np.ndarray | None = None   # (N,) float64 Dirichlet values
    meta: dict = field(default_factory=dict)
    batch: int = 1                   # stacked independent 2-D grids (same shape and faces)

    @property
    def ndim(self):
        return len(self.shape)

    @property
    def N(self):
        return int(np.prod(self.shape)) * self.batch

    def grid_shape(self):
        """numpy array shape (nk, nj, ni) / (nj, ni) of one field."""
        return tuple(reversed(self.shape))


def _cartesian(xs, ys, zs=None):
    if zs is None:
        Y, X = np.meshgrid(ys, xs, indexing="ij")
        return np.stack([X.reshape(-1), Y.reshape(-1)])
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)])


def square(n: int = 65) -> GridSpec:
    """Unit square, uniform n x n nodes, all four sides walls (the 2-D box case)."""
    x = np.arange(n) / (n - 1)
    return GridSpec("square", (n, n), _cartesian(x, x), (WALL, WALL), (WALL, WALL),
                    uniform_h=(1.0 / (n - 1), 1.0 / (n - 1)))


def channel(ni: int = 16, nj: int = 33, height: float = 1.0) -> GridSpec:
    """Channel between walls at y = 0 and y = height, periodic in x with period 1."""
    x = np.arange(ni) / ni
    y = np.arange(nj) / (nj - 1) * height
    return GridSpec("channel", (ni, nj), _cartesian(x, y), (PERIODIC, WALL), (PERIODIC, WALL),
                    period=((1.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0)),
                    uniform_h=(1.0 / ni, height / (nj - 1)))


def plate(ni: int = 16, nj: int = 33, height: float = 1.0, stretch: float = 1.0) -> GridSpec:
    """Flat plate: wall at y = 0, far field at y = height, periodic in x.

    ``stretch`` > 1 clusters nodes geometrically towards the wall."""
    x = np.arange(ni) / ni
    if stretch == 1.0:
        y = np.arange(nj) / (nj - 1) * height
    else:
        y = (stretch ** np.arange(nj) - 1.0) / (stretch ** (nj - 1) - 1.0) * height
    return GridSpec("plate", (ni, nj), _cartesian(x, y), (PERIODIC, WALL), (PERIODIC, FARFIELD),
                    period=((1.0, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0)),
                    uniform_h=(1.0 / ni, height / (nj - 1)) if stretch == 1.0 else None)


def duct(n: int = 256, nx: int | None = None) -> GridSpec:
    """Square duct [0,1]^3: walls at y = 0, 1 and z = 0, 1; periodic in x.

    x_i = i / n (n distinct periodic nodes, or ``nx`` of them at the same spacing),
    y_j = j / (n - 1), z_k = k / (n - 1)."""
    nx = n if nx is None else nx
    x = np.arange(nx) / n
    y = np.arange(n) / (n - 1)
    return GridSpec("duct", (nx, n, n), _cartesian(x, y, y), (PERIODIC, WALL, WALL),
                    (PERIODIC, WALL, WALL),
                    period=((nx / n, 0.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, 0.0)),
                    uniform_h=(1.0 / n, 1.0 / (n - 1), 1.0 / (n - 1)))


def geometric_fraction(nr: int, ratio: float) -> np.ndarray:
    """s_j in [0, 1], j = 0..nr-1, with s_{j+1} - s_j growing by ``ratio`` per node."""
    j = np.arange(nr, dtype=np.float64)
    if ratio == 1.0:
        return j / (nr - 1)
    return (ratio ** j - 1.0) / (ratio ** (nr - 1) - 1.0)


def o_grid(inner_xy, nr: int, nt: int, ratio: float, r_out: float = 10.0, name="ogrid",
           meta=None) -> GridSpec:
    """O-grid from a closed inner curve (callable theta -> (x, y)) to a circle of radius
    r_out along straight lines, with geometric radial clustering at the inner wall.

    i runs over nt distinct angles theta_i = -2 pi i / nt (clockwise, so the Jacobian is
    positive with i fastest and j outwards); j = 0 is the wall, j = nr-1 the far field."""
    th = -2.0 * np.pi * np.arange(nt) / nt
    s = geometric_fraction(nr, ratio)
    xi, yi = inner_xy(th)
    xo, yo = r_out * np.cos(th), r_out * np.sin(th)
    X = (1.0 - s)[:, None] * xi[None, :] + s[:, None] * xo[None, :]
    Y = (1.0 - s)[:, None] * yi[None, :] + s[:, None] * yo[None, :]
    return GridSpec(name, (nt, nr), np.stack([X.reshape(-1), Y.reshape(-1)]),
                    (PERIODIC, WALL), (PERIODIC, FARFIELD), meta=meta or {})


def cylinder(nr: int = 257, nt: int = 512, ratio: float = 1.03, r_wall: float = 0.5,
             r_out: float = 10.0) -> GridSpec:
    """O-grid around a circular cylinder.  r_j = r_wall + dr0 (ratio^j - 1)/(ratio - 1)
    with dr0 chosen so that r_{nr-1} = r_out (nr = 257, ratio 1.03 gives dr0 ~ 1.5e-4)."""
    g = o_grid(lambda th: (r_wall * np.cos(th), r_wall * np.sin(th)), nr, nt, ratio, r_out,
               name="cylinder", meta=dict(r_wall=r_wall, r_out=r_out, ratio=ratio))
    return g


def ellipse(nr: int, nt: int, aspect: float, a: float = 0.5, r_out: float = 10.0) -> GridSpec:
    """O-grid around an ellipse with semi-axes a and a / aspect.  The radial ratio is
    1.03^(256/(nr-1)) so that every size spans the same stretching."""
    b = a / aspect
    ratio = 1.03 ** (256.0 / (nr - 1))
    return o_grid(lambda th: (a * np.cos(th), b * np.sin(th)), nr, nt, ratio, r_out,
                  name="ellipse", meta=dict(a=a, b=b, aspect=aspect, ratio=ratio))


ELLIPSE_SIZES = ((65, 128), (129, 256), (257, 512), (513, 1024), (1025, 2048))


def ellipse_stream(n_requests: int, seed_shapes: int = 9859, sizes=ELLIPSE_SIZES):
    """Seeded request mix: (nr, nt, aspect) with aspect ~ U[1, 4] and a uniform size."""
    rng = np.random.default_rng(seed_shapes)
    out = []
    for _ in range(n_requests):
        nr, nt = sizes[int(rng.integers(len(sizes)))]
        out.append((nr, nt, float(rng.uniform(1.0, 4.0))))
    return out


def poisson_arrivals(n: int, rate: float, seed: int = 2111) -> np.ndarray:
    """Arrival times of a Poisson process with the given rate (requests per second)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def random_field(spec: GridSpec, seed: int, smooth: bool = True, amp: float = 1.0) -> np.ndarray:
    """Seeded test field on the grid: a sum of a few random Fourier modes of the
    coordinates (smooth) or white noise."""
    rng = np.random.default_rng(seed)
    if not smooth:
        return amp * rng.standard_normal(spec.N)
    f = np.zeros(spec.N)
    for _ in range(4):
        k = rng.uniform(0.5, 3.0, size=spec.ndim)
        ph = rng.uniform(0, 2 * np.pi)
        f += rng.uniform(0.2, 1.0) * np.sin((k[:, None] * spec.xyz).sum(0) + ph)
    return amp * f


def stack(specs):
    """Stack same-shape 2-D grids (same boundary kinds) into one GridSpec with batch =
    len(specs): grid k occupies nodes k*N .. (k+1)*N - 1 of every array."""
    first = specs[0]
    assert len(first.shape) == 2
    for s in specs:
        assert s.shape == first.shape and s.bc_lo == first.bc_lo and s.bc_hi == first.bc_hi
    xyz = np.concatenate([s.xyz for s in specs], axis=1)
    mask = None
    if any(s.mask is not None for s in specs):
        mask = np.concatenate([s.mask if s.mask is not None else np.zeros(s.N, np.uint8) for s in specs])
    dval = None
    if any(s.dval is not None for s in specs):
        dval = np.concatenate([s.dval if s.dval is not None else np.zeros(s.N) for s in specs])
    return GridSpec(first.name + f"x{len(specs)}", first.shape, xyz, first.bc_lo, first.bc_hi,
                    period=first.period, L_ref=first.L_ref, mask=mask, dval=dval,
                    meta=dict(members=[s.meta for s in specs]), batch=len(specs))
