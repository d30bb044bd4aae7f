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


# ---- star-shaped propellant port (Sec. 5.5) ------------------------------------------

def star_geometry(r_tip: float = 0.45, r_valley: float = 0.2, points: int = 6, fillet: float = 0.03):
    """Filleted star: `points` tips at r_tip (theta = k 2pi/points) and valleys at r_valley
    in between, joined by straight edges, every corner replaced by the tangent arc of radius
    `fillet`.  Returns a dict with the segments [(p, q)], the arcs [(centre, start angle,
    sweep)] in boundary order, the polygon vertices and the exact perimeter."""
    nv = 2 * points
    ang = np.pi * np.arange(nv) / points
    rad = np.where(np.arange(nv) % 2 == 0, r_tip, r_valley)
    V = np.stack([rad * np.cos(ang), rad * np.sin(ang)], 1)
    tin, tout, arcs = [], [], []
    for k in range(nv):
        P, A, B = V[k], V[k - 1], V[(k + 1) % nv]
        u1 = (A - P) / np.linalg.norm(A - P)
        u2 = (B - P) / np.linalg.norm(B - P)
        beta = np.arccos(np.clip(u1 @ u2, -1.0, 1.0))       # angle between the two edges
        t = fillet / np.tan(beta / 2)
        bis = (u1 + u2) / np.linalg.norm(u1 + u2)
        c = P + bis * fillet / np.sin(beta / 2)
        p1, p2 = P + t * u1, P + t * u2                      # tangent points (in, out)
        a1 = np.arctan2(*(p1 - c)[::-1])
        a2 = np.arctan2(*(p2 - c)[::-1])
        sweep = (a2 - a1 + np.pi) % (2 * np.pi) - np.pi      # minor arc, signed
        tin.append(p1)
        tout.append(p2)
        arcs.append((c, a1, sweep))
    segs = [(tout[k], tin[(k + 1) % nv]) for k in range(nv)]
    length = sum(np.linalg.norm(q - p) for p, q in segs) + sum(fillet * abs(s) for _, _, s in arcs)
    return dict(vertices=V, segments=segs, arcs=arcs, fillet=fillet, perimeter=float(length),
                r_tip=r_tip, r_valley=r_valley, points=points)


def _inside_polygon_star(x, y, V):
    """Points strictly inside the star-shaped (about the origin) polygon V."""
    nv = len(V)
    th = np.mod(np.arctan2(y, x), 2 * np.pi)
    k = np.minimum((th / (2 * np.pi / nv)).astype(np.int64), nv - 1)
    A, B = V[k], V[(k + 1) % nv]
    # ray from the origin at angle th meets edge A-B at parameter r
    dx, dy = np.cos(th), np.sin(th)
    ex, ey = B[:, 0] - A[:, 0], B[:, 1] - A[:, 1]
    den = dx * ey - dy * ex
    r = (A[:, 0] * ey - A[:, 1] * ex) / den
    return np.hypot(x, y) < r


def star_signed_distance(x, y, geom):
    """Exact distance to the filleted star boundary, negative inside the star (the port),
    positive in the propellant."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    d = np.full(x.shape, np.inf)
    for p, q in geom["segments"]:
        e = q - p
        t = np.clip(((x - p[0]) * e[0] + (y - p[1]) * e[1]) / (e @ e), 0.0, 1.0)
        d = np.minimum(d, np.hypot(x - p[0] - t * e[0], y - p[1] - t * e[1]))
    rho = geom["fillet"]
    for c, a1, sw in geom["arcs"]:
        r = np.hypot(x - c[0], y - c[1])
        a = np.arctan2(y - c[1], x - c[0])
        rel = (a - a1) * np.sign(sw)
        rel = np.mod(rel, 2 * np.pi)
        on = rel <= abs(sw)
        e1 = c + rho * np.array([np.cos(a1), np.sin(a1)])
        e2 = c + rho * np.array([np.cos(a1 + sw), np.sin(a1 + sw)])
        dend = np.minimum(np.hypot(x - e1[0], y - e1[1]), np.hypot(x - e2[0], y - e2[1]))
        d = np.minimum(d, np.where(on, np.abs(r - rho), dend))
    inside = _inside_polygon_star(x, y, geom["vertices"])
    # corner slivers: a tip fillet removes the part of the polygon beyond its arc, a valley
    # fillet adds the part of the outside beyond its arc
    V = geom["vertices"]
    for k, (c, a1, sw) in enumerate(geom["arcs"]):
        P = V[k]
        p1 = c + rho * np.array([np.cos(a1), np.sin(a1)])
        p2 = c + rho * np.array([np.cos(a1 + sw), np.sin(a1 + sw)])
        tri = _in_triangle(x, y, P, p1, p2)
        beyond = tri & (np.hypot(x - c[0], y - c[1]) > rho)
        if k % 2 == 0:
            inside &= ~beyond
        else:
            inside |= beyond
    return np.where(inside, -d, d)


def _in_triangle(x, y, a, b, c):
    def side(p, q):
        return (q[0] - p[0]) * (y - p[1]) - (q[1] - p[1]) * (x - p[0])
    s1, s2, s3 = side(a, b), side(b, c), side(c, a)
    return ((s1 >= 0) & (s2 >= 0) & (s3 >= 0)) | ((s1 <= 0) & (s2 <= 0) & (s3 <= 0))


def star(n: int = 1025, geom=None, band: int = 3) -> GridSpec:
    """Star-shaped port on the Cartesian box [-1, 1]^2 with n x n nodes (h = 2/(n-1)).  The
    box edges take the paper's zero-gradient far-field condition (Sec. 3.5): with outflow
    extrapolation on all four edges the nearly inviscid LAD solve grows a mode from the box
    corners.  Solid (port) nodes are Dirichlet: phi = signed distance (negative) within
    `band` cells of the interface, clamped at -band h deeper in."""
    geom = geom or star_geometry()
    x = -1.0 + 2.0 * np.arange(n) / (n - 1)
    xyz = _cartesian(x, x)
    h = 2.0 / (n - 1)
    sd = star_signed_distance(xyz[0], xyz[1], geom)
    mask = (sd <= 0.0).astype(np.uint8)
    dval = np.where(mask == 1, np.maximum(sd, -band * h), 0.0)
    return GridSpec("star", (n, n), xyz, (NEUMANN, NEUMANN), (NEUMANN, NEUMANN),
                    uniform_h=(h, h), mask=mask, dval=dval,
                    meta=dict(geom=geom, h=h, band=band, signed_distance=sd))
