"""FP64 CPU oracle of the HJ / LAD pseudo-HJ wall-distance method (arXiv 2111.09859).

TEST INFRASTRUCTURE ONLY.  The oracle is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline / reference leg, and by
nothing else.  It shares no code with the CUDA path: the arithmetic lives in
``wd_oracle.c`` (plain C, one thread, double precision); this module compiles it with gcc
and marshals numpy arrays through ctypes.  The baseline upwind scheme (Sec. 3.2.1) and the
level-set march (Sec. 5.5) are in the C file too.  Two small pieces of the unsteady case are
plain numpy here: the receding-surface update (Sec. 5.5) and the marching-squares length of
a level set (the burning perimeter).

Parity of every oracle function is pinned by ``tests/test_oracle_*.py`` against things
other than the oracle itself: closed forms, polynomial exactness, Fourier symbols,
dense linear algebra, analytic metrics and brute-force distances.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wd_oracle.c")
_LIB = os.path.join(_HERE, "libwd_oracle.so")
_lock = threading.Lock()
_lib = None

BC_WALL, BC_FARFIELD, BC_NEUMANN, BC_PERIODIC = 0, 1, 2, 3
E2, E4, E6, C4, C6, UW = 0, 1, 2, 3, 4, 5
HJ_STD, HJ_LAD, EIKONAL = 0, 1, 2
INIT_ZERO, INIT_POISSON, INIT_GIVEN = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libwd_oracle.so`` (gcc, -O2, no FP contraction
    so that x86 and Arm hosts give the same bits)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "wd_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class _Desc(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int * 3), ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3),
        ("period", (C.c_double * 3) * 3), ("L_ref", C.c_double),
    ]


class _Params(C.Structure):
    _fields_ = [
        ("equation", C.c_int), ("scheme", C.c_int), ("curvature", C.c_int),
        ("eps", C.c_double), ("C_lad", C.c_double), ("lad_exp", C.c_double),
        ("alpha_f", C.c_double), ("filter", C.c_int), ("cfl", C.c_double), ("eps0", C.c_double),
        ("tol_l2", C.c_double), ("tol_linf", C.c_double), ("max_iters", C.c_int),
        ("check_every", C.c_int), ("init", C.c_int), ("poisson_tol", C.c_double),
        ("poisson_max_iters", C.c_int),
    ]


class _Stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int), ("poisson_iters", C.c_int), ("res_l2", C.c_double),
        ("res_linf", C.c_double), ("converged", C.c_int), ("diverged", C.c_int),
    ]


_DP = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp = C.c_void_p
            L.or_create.restype = vp
            L.or_create.argtypes = [C.POINTER(_Desc), _DP, C.c_int, vp, vp]
            L.or_destroy.argtypes = [vp]
            L.or_set_dirichlet.argtypes = [vp, vp, vp]
            L.or_get_metrics.argtypes = [vp, _DP, _DP, _DP]
            L.or_deriv.argtypes = [vp, C.c_int, C.c_int, _DP, _DP]
            L.or_filter.argtypes = [vp, C.c_double, C.c_int, _DP, _DP]
            L.or_rhs_hj.argtypes = [vp, C.POINTER(_Params), _DP, _DP, _DP]
            L.or_rhs_poisson.argtypes = [vp, C.POINTER(_Params), _DP, _DP, _DP]
            L.or_spalding.argtypes = [vp, C.POINTER(_Params), _DP, _DP]
            L.or_apply_bc.argtypes = [vp, _DP]
            L.or_hj_steps.argtypes = [vp, C.POINTER(_Params), _DP, C.c_int, C.POINTER(_Stats)]
            L.or_poisson_steps.argtypes = [vp, C.POINTER(_Params), _DP, C.c_int, C.POINTER(_Stats)]
            L.or_solve.restype = C.c_int
            L.or_solve.argtypes = [vp, C.POINTER(_Params), _DP, C.POINTER(_Stats)]
            L.or_tridiag.argtypes = [C.c_int, C.c_int, _DP, _DP, _DP, _DP, _DP]
            L.or_filter_coeffs.argtypes = [C.c_int, C.c_double, _DP]
            L.or_upwind_advection.argtypes = [vp, _DP, _DP]
            L.or_upwind_slope.restype = C.c_double
            L.or_upwind_slope.argtypes = [C.c_double, C.c_double]
            L.or_levelset_gradmag.argtypes = [vp, C.c_double, _DP, _DP]
            L.or_levelset_steps.argtypes = [vp, C.c_double, C.c_double, _DP, C.c_int]
            _lib = L
    return _lib


DEFAULT_PARAMS = dict(
    equation=HJ_STD, scheme=E4, curvature=0, eps=0.2, C_lad=0.1, lad_exp=3.0,
    alpha_f=0.49, filter=1, cfl=0.8, eps0=1e-8, tol_l2=1e-10, tol_linf=0.0,
    max_iters=20000, check_every=10, init=INIT_POISSON, poisson_tol=0.0,
    poisson_max_iters=100,
)


def make_params(**kw) -> _Params:
    d = dict(DEFAULT_PARAMS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError(f"unknown oracle parameter {k!r}")
        d[k] = v
    p = _Params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64).reshape(-1)


class Grid:
    """Oracle grid: coordinates ``xyz`` of shape (ndim, nk, nj, ni) or (ndim, nj, ni)."""

    def __init__(self, shape, xyz, bc_lo, bc_hi, scheme=E4, mask=None, dval=None,
                 period=None, L_ref=1.0):
        self.shape = tuple(int(s) for s in shape)        # (ni, nj[, nk])
        self.ndim = len(self.shape)
        n = list(self.shape) + [1] * (3 - self.ndim)
        self.n = n
        self.N = n[0] * n[1] * n[2]
        d = _Desc()
        d.ndim = self.ndim
        for k in range(3):
            d.n[k] = n[k]
            d.bc_lo[k] = bc_lo[k] if k < self.ndim else BC_WALL
            d.bc_hi[k] = bc_hi[k] if k < self.ndim else BC_WALL
            for m in range(3):
                d.period[k][m] = 0.0 if period is None else float(period[k][m])
        d.L_ref = L_ref
        self._desc = d
        x = np.zeros((3, self.N))
        xyz = np.asarray(xyz, dtype=np.float64).reshape(self.ndim, -1)
        x[: self.ndim] = xyz
        self._xyz = np.ascontiguousarray(x)
        self._mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self._dval = None if dval is None else _f64(dval)
        self.scheme = scheme
        self._h = lib().or_create(
            C.byref(d), self._xyz.reshape(-1), scheme,
            None if self._mask is None else self._mask.ctypes.data,
            None if self._dval is None else self._dval.ctypes.data,
        )
        if not self._h:
            raise ValueError("oracle rejected the grid description")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    # ---- array helpers -------------------------------------------------------------
    def _out(self):
        return np.zeros(self.N)

    # ---- operators -----------------------------------------------------------------
    def set_dirichlet(self, mask, dval=None):
        self._mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self._dval = None if dval is None else _f64(dval)
        lib().or_set_dirichlet(self._h, None if self._mask is None else self._mask.ctypes.data,
                               None if self._dval is None else self._dval.ctypes.data)

    def metrics(self):
        xi, J, dx = np.zeros(9 * self.N), np.zeros(self.N), np.zeros(3 * self.N)
        lib().or_get_metrics(self._h, xi, J, dx)
        return xi.reshape(3, 3, self.N), J, dx.reshape(3, self.N)

    def deriv(self, f, dir, scheme=None):
        out = self._out()
        lib().or_deriv(self._h, self.scheme if scheme is None else scheme, dir, _f64(f), out)
        return out

    def filter(self, f, dir, alpha_f):
        out = self._out()
        lib().or_filter(self._h, alpha_f, dir, _f64(f), out)
        return out

    def rhs_hj(self, phi, **params):
        R, dt = self._out(), self._out()
        p = make_params(**params)
        lib().or_rhs_hj(self._h, C.byref(p), _f64(phi), R, dt)
        return R, dt

    def rhs_poisson(self, phi, **params):
        R, dt = self._out(), self._out()
        p = make_params(**params)
        lib().or_rhs_poisson(self._h, C.byref(p), _f64(phi), R, dt)
        return R, dt

    def spalding(self, phip, **params):
        out = self._out()
        p = make_params(**params)
        lib().or_spalding(self._h, C.byref(p), _f64(phip), out)
        return out

    def apply_bc(self, phi):
        a = _f64(phi).copy()
        lib().or_apply_bc(self._h, a)
        return a

    def hj_steps(self, phi, n, **params):
        a = _f64(phi).copy()
        st = _Stats()
        p = make_params(**params)
        lib().or_hj_steps(self._h, C.byref(p), a, int(n), C.byref(st))
        return a, _stats_dict(st)

    def poisson_steps(self, phip, n, **params):
        a = _f64(phip).copy()
        st = _Stats()
        p = make_params(**params)
        lib().or_poisson_steps(self._h, C.byref(p), a, int(n), C.byref(st))
        return a, _stats_dict(st)

    def upwind_advection(self, phi):
        """U.grad(phi) of the baseline upwind scheme (Eqs. UW1-UW5)."""
        out = self._out()
        lib().or_upwind_advection(self._h, _f64(phi), out)
        return out

    def levelset_gradmag(self, phi, F):
        """|grad phi| from the upwind slopes, for a front of normal speed F."""
        out = self._out()
        lib().or_levelset_gradmag(self._h, float(F), _f64(phi), out)
        return out

    def levelset_steps(self, phi, F, dt, n):
        """n RK4 steps of d(phi)/dt + F |grad phi| = 0 (Sec. 5.5) with time step dt."""
        a = _f64(phi).copy()
        lib().or_levelset_steps(self._h, float(F), float(dt), a, int(n))
        return a

    def solve(self, phi=None, **params):
        a = np.zeros(self.N) if phi is None else _f64(phi).copy()
        st = _Stats()
        p = make_params(**params)
        rc = lib().or_solve(self._h, C.byref(p), a, C.byref(st))
        d = _stats_dict(st)
        d["rc"] = rc
        return a, d


def _stats_dict(st):
    return dict(iters=st.iters, poisson_iters=st.poisson_iters, res_l2=st.res_l2,
                res_linf=st.res_linf, converged=bool(st.converged), diverged=bool(st.diverged))


def tridiag(a, b, c, d, cyclic=False):
    n = len(b)
    x = np.zeros(n)
    lib().or_tridiag(n, int(cyclic), _f64(a), _f64(b), _f64(c), _f64(d), x)
    return x


def upwind_slope(B, F):
    """The upwind slope of Eqs. UW3-UW5 from one backward and one forward difference."""
    return lib().or_upwind_slope(float(B), float(F))


def filter_coeffs(hw, alpha_f):
    a = np.zeros(6)
    lib().or_filter_coeffs(int(hw), float(alpha_f), a)
    return a[: hw + 1]


def recede(phi, s, floor):
    """Receding surface of Sec. 5.5 (reading: the surface recedes by s into the
    propellant, so the distance to it is phi - s, which is also the warm start of the next
    solve; the burned set is {phi - s <= 0}, whose nodes become Dirichlet nodes holding
    phi - s floored at ``floor``).  Returns (phi - s, mask, dval)."""
    new = np.asarray(phi, dtype=np.float64) - s
    mask = (new <= 0.0).astype(np.uint8)
    dval = np.where(mask == 1, np.maximum(new, floor), 0.0)
    return new, mask, dval


def level_length(x, y, phi, shape, level=0.0, periodic=(False, False), period=None):
    """Length of {phi = level} on a 2-D structured grid (i fastest) by marching squares:
    in every cell the zero crossings of phi - level are interpolated linearly along the cell
    edges (in physical coordinates) and joined; a cell with four crossings is split by the
    sign of the mean of its corners.  A periodic direction d adds the cells that close the
    grid (node n-1 to node 0, whose coordinates are shifted by period[d]).  Plain numpy over
    all cells."""
    ni, nj = shape
    v = (np.asarray(phi, dtype=np.float64) - level).reshape(nj, ni)
    X = np.asarray(x, dtype=np.float64).reshape(nj, ni)
    Y = np.asarray(y, dtype=np.float64).reshape(nj, ni)
    per = np.zeros((2, 2)) if period is None else np.asarray(period, dtype=np.float64)[:2, :2]
    if periodic[0]:
        v = np.concatenate([v, v[:, :1]], 1)
        X = np.concatenate([X, X[:, :1] + per[0, 0]], 1)
        Y = np.concatenate([Y, Y[:, :1] + per[0, 1]], 1)
    if periodic[1]:
        v = np.concatenate([v, v[:1, :]], 0)
        X = np.concatenate([X, X[:1, :] + per[1, 0]], 0)
        Y = np.concatenate([Y, Y[:1, :] + per[1, 1]], 0)
    # corners 0 (i, j), 1 (i+1, j), 2 (i+1, j+1), 3 (i, j+1) of every cell
    def corner(a, k):
        return {0: a[:-1, :-1], 1: a[:-1, 1:], 2: a[1:, 1:], 3: a[1:, :-1]}[k]
    V = [corner(v, k).ravel() for k in range(4)]
    CX = [corner(X, k).ravel() for k in range(4)]
    CY = [corner(Y, k).ravel() for k in range(4)]
    neg = [V[k] < 0.0 for k in range(4)]
    px, py, has = [], [], []
    for k in range(4):
        a, b = k, (k + 1) % 4
        h = neg[a] != neg[b]
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(h, V[a] / (V[a] - V[b]), 0.0)
        px.append(CX[a] + t * (CX[b] - CX[a]))
        py.append(CY[a] + t * (CY[b] - CY[a]))
        has.append(h)
    nc = sum(h.astype(int) for h in has)
    total = 0.0
    # two crossings: join them
    two = nc == 2
    idx = np.nonzero(two)[0]
    pts = []
    for q in idx:
        ks = [k for k in range(4) if has[k][q]]
        pts.append(np.hypot(px[ks[1]][q] - px[ks[0]][q], py[ks[1]][q] - py[ks[0]][q]))
    total += float(np.sum(pts)) if pts else 0.0
    # saddles
    for q in np.nonzero(nc == 4)[0]:
        ctr = 0.25 * (V[0][q] + V[1][q] + V[2][q] + V[3][q])
        seg = lambda a, b: np.hypot(px[b][q] - px[a][q], py[b][q] - py[a][q])
        if (ctr < 0.0) == neg[0][q]:
            total += seg(0, 1) + seg(2, 3)
        else:
            total += seg(3, 0) + seg(1, 2)
    return total
