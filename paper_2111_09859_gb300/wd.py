"""Thin ctypes binding of libwd (include/wd.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of libwd.
PyTorch supplies device memory (tensors) and the current CUDA stream.  There is no CPU
fallback: if the compiled library is missing, loading fails with an error that says how
to build it.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libwd.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_TIMEOUT = range(7)
BC_WALL, BC_FARFIELD, BC_NEUMANN, BC_PERIODIC = 0, 1, 2, 3
FP64, FP32_METRIC64, FP32 = 0, 1, 2
HJ_STD, HJ_LAD, EIKONAL = 0, 1, 2
E2, E4, E6, C4, C6, UW = 0, 1, 2, 3, 4, 5
INIT_ZERO, INIT_POISSON, INIT_GIVEN = 0, 1, 2


class WDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libwd status {status}: {msg}")
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("n", C.c_int * 3), ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3),
        ("period", (C.c_double * 3) * 3), ("precision", C.c_int), ("scheme", C.c_int),
        ("L_ref", C.c_double),
    ]


class SolveParams(C.Structure):
    _fields_ = [
        ("equation", C.c_int), ("curvature", C.c_int), ("eps", C.c_double), ("C_lad", C.c_double),
        ("lad_exp", C.c_double), ("alpha_f", C.c_double), ("filter", C.c_int), ("cfl", C.c_double),
        ("eps0", C.c_double), ("tol_l2", C.c_double), ("tol_linf", C.c_double),
        ("max_iters", C.c_int), ("check_every", C.c_int), ("init", C.c_int),
        ("poisson_tol", C.c_double), ("poisson_max_iters", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("iters", C.c_int), ("poisson_iters", C.c_int), ("res_l2", C.c_double),
        ("res_linf", C.c_double), ("converged", C.c_int), ("diverged", C.c_int),
        ("stalled", C.c_int), ("seconds", C.c_double), ("device_bytes", C.c_size_t),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerConfig(C.Structure):
    _fields_ = [("max_device_bytes", C.c_size_t), ("max_active", C.c_int), ("pool_per_shape", C.c_int)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes); mirrors include/wd.h
_vp, _i, _d = C.c_void_p, C.c_int, C.c_double
SIGNATURES = {
    "wd_default_params": (None, [_i, C.POINTER(SolveParams)]),
    "wd_create_grid": (_i, [C.POINTER(GridDesc), _vp, _vp, _vp, _vp, C.POINTER(_vp)]),
    "wd_destroy_grid": (None, [_vp]),
    "wd_set_stream": (_i, [_vp, _vp]),
    "wd_solve": (_i, [_vp, C.POINTER(SolveParams), _vp, C.POINTER(Stats)]),
    "wd_step_unsteady": (_i, [_vp, _vp, _vp, C.POINTER(SolveParams), _vp, C.POINTER(Stats)]),
    "wd_solve_batch": (_i, [C.POINTER(_vp), _i, C.POINTER(SolveParams), C.POINTER(_vp), C.POINTER(Stats)]),
    "wd_query_footprint": (C.c_size_t, [C.POINTER(GridDesc), C.POINTER(SolveParams)]),
    "wd_status_string": (C.c_char_p, [_i]),
    "wd_last_error": (C.c_char_p, []),
    "wd_get_metrics": (_i, [_vp, _vp, _vp, _vp]),
    "wd_derivative": (_i, [_vp, _i, _vp, _vp]),
    "wd_filter": (_i, [_vp, _d, _i, _vp, _vp]),
    "wd_rhs": (_i, [_vp, C.POINTER(SolveParams), _i, _vp, _vp, _vp]),
    "wd_spalding": (_i, [_vp, _vp, _vp]),
    "wd_apply_bc": (_i, [_vp, _vp]),
    "wd_steps": (_i, [_vp, C.POINTER(SolveParams), _i, _vp, _i, C.POINTER(Stats)]),
    "wd_profile": (_i, [_vp, _i]),
    "wd_profile_read": (_i, [_vp, _i, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "wd_change_norms_noalloc": (_i, [_vp, _vp, _vp, C.c_longlong, _i, _d, _vp, _vp]),
    "wd_reset_geometry": (_i, [_vp, _vp, _vp, _vp]),
    "wd_get_tuning": (_i, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "wd_recede": (_i, [_vp, _vp, _d, _d, _vp, _vp]),
    "wd_level_length": (_i, [_vp, _vp, _d, C.POINTER(C.c_double)]),
    "wd_levelset": (_i, [_vp, _vp, _d, _d, _i]),
    "wd_server_create": (_i, [C.POINTER(ServerConfig), C.POINTER(_vp)]),
    "wd_server_submit": (_i, [_vp, C.POINTER(GridDesc), _vp, _vp, _vp, C.POINTER(SolveParams), _vp,
                              C.POINTER(C.c_longlong)]),
    "wd_server_submit_grid": (_i, [_vp, _vp, _vp, _vp, _i, C.POINTER(SolveParams), _vp,
                                   C.POINTER(C.c_longlong)]),
    "wd_server_wait": (_i, [_vp, C.c_longlong, _d, C.POINTER(Stats), C.POINTER(C.c_double)]),
    "wd_server_info": (_i, [_vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                            C.POINTER(C.c_longlong), C.POINTER(C.c_size_t), C.POINTER(C.c_longlong)]),
    "wd_server_destroy": (None, [_vp]),
}

K_DERIV, K_DIV, K_FILTER, K_GAUSS, K_POINT, K_BC, K_NORM, K_LINE0, K_LINE1 = range(9)
K_NAMES = ("deriv", "div", "filter", "gauss", "point", "bc", "norm", "line0", "line1")


def lib(path: str | None = None):
    """Loads libwd.so (built by paper_2111_09859_gb300.build / __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(
                    f"libwd.so not found at {p}: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = C.CDLL(p)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status):
    if status != OK:
        msg = lib().wd_last_error().decode(errors="replace")
        raise WDError(status, msg)


def default_params(scheme: int, **overrides) -> SolveParams:
    p = SolveParams()
    lib().wd_default_params(scheme, C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise KeyError(f"unknown solve parameter {k!r}")
        setattr(p, k, v)
    return p


def _stream_handle(stream=None):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _grid_inputs(spec, precision, scheme):
    """(GridDesc, xyz, mask, dval, n) of a GridSpec-like object, arrays as contiguous numpy."""
    shape = tuple(int(s) for s in spec.shape)
    ndim = len(shape)
    batch = int(getattr(spec, "batch", 1))
    n = list(shape) + [1] * (3 - ndim)
    if ndim == 2:
        n[2] = batch
    d = GridDesc()
    d.ndim = ndim
    for k in range(3):
        d.n[k] = n[k]
        d.bc_lo[k] = spec.bc_lo[k] if k < ndim else BC_WALL
        d.bc_hi[k] = spec.bc_hi[k] if k < ndim else BC_WALL
        for m in range(3):
            d.period[k][m] = float(spec.period[k][m]) if spec.period is not None else 0.0
    d.precision = precision
    d.scheme = scheme
    d.L_ref = float(getattr(spec, "L_ref", 1.0))
    xyz = np.ascontiguousarray(np.asarray(spec.xyz, dtype=np.float64).reshape(ndim, -1))
    mask = getattr(spec, "mask", None)
    dval = getattr(spec, "dval", None)
    mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    dval = None if dval is None else np.ascontiguousarray(dval, dtype=np.float64).reshape(-1)
    return d, xyz, mask, dval, n


def _np_ptr(a):
    return None if a is None else a.ctypes.data


class Grid:
    """A structured grid on the GPU (wd_create_grid).

    ``spec`` needs: ``shape`` (ni, nj[, nk]), ``xyz`` (ndim, N) float64 coordinates,
    ``bc_lo`` / ``bc_hi``, ``period``, ``L_ref``, optional ``mask`` / ``dval``."""

    def __init__(self, spec, precision=FP64, scheme=E4, stream=None):
        import torch

        self.shape = tuple(int(s) for s in spec.shape)
        self.ndim = len(self.shape)
        self.batch = int(getattr(spec, "batch", 1))
        d, xyz, mask, dval, n = _grid_inputs(spec, precision, scheme)
        self.n = n
        self.N = n[0] * n[1] * n[2]
        self.precision = precision
        self.scheme = scheme
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        self.desc = d
        self.stream = stream
        h = C.c_void_p()
        _check(lib().wd_create_grid(C.byref(d), xyz.ctypes.data, _np_ptr(mask), _np_ptr(dval),
                                    _stream_handle(stream), C.byref(h)))
        self._h = h
        self._device = torch.device("cuda", torch.cuda.current_device())

    def close(self):
        if getattr(self, "_h", None):
            lib().wd_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tuning(self):
        """(stage kernel block size, stencil block rows, batch parts) chosen by the autotuner
        (0: default)."""
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _check(lib().wd_get_tuning(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def reset_geometry(self, spec):
        """New coordinates / Dirichlet set of the same shape (wd_reset_geometry)."""
        d, xyz, mask, dval, n = _grid_inputs(spec, self.precision, self.scheme)
        if list(n) != list(self.n):
            raise ValueError("reset_geometry needs the grid's shape")
        self._sync_stream()
        _check(lib().wd_reset_geometry(self._h, xyz.ctypes.data, _np_ptr(mask), _np_ptr(dval)))

    def recede(self, phi, s, floor):
        """Surface receded by s (wd_recede): phi is shifted by -s in place (the warm start of
        the next solve); returns (mask uint8 tensor, dval tensor)."""
        import torch

        mask = torch.empty(self.N, dtype=torch.uint8, device=self._device)
        dval = self.empty()
        self._sync_stream()
        _check(lib().wd_recede(self._h, _ptr(phi), float(s), float(floor), _ptr(mask), _ptr(dval)))
        return mask, dval

    def levelset(self, phi, F, dt, nsteps):
        """nsteps RK4 steps of d(phi)/dt + F |grad phi| = 0 (Sec. 5.5) on ``phi`` in place."""
        if phi.numel() != self.N or phi.dtype != self.dtype or not phi.is_contiguous():
            raise ValueError("levelset needs a contiguous field of the grid's size and dtype")
        self._sync_stream()
        _check(lib().wd_levelset(self._h, _ptr(phi), float(F), float(dt), int(nsteps)))
        return phi

    def level_length(self, phi, level=0.0):
        out = C.c_double()
        self._sync_stream()
        _check(lib().wd_level_length(self._h, _ptr(phi), float(level), C.byref(out)))
        return out.value

    def _sync_stream(self):
        lib().wd_set_stream(self._h, _stream_handle(self.stream))

    def empty(self):
        import torch

        return torch.empty(self.N, dtype=self.dtype, device=self._device)

    def as_field(self, a):
        import torch

        t = torch.as_tensor(np.asarray(a).reshape(-1), dtype=self.dtype)
        return t.to(self._device).contiguous()

    # ---- method ------------------------------------------------------------------------
    def solve(self, params: SolveParams, phi=None, allow_fail=False):
        """Steady solve; returns (phi tensor, stats dict)."""
        phi = self.empty() if phi is None else phi
        st = Stats()
        self._sync_stream()
        s = lib().wd_solve(self._h, C.byref(params), _ptr(phi), C.byref(st))
        if not allow_fail and s not in (OK, ERR_NOT_CONVERGED):
            _check(s)
        d = st.as_dict()
        d["status"] = s
        return phi, d

    def step_unsteady(self, params, phi, mask=None, dval=None):
        st = Stats()
        self._sync_stream()
        s = lib().wd_step_unsteady(self._h, _ptr(mask), _ptr(dval), C.byref(params), _ptr(phi),
                                   C.byref(st))
        if s not in (OK, ERR_NOT_CONVERGED):
            _check(s)
        d = st.as_dict()
        d["status"] = s
        return phi, d

    def steps(self, params, phi, n, kind=0):
        st = Stats()
        self._sync_stream()
        _check(lib().wd_steps(self._h, C.byref(params), kind, _ptr(phi), int(n), C.byref(st)))
        return phi, st.as_dict()

    def rhs(self, params, phi, kind=0):
        R, dt = self.empty(), self.empty()
        self._sync_stream()
        _check(lib().wd_rhs(self._h, C.byref(params), kind, _ptr(phi), _ptr(R), _ptr(dt)))
        return R, dt

    def derivative(self, f, dir):
        out = self.empty()
        self._sync_stream()
        _check(lib().wd_derivative(self._h, int(dir), _ptr(f), _ptr(out)))
        return out

    def filter(self, f, dir, alpha_f):
        out = self.empty()
        self._sync_stream()
        _check(lib().wd_filter(self._h, float(alpha_f), int(dir), _ptr(f), _ptr(out)))
        return out

    def spalding(self, phip):
        out = self.empty()
        self._sync_stream()
        _check(lib().wd_spalding(self._h, _ptr(phip), _ptr(out)))
        return out

    def apply_bc(self, phi):
        self._sync_stream()
        _check(lib().wd_apply_bc(self._h, _ptr(phi)))
        return phi

    def profile(self, enable=True):
        _check(lib().wd_profile(self._h, int(bool(enable))))

    def profile_read(self):
        out = {}
        for k, name in enumerate(K_NAMES):
            ms, n = C.c_double(), C.c_longlong()
            _check(lib().wd_profile_read(self._h, k, C.byref(ms), C.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    def metrics(self):
        import torch

        xi = torch.zeros(9 * self.N, dtype=torch.float64, device=self._device)
        J = torch.zeros(self.N, dtype=torch.float64, device=self._device)
        dx = torch.zeros(3 * self.N, dtype=torch.float64, device=self._device)
        self._sync_stream()
        _check(lib().wd_get_metrics(self._h, _ptr(xi), _ptr(J), _ptr(dx)))
        return xi.view(3, 3, self.N), J, dx.view(3, self.N)


def solve_batch(grids, params, phis):
    n = len(grids)
    hs = (C.c_void_p * n)(*[g._h for g in grids])
    ps = (C.c_void_p * n)(*[p.data_ptr() for p in phis])
    sts = (Stats * n)()
    for g in grids:
        g._sync_stream()
    s = lib().wd_solve_batch(hs, n, C.byref(params), ps, sts)
    return s, [st.as_dict() for st in sts]


def footprint(spec, precision=FP64, scheme=E4):
    d = GridDesc()
    shape = tuple(spec.shape)
    d.ndim = len(shape)
    for k in range(3):
        d.n[k] = shape[k] if k < len(shape) else 1
        d.bc_lo[k] = spec.bc_lo[k] if k < len(shape) else BC_WALL
        d.bc_hi[k] = spec.bc_hi[k] if k < len(shape) else BC_WALL
    d.precision = precision
    d.scheme = scheme
    d.L_ref = 1.0
    return lib().wd_query_footprint(C.byref(d), None)


def solve_batch(grids, params, outs=None):
    """wd_solve_batch: the solves of every Grid in grids, side by side on the GPU; returns
    (list of result tensors, list of stats dicts, status).  outs: optional result tensors
    (one per grid, the grid's precision)."""
    n = len(grids)
    outs = [g.empty() for g in grids] if outs is None else list(outs)
    harr = (C.c_void_p * n)(*[g._h for g in grids])
    parr = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    st = (Stats * n)()
    s = lib().wd_solve_batch(harr, n, C.byref(params), parr, st)
    if s not in (OK, ERR_NOT_CONVERGED):
        _check(s)
    return outs, [st[i].as_dict() for i in range(n)], s


def _noalloc_inputs(new, old, mask, out):
    """Checks the arrays of change_norms_noalloc before anything reaches the library, so
    that a wrong dtype, length or layout can never make the kernel read past an array:
    new and old of float32 or float64 with the same dtype and length, contiguous; mask
    None or a contiguous uint8 / bool tensor of the same length; out None or a contiguous
    float64 tensor of 2 entries; every tensor on one CUDA device (checked last).  Returns
    the precision code of the state."""
    import torch

    if new.dtype not in (torch.float32, torch.float64):
        raise ValueError(f"change_norms_noalloc: new must be float32 or float64, not {new.dtype}")
    if old.dtype != new.dtype:
        raise ValueError(f"change_norms_noalloc: old is {old.dtype}, new is {new.dtype}")
    if old.numel() != new.numel() or new.numel() == 0:
        raise ValueError(f"change_norms_noalloc: lengths differ or are zero ({new.numel()}, {old.numel()})")
    if mask is not None and (mask.dtype not in (torch.uint8, torch.bool) or mask.numel() != new.numel()):
        raise ValueError("change_norms_noalloc: mask must be uint8 / bool with one entry per node")
    if out is not None and (out.dtype != torch.float64 or out.numel() != 2):
        raise ValueError("change_norms_noalloc: out must be a float64 tensor of 2 entries")
    ts = [t for t in (new, old, mask, out) if t is not None]
    if not all(t.is_contiguous() for t in ts):
        raise ValueError("change_norms_noalloc: every tensor must be contiguous")
    if not all(t.is_cuda and t.device == new.device for t in ts):
        raise ValueError("change_norms_noalloc: every tensor must be on the same CUDA device")
    return FP64 if new.dtype == torch.float64 else FP32


def change_norms_noalloc(new, old, mask=None, scale=1.0, stream=None, out=None):
    """RMS and max of new - old over entries with mask == 0, through the allocation-free
    entry point (wd_change_norms_noalloc); returns ``out`` (a device tensor of 2 doubles,
    created here when None), enqueued on ``stream`` (default: the current stream of the
    tensors' device).  The call runs with the tensors' device current, because the library
    finds its scratch array on the current device."""
    import torch

    prec = _noalloc_inputs(new, old, mask, out)
    with torch.cuda.device(new.device):
        if out is None:
            out = torch.empty(2, dtype=torch.float64, device=new.device)
        s = stream if stream is not None else torch.cuda.current_stream(new.device)
        _check(lib().wd_change_norms_noalloc(_ptr(new), _ptr(old), _ptr(mask), new.numel(), prec,
                                             float(scale), _ptr(out), C.c_void_p(s.cuda_stream)))
    return out


class Server:
    """Request loop of the library (wd_server_*): continuous batching of independent solves.

    ``submit(spec, params, out)`` queues a solve of a new grid (the server creates or re-uses
    one) and returns a ticket; ``submit_grid(grid, params, phi, ...)`` queues a solve on a
    caller-owned Grid.  ``wait(ticket)`` returns (status, stats dict, latency seconds).
    Output tensors must stay alive until their request is done."""

    def __init__(self, max_device_bytes=0, max_active=0, pool_per_shape=0):
        import torch

        cfg = ServerConfig()
        cfg.max_device_bytes = int(max_device_bytes)
        cfg.max_active = int(max_active)
        cfg.pool_per_shape = int(pool_per_shape)
        h = C.c_void_p()
        _check(lib().wd_server_create(C.byref(cfg), C.byref(h)))
        self._h = h
        self._device = torch.device("cuda", torch.cuda.current_device())
        self._keep = {}

    def submit(self, spec, params, out=None, precision=FP32_METRIC64, scheme=C6):
        import torch

        d, xyz, mask, dval, n = _grid_inputs(spec, precision, scheme)
        if out is None:
            out = torch.empty(n[0] * n[1] * n[2], device=self._device,
                              dtype=torch.float64 if precision == FP64 else torch.float32)
        t = C.c_longlong()
        _check(lib().wd_server_submit(self._h, C.byref(d), xyz.ctypes.data, _np_ptr(mask),
                                      _np_ptr(dval), C.byref(params), _ptr(out), C.byref(t)))
        self._keep[t.value] = out
        return t.value, out

    def submit_grid(self, grid, params, phi, warm=False, mask=None, dval=None):
        grid._sync_stream()
        t = C.c_longlong()
        _check(lib().wd_server_submit_grid(self._h, grid._h, _ptr(mask), _ptr(dval), int(bool(warm)),
                                           C.byref(params), _ptr(phi), C.byref(t)))
        self._keep[t.value] = (phi, mask, dval)
        return t.value

    def wait(self, ticket, timeout=-1.0):
        st = Stats()
        lat = C.c_double()
        s = lib().wd_server_wait(self._h, int(ticket), float(timeout), C.byref(st), C.byref(lat))
        if s == ERR_TIMEOUT:
            return s, None, None
        self._keep.pop(ticket, None)
        if s not in (OK, ERR_NOT_CONVERGED):
            _check(s)
        d = st.as_dict()
        d["status"] = s
        return s, d, lat.value

    def info(self):
        q, r, dn, pk = C.c_longlong(), C.c_longlong(), C.c_longlong(), C.c_longlong()
        b = C.c_size_t()
        _check(lib().wd_server_info(self._h, C.byref(q), C.byref(r), C.byref(dn), C.byref(b), C.byref(pk)))
        return {"queued": q.value, "running": r.value, "done": dn.value, "admitted_bytes": b.value,
                "peak_running": pk.value}

    def close(self):
        if getattr(self, "_h", None):
            lib().wd_server_destroy(self._h)
            self._h = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
