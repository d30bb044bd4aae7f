"""Shared test helpers: building the same grid for the oracle and for libwd, and one
parameter set for both."""
import numpy as np

ORACLE_KEYS = ("equation", "curvature", "eps", "C_lad", "lad_exp", "alpha_f", "filter", "cfl",
               "eps0", "tol_l2", "tol_linf", "max_iters", "check_every", "init",
               "poisson_tol", "poisson_max_iters")


def base_params(scheme, **kw):
    d = dict(equation=1, curvature=0, eps=0.2, C_lad=0.1, lad_exp=3.0, alpha_f=0.49, filter=1,
             cfl=0.6 if scheme >= 3 else 0.8, eps0=1e-8, tol_l2=1e-10, tol_linf=0.0,
             max_iters=20000, check_every=10, init=1, poisson_tol=0.0, poisson_max_iters=100)
    d.update(kw)
    return d


def oracle_grid(O, spec, scheme):
    return O.Grid(spec.shape, spec.xyz, spec.bc_lo, spec.bc_hi, scheme=scheme,
                  period=spec.period, mask=spec.mask, dval=spec.dval, L_ref=spec.L_ref)


def oracle_kw(scheme, prm):
    kw = {k: prm[k] for k in ORACLE_KEYS}
    kw["scheme"] = scheme
    return kw


def gpu_params(wd, scheme, prm):
    p = wd.default_params(scheme)
    for k in ORACLE_KEYS:
        setattr(p, k, prm[k])
    return p


def to_np(t):
    return t.detach().double().cpu().numpy()


def smooth_state(spec, exact, seed=1, amp=0.02):
    """exact distance plus a smooth seeded perturbation, zero on the walls' value set by BCs"""
    from paper_2111_09859_gb300 import workloads as W

    return exact + amp * W.random_field(spec, seed)
