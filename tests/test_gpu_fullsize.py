"""Full-size parity against the FP64 oracle, at the sizes and parameters the benchmark runs.

- The headline batch (16 stacked cylinder O-grids 257 x 512, C6 + LAD + curvature,
  alpha_f 0.495, FP32 state on FP64 metric Jacobians, tolerance 1e-6) and the plain FP64
  single-cylinder solve (tolerance 1e-10) against the stored oracle solutions
  (tests/golden/cylinder257x512_c6_lad_curv.json, written by make_cylinder_golden.py from the
  oracle alone, solved to 1e-12): each cylinder's oracle field depends on the radial index
  only (rotational symmetry), up to the stored spread over the angular index.
- Pseudo steps of the two largest ellipse O-grids of the serving stream (513 x 1024 and
  1025 x 2048, whose lines need the 32-, 33- and 64-row partition solves) and of the 1025^2
  star port with the receding-grain parameters, against the oracle run live on the same
  inputs, element by element.

Tolerances: full solves 1e-6 L (FP64) and 2e-4 L (FP32) plus the golden's spread; pseudo
steps 1e-10 (FP64) and 1e-5 (FP32) of the field scale, as in test_gpu_parity."""
import json
import os

import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W
from tests.helpers import to_np

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cylinder257x512_c6_lad_curv.json")


@pytest.fixture(scope="module")
def wd():
    import torch

    assert torch.cuda.is_available()
    from paper_2111_09859_gb300 import build, wd as _wd

    build.build()
    return _wd


@pytest.fixture(scope="module")
def golden():
    return json.load(open(GOLDEN))


def scale(a):
    return max(1.0, float(np.abs(a).max()))


def cyl_params(wd, tol):
    # the benchmark's parameters (bench.py solve_params)
    return wd.default_params(wd.C6, equation=wd.HJ_LAD, curvature=1, alpha_f=0.495, tol_l2=tol, max_iters=20000,
                             check_every=10, poisson_max_iters=100)


def test_golden_matches_its_writer(golden):
    """The stored oracle parameters are the benchmark's (C6, LAD, curvature, alpha_f 0.495,
    compact CFL 0.6, 100 Poisson steps), every member converged, and the angular spread is
    rounding-level."""
    p = golden["params"]
    assert (p["scheme"], p["equation"], p["curvature"], p["alpha_f"], p["cfl"], p["poisson_max_iters"]) == (4, 1, 1, 0.495, 0.6, 100)
    assert len(golden["members"]) == 16
    for m in golden["members"]:
        assert m["converged"] and m["res_l2"] <= 1e-12 and m["spread_over_i"] <= 1e-9 and len(m["d"]) == 257


def test_headline_fp32_batch_matches_oracle(wd, golden):
    import torch

    members = [W.cylinder(257, 512, 1.03, r_wall=0.5 * (1 + 0.01 * k)) for k in range(16)]
    spec = W.stack(members)
    g = wd.Grid(spec, wd.FP32_METRIC64, wd.C6)
    phi, st = g.solve(cyl_params(wd, 1e-6))
    torch.cuda.synchronize()
    assert st["converged"], st
    a = to_np(phi).reshape(16, 257, 512)
    errs = []
    for k, m in enumerate(golden["members"]):
        assert abs(m["r_wall"] - members[k].meta["r_wall"]) < 1e-15
        ref = np.asarray(m["d"])[:, None]
        err = float(np.abs(a[k] - ref).max())
        errs.append(err)
        assert err <= 2e-4 * spec.L_ref + m["spread_over_i"], (k, err)
    print("FP32 batch: max |d - d_oracle| per cylinder:", ["%.2e" % e for e in errs])


def test_fp64_plain_cylinder_matches_oracle(wd, golden):
    import torch

    spec = W.cylinder(257, 512, 1.03, r_wall=0.5)
    g = wd.Grid(spec, wd.FP64, wd.C6)
    phi, st = g.solve(cyl_params(wd, 1e-10))
    torch.cuda.synchronize()
    assert st["converged"], st
    m = golden["members"][0]
    err = float(np.abs(to_np(phi).reshape(257, 512) - np.asarray(m["d"])[:, None]).max())
    print("FP64 plain cylinder: max |d - d_oracle| = %.3e" % err)
    assert err <= 1e-6 * spec.L_ref + m["spread_over_i"], err


def _radial_start(spec):
    r = np.hypot(*spec.xyz[:2])
    rr = r.reshape(spec.shape[1], spec.shape[0])
    return (rr - rr[:1, :]).reshape(-1)


ELLIPSES = {"ellipse513x1024": (513, 1024, 1.7), "ellipse1025x2048": (1025, 2048, 3.1)}
_oracle_cache = {}


def _ellipse_reference(oracle, name):
    """oracle: 3 HJ pseudo steps from a distance-like start and 2 Poisson steps from zero
    (C6 + LAD, alpha_f 0.49: the serving stream's parameters)"""
    if name not in _oracle_cache:
        nr, nt, ar = ELLIPSES[name]
        spec = W.ellipse(nr, nt, ar)
        og = oracle.Grid(spec.shape, spec.xyz, spec.bc_lo, spec.bc_hi, scheme=oracle.C6, period=spec.period)
        r = _radial_start(spec)
        phi0 = og.apply_bc(r + 0.05 * np.minimum(r, 1.0) * W.random_field(spec, 4))
        kw = dict(equation=1, scheme=4, alpha_f=0.49, cfl=0.6)
        ref, ost = og.hj_steps(phi0, 3, **kw)
        refp, _ = og.poisson_steps(np.zeros(spec.N), 2, **kw)
        _oracle_cache[name] = (spec, phi0, ref, ost, refp)
    return _oracle_cache[name]


@pytest.mark.parametrize("name", list(ELLIPSES))
@pytest.mark.parametrize("prec", [0, 1])
def test_large_ellipse_steps_match_oracle(wd, oracle, name, prec):
    spec, phi0, ref, ost, refp = _ellipse_reference(oracle, name)
    p = wd.default_params(wd.C6, equation=wd.HJ_LAD, alpha_f=0.49)
    g = wd.Grid(spec, prec, wd.C6)
    out, st = g.steps(p, g.as_field(phi0), 3, kind=0)
    outp, _ = g.steps(p, g.as_field(np.zeros(spec.N)), 2, kind=1)
    tol = 1e-10 if prec == 0 else 1e-5
    np.testing.assert_allclose(to_np(out), ref, atol=tol * scale(ref), rtol=0)
    np.testing.assert_allclose(to_np(outp), refp, atol=tol * scale(refp), rtol=0)
    assert st["res_l2"] == pytest.approx(ost["res_l2"], rel=1e-8 if prec == 0 else 1e-2)
    g.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_star_1025_steps_match_oracle(wd, oracle, prec):
    """4 pseudo steps of the 1025^2 star port with the receding-grain parameters (E4 + LAD,
    eps 0.15, alpha_f 0.45, Delta x^4 LAD scale) from the exact signed distance (the port
    solid, Dirichlet values floored at -3h)."""
    sp = W.star(1025)
    if "star" not in _oracle_cache:
        og = oracle.Grid(sp.shape, sp.xyz, sp.bc_lo, sp.bc_hi, scheme=oracle.E4, mask=sp.mask, dval=sp.dval)
        phi0 = og.apply_bc(np.where(sp.mask == 1, sp.dval, sp.meta["signed_distance"]))
        ref, ost = og.hj_steps(phi0, 4, equation=1, scheme=1, eps=0.15, alpha_f=0.45, lad_exp=4.0, cfl=0.8)
        _oracle_cache["star"] = (phi0, ref, ost)
    phi0, ref, ost = _oracle_cache["star"]
    p = wd.default_params(wd.E4, equation=wd.HJ_LAD, eps=0.15, alpha_f=0.45, lad_exp=4.0)
    g = wd.Grid(sp, prec, wd.E4)
    out, st = g.steps(p, g.as_field(phi0), 4, kind=0)
    tol = 1e-10 if prec == 0 else 1e-5
    np.testing.assert_allclose(to_np(out), ref, atol=tol * scale(ref), rtol=0)
    assert st["res_l2"] == pytest.approx(ost["res_l2"], rel=1e-8 if prec == 0 else 1e-2)
    g.close()
