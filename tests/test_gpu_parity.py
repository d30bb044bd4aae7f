"""GPU parity: every step of the method on the GPU (through the C ABI) against the FP64
oracle on identical seeded inputs, at sizes the oracle finishes in seconds that still
span several line chunks, shared-memory tiles and ragged tails.

Tolerances: FP64 operators agree to 1e-11 of the field scale (only summation order and FMA
contraction differ); FP32 operators to 2e-6 of the scale (float rounding of a few dozen
operations, amplified by the filter and derivative weights where noted); FP64 full solves
to 1e-6 L and FP32 full solves to 2e-4 L."""
import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W
from tests.helpers import base_params, gpu_params, oracle_grid, oracle_kw, to_np

pytestmark = pytest.mark.gpu

FP64_OP = 1e-11
FP32_OP = 2e-6


@pytest.fixture(scope="module")
def wd():
    import torch

    assert torch.cuda.is_available()
    from paper_2111_09859_gb300 import build, wd as _wd

    build.build()
    return _wd


def exact_of(spec):
    x = spec.xyz
    if spec.name == "square":
        return np.minimum.reduce([x[0], 1 - x[0], x[1], 1 - x[1]])
    if spec.name in ("cylinder",):
        return np.hypot(x[0], x[1]) - spec.meta.get("r_wall", 0.5)
    if spec.name == "duct":
        return np.minimum.reduce([x[1], 1 - x[1], x[2], 1 - x[2]])
    if spec.name == "plate":
        return x[1].copy()
    if spec.name == "channel":
        return np.minimum(x[1], 1 - x[1])
    if spec.name == "ellipse":
        return None
    raise KeyError(spec.name)


GRIDS = {
    "square33": lambda: W.square(33),
    "cyl33x64": lambda: W.cylinder(33, 64, 1.03 ** 8),
    "duct12x8": lambda: W.duct(12, nx=8),
    "plate": lambda: W.plate(16, 40, height=2.0, stretch=1.05),
    "ellipse": lambda: W.ellipse(33, 64, 2.5),
    "square71": lambda: W.square(71),
}


def scale(a):
    return max(1.0, float(np.abs(a).max()))


@pytest.mark.parametrize("gname", ["square33", "cyl33x64", "duct12x8", "plate", "ellipse"])
@pytest.mark.parametrize("scheme", [1, 2, 4])
def test_metrics(wd, oracle, gname, scheme):
    spec = GRIDS[gname]()
    og = oracle_grid(oracle, spec, scheme)
    g = wd.Grid(spec, wd.FP64, scheme)
    xi, J, dx = [to_np(t) for t in g.metrics()]
    oxi, oJ, odx = og.metrics()
    for l in range(spec.ndim):
        for m in range(spec.ndim):
            np.testing.assert_allclose(xi[l, m], oxi[l, m], atol=FP64_OP * scale(oxi[l, m]), rtol=0)
        np.testing.assert_allclose(dx[l], odx[l], atol=FP64_OP * scale(odx[l]), rtol=0)
    np.testing.assert_allclose(J, oJ, atol=FP64_OP * scale(oJ), rtol=0)


@pytest.mark.parametrize("gname", ["square71", "cyl33x64", "duct12x8", "ellipse"])
@pytest.mark.parametrize("scheme", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("prec", [0, 2])
def test_derivative(wd, oracle, gname, scheme, prec):
    spec = GRIDS[gname]()
    og = oracle_grid(oracle, spec, scheme)
    g = wd.Grid(spec, prec, scheme)
    f = W.random_field(spec, 3) + 0.1 * W.random_field(spec, 4, smooth=False)
    tol = FP64_OP if prec == 0 else FP32_OP
    for d in range(spec.ndim):
        ref = og.deriv(f, d, scheme)
        out = to_np(g.derivative(g.as_field(f), d))
        np.testing.assert_allclose(out, ref, atol=tol * scale(ref) * 10, rtol=0)


@pytest.mark.parametrize("gname", ["square71", "cyl33x64", "duct12x8"])
@pytest.mark.parametrize("alpha", [0.3, 0.49, 0.495])
@pytest.mark.parametrize("prec", [0, 2])
def test_filter(wd, oracle, gname, alpha, prec):
    spec = GRIDS[gname]()
    og = oracle_grid(oracle, spec, 1)
    g = wd.Grid(spec, prec, 1)
    f = W.random_field(spec, 5) + 0.3 * W.random_field(spec, 6, smooth=False)
    tol = FP64_OP if prec == 0 else FP32_OP * 20    # alpha -> 1/2 amplifies float rounding
    for d in range(spec.ndim):
        ref = og.filter(f, d, alpha)
        out = to_np(g.filter(g.as_field(f), d, alpha))
        np.testing.assert_allclose(out, ref, atol=tol * scale(ref), rtol=0)


RHS_CASES = [
    ("square33", 1, dict(equation=0)),
    ("square33", 1, dict(equation=1)),
    ("square71", 2, dict(equation=1)),
    ("cyl33x64", 4, dict(equation=1, curvature=1, alpha_f=0.495)),
    ("cyl33x64", 4, dict(equation=0, curvature=1)),
    ("duct12x8", 2, dict(equation=1)),
    ("ellipse", 4, dict(equation=1)),
    ("plate", 4, dict(equation=2)),
]


@pytest.mark.parametrize("case", range(len(RHS_CASES)))
@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("kind", [0, 1])
def test_rhs(wd, oracle, case, prec, kind):
    gname, scheme, kw = RHS_CASES[case]
    spec = GRIDS[gname]()
    prm = base_params(scheme, **kw)
    og = oracle_grid(oracle, spec, scheme)
    g = wd.Grid(spec, prec, scheme)
    ex = exact_of(spec)
    if ex is None:
        ex = np.hypot(*spec.xyz) - 0.5
    phi = og.apply_bc(ex + 0.02 * W.random_field(spec, 7))
    okw = oracle_kw(scheme, prm)
    if kind == 0:
        R0, dt0 = og.rhs_hj(phi, **okw)
    else:
        R0, dt0 = og.rhs_poisson(phi, **okw)
    R, dt = g.rhs(gpu_params(wd, scheme, prm), g.as_field(phi), kind)
    tol = FP64_OP * 100 if prec == 0 else 1e-4
    if prec == 2 and gname in ("cyl33x64", "ellipse"):
        # WD_FP32 differentiates FP32-rounded coordinates: rounding 2^-24 |x| against the
        # wall spacing (~1.3e-3 at r = 0.5 on this grid), times the stencil weights (~10),
        # gives ~2e-4 relative metric error near the wall, amplified once more by D(D)
        tol = 2e-3
    np.testing.assert_allclose(to_np(R), R0, atol=tol * scale(R0), rtol=0)
    np.testing.assert_allclose(to_np(dt), dt0, atol=tol * scale(dt0), rtol=tol)


@pytest.mark.parametrize("gname", ["square33", "cyl33x64", "duct12x8", "plate"])
@pytest.mark.parametrize("prec", [0, 2])
def test_spalding_and_bc(wd, oracle, gname, prec):
    spec = GRIDS[gname]()
    scheme = 4 if gname == "cyl33x64" else 1
    og = oracle_grid(oracle, spec, scheme)
    g = wd.Grid(spec, prec, scheme)
    phip = 0.1 + 0.05 * W.random_field(spec, 8) ** 2
    ref = og.spalding(phip, scheme=scheme)
    out = to_np(g.spalding(g.as_field(phip)))
    # float: the one-sided wall derivative of phi' (weights summing to 128/12 in absolute
    # value) times |grad eta| ~ 1/dr0 turns the float rounding of phi' ~ 0.1 into ~5e-5 of
    # |grad phi'| on the stretched O-grid's wall row; Eq. 4 passes it on at the same size
    tol = FP64_OP * 10 if prec == 0 else 2e-4
    np.testing.assert_allclose(out, ref, atol=tol * scale(ref), rtol=0)
    junk = W.random_field(spec, 9)
    ref = og.apply_bc(junk)
    out = to_np(g.apply_bc(g.as_field(junk)))
    np.testing.assert_allclose(out, ref, atol=tol * scale(ref) * 10, rtol=0)


STEP_CASES = [
    ("square33", 1, dict(equation=0)),
    ("square33", 1, dict(equation=1)),
    ("cyl33x64", 4, dict(equation=1, curvature=1, alpha_f=0.495)),
    ("duct12x8", 2, dict(equation=1)),
    ("ellipse", 4, dict(equation=1)),
    ("plate", 4, dict(equation=1)),
]


@pytest.mark.parametrize("case", range(len(STEP_CASES)))
@pytest.mark.parametrize("prec", [0, 1])
def test_pseudo_steps(wd, oracle, case, prec):
    gname, scheme, kw = STEP_CASES[case]
    spec = GRIDS[gname]()
    prm = base_params(scheme, **kw)
    og = oracle_grid(oracle, spec, scheme)
    g = wd.Grid(spec, prec, scheme)
    ex = exact_of(spec)
    if ex is None:
        ex = np.hypot(*spec.xyz) - 0.5
    phi0 = og.apply_bc(ex + 0.02 * W.random_field(spec, 11))
    ref, ost = og.hj_steps(phi0, 4, **oracle_kw(scheme, prm))
    out, st = g.steps(gpu_params(wd, scheme, prm), g.as_field(phi0), 4, kind=0)
    tol = 1e-10 if prec == 0 else 1e-5
    np.testing.assert_allclose(to_np(out), ref, atol=tol * scale(ref), rtol=0)
    assert abs(st["res_l2"] - ost["res_l2"]) <= (1e-8 if prec == 0 else 1e-2) * ost["res_l2"] + 1e-12
    # Poisson pseudo steps from zero
    refp, _ = og.poisson_steps(np.zeros(spec.N), 20, **oracle_kw(scheme, prm))
    outp, _ = g.steps(gpu_params(wd, scheme, prm), g.as_field(np.zeros(spec.N)), 20, kind=1)
    np.testing.assert_allclose(to_np(outp), refp, atol=tol * scale(refp), rtol=0)


SOLVE_CASES = [
    # name, spec, scheme, params, precision, tolerance (x L)
    ("square65-E4-std-fp64", lambda: W.square(65), 1, dict(equation=0), 0, 1e-6),
    ("square65-E4-lad-fp32", lambda: W.square(65), 1, dict(equation=1, tol_l2=1e-7), 2, 2e-4),
    ("cyl-C6-lad-curv-fp64", lambda: W.cylinder(49, 96, 1.03 ** (256 / 48)), 4,
     dict(equation=1, curvature=1, alpha_f=0.495), 0, 1e-6),
    ("cyl-C6-lad-curv-fp32m64", lambda: W.cylinder(49, 96, 1.03 ** (256 / 48)), 4,
     dict(equation=1, curvature=1, alpha_f=0.495, tol_l2=1e-7), 1, 2e-4),
    ("duct-E6-lad-fp32", lambda: W.duct(24, nx=8), 2, dict(equation=1, tol_l2=1e-7), 2, 2e-4),
    ("ellipse-C6-lad-fp32", lambda: W.ellipse(33, 64, 3.0), 4, dict(equation=1, tol_l2=1e-7), 2, 2e-4),
]


@pytest.mark.parametrize("case", range(len(SOLVE_CASES)), ids=[c[0] for c in SOLVE_CASES])
def test_full_solve(wd, oracle, case):
    name, mk, scheme, kw, prec, tol = SOLVE_CASES[case]
    spec = mk()
    prm = base_params(scheme, **kw)
    og = oracle_grid(oracle, spec, scheme)
    oprm = dict(prm, tol_l2=1e-12)
    ref, ost = og.solve(**oracle_kw(scheme, oprm))
    assert ost["converged"], ost
    g = wd.Grid(spec, prec, scheme)
    out, st = g.solve(gpu_params(wd, scheme, prm))
    assert st["converged"], st
    err = np.abs(to_np(out) - ref).max()
    assert err <= tol * spec.L_ref, (name, err, st, ost)


GENERIC_CASES = [0, 2, 4, 5]   # 2-D cases of STEP_CASES


@pytest.mark.parametrize("case", GENERIC_CASES)
def test_pseudo_steps_generic_path(wd, oracle, case, monkeypatch):
    """2-D grids normally take the fused pseudo step; WD_FORCE_GENERIC=1 at grid creation
    selects the generic kernel sequence, which must agree with the oracle as well."""
    monkeypatch.setenv("WD_FORCE_GENERIC", "1")
    gname, scheme, kw = STEP_CASES[case]
    spec = GRIDS[gname]()
    prm = base_params(scheme, **kw)
    og = oracle_grid(oracle, spec, scheme)
    g = wd.Grid(spec, 0, scheme)
    ex = exact_of(spec)
    if ex is None:
        ex = np.hypot(*spec.xyz) - 0.5
    phi0 = og.apply_bc(ex + 0.02 * W.random_field(spec, 11))
    ref, _ = og.hj_steps(phi0, 4, **oracle_kw(scheme, prm))
    out, _ = g.steps(gpu_params(wd, scheme, prm), g.as_field(phi0), 4, kind=0)
    np.testing.assert_allclose(to_np(out), ref, atol=1e-10 * scale(ref), rtol=0)


def _cyl_batch(radii, nr=33, nt=64):
    return [W.cylinder(nr, nt, 1.03 ** (256 / (nr - 1)), r_wall=r) for r in radii]


@pytest.mark.parametrize("prec", [0, 1])
def test_stacked_grids_match_single_grids(wd, oracle, prec):
    """Stacked 2-D grids (n[2] = batch) run the same launches for every member: K pseudo
    steps of the stack equal K steps of each grid alone, bit for bit, and the oracle."""
    import torch

    members = _cyl_batch([0.5, 0.45, 0.55])
    spec = W.stack(members)
    prm = base_params(4, equation=1, curvature=1, alpha_f=0.495)
    gb = wd.Grid(spec, prec, 4)
    exact = [np.hypot(*m.xyz) - m.meta["r_wall"] for m in members]
    phi0 = np.concatenate([oracle_grid(oracle, m, 4).apply_bc(e + 0.02 * W.random_field(m, 3))
                           for m, e in zip(members, exact)])
    outb, stb = gb.steps(gpu_params(wd, 4, prm), gb.as_field(phi0), 4)
    outb = to_np(outb)
    N = members[0].N
    worst = 0.0
    for k, m in enumerate(members):
        g = wd.Grid(m, prec, 4)
        out, st = g.steps(gpu_params(wd, 4, prm), g.as_field(phi0[k * N:(k + 1) * N]), 4)
        np.testing.assert_array_equal(outb[k * N:(k + 1) * N], to_np(out))
        worst = max(worst, st["res_l2"])
        ref, _ = oracle_grid(oracle, m, 4).hj_steps(phi0[k * N:(k + 1) * N], 4, **oracle_kw(4, prm))
        tol = 1e-10 if prec == 0 else 1e-5
        np.testing.assert_allclose(outb[k * N:(k + 1) * N], ref, atol=tol * scale(ref), rtol=0)
    assert stb["res_l2"] == pytest.approx(worst, rel=1e-12)


def test_stacked_solve_against_oracle(wd, oracle):
    members = _cyl_batch([0.5, 0.4])
    spec = W.stack(members)
    prm = base_params(4, equation=1, curvature=1, alpha_f=0.495, tol_l2=1e-7)
    gb = wd.Grid(spec, wd.FP32_METRIC64, 4)
    out, st = gb.solve(gpu_params(wd, 4, prm))
    assert st["converged"], st
    out = to_np(out)
    N = members[0].N
    for k, m in enumerate(members):
        ref, ost = oracle_grid(oracle, m, 4).solve(**oracle_kw(4, dict(prm, tol_l2=1e-12)))
        assert ost["converged"]
        assert np.abs(out[k * N:(k + 1) * N] - ref).max() <= 2e-4


@pytest.mark.parametrize("scheme,eq", [(2, 1), (1, 0), (0, 2)])
@pytest.mark.parametrize("generic", [False, True])
def test_duct_steps_both_paths(wd, oracle, scheme, eq, generic, monkeypatch):
    """Uniform Cartesian 3-D grids take the stencil path (wd_cart3d.cu) unless
    WD_FORCE_GENERIC=1; both agree with the oracle over 4 pseudo steps (and Poisson steps)."""
    if generic:
        monkeypatch.setenv("WD_FORCE_GENERIC", "1")
    spec = W.duct(14, nx=10)
    prm = base_params(scheme, equation=eq)
    og = oracle_grid(oracle, spec, scheme)
    g = wd.Grid(spec, 0, scheme)
    phi0 = og.apply_bc(exact_of(spec) + 0.02 * W.random_field(spec, 21))
    ref, _ = og.hj_steps(phi0, 4, **oracle_kw(scheme, prm))
    out, _ = g.steps(gpu_params(wd, scheme, prm), g.as_field(phi0), 4, kind=0)
    np.testing.assert_allclose(to_np(out), ref, atol=1e-10 * scale(ref), rtol=0)
    refp, _ = og.poisson_steps(np.zeros(spec.N), 10, **oracle_kw(scheme, prm))
    outp, _ = g.steps(gpu_params(wd, scheme, prm), g.as_field(np.zeros(spec.N)), 10, kind=1)
    np.testing.assert_allclose(to_np(outp), refp, atol=1e-10 * scale(refp), rtol=0)


def test_fp64_jacobians_vs_fp32_coordinates(wd, oracle):
    """Precision modes on the stretched cylinder O-grid (257 x 512, ratio 1.03): with
    WD_FP32_METRIC64 the metric Jacobians are computed in FP64 and match the oracle to FP64
    round-off; WD_FP32 differentiates FP32-rounded coordinates, whose rounding (~1e-7 of
    r ~ 10) against the wall spacing 1.5e-4 costs several digits of the metrics."""
    spec = W.cylinder(257, 512, 1.03)
    og = oracle_grid(oracle, spec, 4)
    oxi, _, _ = og.metrics()
    err = {}
    for prec in (1, 2):
        g = wd.Grid(spec, prec, 4)
        xi = to_np(g.metrics()[0])
        err[prec] = max(np.abs(xi[l, m] - oxi[l, m]).max() / scale(oxi[l, m])
                        for l in range(2) for m in range(2))
        g.close()
    print("metric error: FP32_METRIC64 %.2e, FP32 %.2e" % (err[1], err[2]))
    assert err[1] <= 1e-11
    assert err[2] > 100 * err[1] and err[2] <= 1e-2


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("gname,scheme,kw", [
    ("cyl16x257x512", 4, dict(equation=1, curvature=1, alpha_f=0.495)),
    ("ellipse129x256", 4, dict(equation=1)),
    ("channel128x65", 4, dict(equation=0)),
    ("square65", 1, dict(equation=0)),
    ("ellipse1025x2048", 4, dict(equation=1)),
])
def test_partition_passes_match_pcr_passes(wd, monkeypatch, prec, gname, scheme, kw):
    """The fused 2-D step with the warp partition line solves (wd_part2d.cu) against the
    same step with the PCR line solves (WD_PART_OFF=1): the same systems, only the
    elimination order differs (FP64 to round-off, FP32 to a few ulps of the field)."""
    mk = {"cyl16x257x512": lambda: W.stack([W.cylinder(257, 512, 1.03, r_wall=0.5 * (1 + 0.01 * k)) for k in range(4)]),
          "ellipse129x256": lambda: W.ellipse(129, 256, 2.7),
          "channel128x65": lambda: W.channel(128, 65),
          "square65": lambda: W.square(65),
          "ellipse1025x2048": lambda: W.ellipse(1025, 2048, 3.1)}[gname]
    spec = mk()
    p = wd.default_params(scheme, **kw)
    r = np.hypot(*spec.xyz[:2])
    if gname.startswith(("cyl", "ellipse")):
        # O-grids: radial distance from the wall node of each ray (0 on the wall); a field
        # with a jump at the wall overflows within a step on the finest ellipse grid
        rr = r.reshape(-1, spec.shape[1], spec.shape[0])
        r = (rr - rr[:, :1, :]).reshape(-1)
    phi0 = W.random_field(spec, 4) * 0.05 * np.minimum(r, 1.0) + r
    out = {}
    for off in ("0", "1"):
        monkeypatch.setenv("WD_PART_OFF", off)
        g = wd.Grid(spec, prec, scheme)
        r, _ = g.steps(p, g.as_field(phi0), 3, kind=0)
        rp, _ = g.steps(p, g.as_field(phi0), 2, kind=1)
        out[off] = (to_np(r), to_np(rp))
        g.close()
    tol = 1e-11 if prec == 0 else 2e-5
    for a, b in zip(out["0"], out["1"]):
        np.testing.assert_allclose(a, b, atol=tol * scale(b), rtol=0)


@pytest.mark.parametrize("generic", [False, True])
@pytest.mark.parametrize("eq", [0, 1])
def test_cartesian_2d_steps_with_neumann_faces(wd, oracle, generic, eq, monkeypatch):
    """Single uniform 2-D grids whose faces rule out the fused path (the star port with
    zero-gradient box edges and an immersed Dirichlet port) take the Cartesian stencil path
    unless WD_FORCE_GENERIC=1; both agree with the oracle over HJ and Poisson steps."""
    if generic:
        monkeypatch.setenv("WD_FORCE_GENERIC", "1")
    spec = W.star(97)
    prm = base_params(1, equation=eq, lad_exp=4.0, eps=0.15)
    og = oracle_grid(oracle, spec, 1)
    g = wd.Grid(spec, 0, 1)
    phi0 = og.apply_bc(np.where(spec.mask == 1, spec.dval, spec.meta["signed_distance"])
                       + 0.01 * W.random_field(spec, 5))
    ref, _ = og.hj_steps(phi0, 4, **oracle_kw(1, prm))
    out, _ = g.steps(gpu_params(wd, 1, prm), g.as_field(phi0), 4, kind=0)
    np.testing.assert_allclose(to_np(out), ref, atol=1e-10 * scale(ref), rtol=0)
    refp, _ = og.poisson_steps(np.zeros(spec.N), 10, **oracle_kw(1, prm))
    outp, _ = g.steps(gpu_params(wd, 1, prm), g.as_field(np.zeros(spec.N)), 10, kind=1)
    np.testing.assert_allclose(to_np(outp), refp, atol=1e-10 * scale(refp), rtol=0)


@pytest.mark.parametrize("case", ["cylinder", "duct", "star", "stack4"])
def test_autotuned_shapes_do_not_change_results(wd, monkeypatch, case):
    """The autotuner only picks launch shapes and the split of a stacked batch into parts:
    solves with and without it are bit-identical, and the choices are among the candidates."""
    spec, scheme, prec, kw = {
        "cylinder": (W.cylinder(65, 128, 1.1), 4, 1, dict(equation=1, curvature=1)),
        "duct": (W.duct(32, nx=16), 2, 1, dict(equation=1)),
        "star": (W.star(97), 1, 1, dict(equation=1, lad_exp=4.0, eps=0.15)),
        "stack4": (W.stack(_cyl_batch([0.5, 0.45, 0.55, 0.6], nr=65, nt=128)), 4, 1, dict(equation=1, curvature=1)),
    }[case]
    p = wd.default_params(scheme, tol_l2=1e-6, max_iters=400, **kw)
    out = {}
    for tune in ("0", "1"):
        monkeypatch.setenv("WD_AUTOTUNE", tune)
        g = wd.Grid(spec, prec, scheme)
        phi, st = g.solve(p)
        out[tune] = (to_np(phi), st["iters"], g.tuning())
        g.close()
    np.testing.assert_array_equal(out["0"][0], out["1"][0])
    assert out["0"][1] == out["1"][1]
    assert out["0"][2] == (0, 0, 0)
    threads, rows, parts = out["1"][2]
    if case in ("cylinder", "stack4"):
        assert threads in (128, 256, 512)
    else:
        assert rows in (4, 8, 16)
    if case == "stack4":
        assert parts in (1, 2, 4)


def test_batch_parts_are_bit_identical(wd, monkeypatch):
    """A stack of 2-D grids on the line-resident path split into 1, 2 or 4 parts (each part's
    launches on its own stream) gives bit-identical fields, norms and iteration counts."""
    spec = W.stack(_cyl_batch([0.5, 0.45, 0.55, 0.6, 0.52], nr=65, nt=128))
    p = wd.default_params(4, equation=1, curvature=1, tol_l2=1e-6, max_iters=400)
    out = {}
    for parts in ("1", "2", "4"):
        monkeypatch.setenv("WD_BATCH_PARTS", parts)
        g = wd.Grid(spec, wd.FP32_METRIC64, 4)
        phi, st = g.solve(p)
        out[parts] = (to_np(phi), st["iters"], st["res_l2"])
        g.close()
    for k in ("2", "4"):
        np.testing.assert_array_equal(out[k][0], out["1"][0])
        assert out[k][1:] == out["1"][1:]


@pytest.mark.parametrize("scheme,prec,tol", [(1, 0, 1e-6), (4, 0, 1e-6), (1, 1, 2e-4)])
def test_eikonal_full_solve(wd, oracle, scheme, prec, tol):
    """Eikonal (Gamma = 0) full solves of the channel on the fused 2-D path against the
    oracle at the parity bar."""
    spec = W.channel(16, 65)
    prm = base_params(scheme, equation=2)
    og = oracle_grid(oracle, spec, scheme)
    ref, ost = og.solve(**oracle_kw(scheme, prm))
    g = wd.Grid(spec, prec, scheme)
    p = gpu_params(wd, scheme, prm)
    if prec != 0:
        p.tol_l2 = 1e-7
    phi, st = g.solve(p)
    assert st["converged"] == 1
    np.testing.assert_allclose(to_np(phi), ref, atol=tol, rtol=0)
