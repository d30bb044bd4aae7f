"""The 4-wide passes of FP32 uniform Cartesian 3-D grids (wd_cart3d.cu, k_c3_u4 / k_c3_stage4:
4 consecutive x nodes per thread, 16-byte stencil rows) against the FP64 oracle: 4 pseudo
steps (HJ) and 10 Poisson steps at the FP32 step bar (1e-5 of the field scale), and against
the per-node passes (WD_LINE2D_OFF=1) on the same grid at 2e-6 of the scale (the same
formulas; only the compiler's contraction of products into fused multiply-adds may differ),
on grids that exercise the split between 4-wide groups and per-node fallbacks:
  - every explicit scheme (E2 / E4 / E6) and every equation (LAD, standard, eikonal);
  - row lengths that are not multiples of 4 (ragged groups; a periodic row of 10 runs every
    node on the per-node bodies) and a periodic row of 8 (both groups at the wrap, their
    neighbour groups taken from the other end of the row);
  - non-periodic faces in x, y and z (the fallback's closure rows), and periodic z;
and the streamed direction-2 filter with the commit (wd_zfilter.cu) in FP64 and FP32."""
import numpy as np
import pytest

from paper_2111_09859_gb300 import workloads as W
from tests.helpers import base_params, gpu_params, oracle_grid, oracle_kw, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wd():
    import torch

    assert torch.cuda.is_available()
    from paper_2111_09859_gb300 import build, wd as _wd

    build.build()
    return _wd


def scale(a):
    return max(1.0, float(np.abs(a).max()))


def box(shape, per):
    """uniform box, spacing 1/(n_1 - 1) in every direction; periodic directions (per[l] = 1)
    have period n_l h, the others walls at both ends"""
    h = 1.0 / (shape[1] - 1)
    axes = [np.arange(n) * h for n in shape]
    Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    xyz = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)])
    bc = tuple(W.PERIODIC if p else W.WALL for p in per)
    period = tuple(tuple(shape[l] * h if (p and m == l) else 0.0 for m in range(3)) for l, p in enumerate(per))
    return W.GridSpec("box", tuple(shape), xyz, bc, bc, period=period, uniform_h=(h, h, h))


def wall_distance(spec, per):
    d = np.full(spec.N, np.inf)
    for l, p in enumerate(per):
        if not p:
            c = spec.xyz[l]
            d = np.minimum(d, np.minimum(c - c.min(), c.max() - c))
    return d


CASES = {
    # name: (spec, periodic directions, scheme, equation: 0 standard, 1 LAD, 2 eikonal)
    "duct10x14-E2-lad": (lambda: W.duct(14, nx=10), (1, 0, 0), 0, 1),
    "duct10x14-E4-std": (lambda: W.duct(14, nx=10), (1, 0, 0), 1, 0),
    "duct10x14-E6-eik": (lambda: W.duct(14, nx=10), (1, 0, 0), 2, 2),
    "duct8x14-E6-lad": (lambda: W.duct(14, nx=8), (1, 0, 0), 2, 1),
    "duct33x41-E6-lad": (lambda: W.duct(41, nx=33), (1, 0, 0), 2, 1),
    "duct33x41-E2-std": (lambda: W.duct(41, nx=33), (1, 0, 0), 0, 0),
    "duct64x40-E6-lad": (lambda: W.duct(40, nx=64), (1, 0, 0), 2, 1),
    "box40x21x70-perxz-E6-lad": (lambda: box((40, 21, 70), (1, 0, 1)), (1, 0, 1), 2, 1),
    "box37x24x70-pery-E4-lad": (lambda: box((37, 24, 70), (0, 1, 0)), (0, 1, 0), 1, 1),
    "box96x40x24-walls-E6-std": (lambda: box((96, 40, 24), (0, 0, 0)), (0, 0, 0), 2, 0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_cart3d_v4_steps_match_oracle(wd, oracle, monkeypatch, name):
    mk, per, scheme, eq = CASES[name]
    spec = mk()
    prm = base_params(scheme, equation=eq)
    og = oracle_grid(oracle, spec, scheme)
    phi0 = og.apply_bc(wall_distance(spec, per) + 0.02 * W.random_field(spec, 21))
    ref, ost = og.hj_steps(phi0, 4, **oracle_kw(scheme, prm))
    refp, _ = og.poisson_steps(np.zeros(spec.N), 10, **oracle_kw(scheme, prm))
    out = {}
    monkeypatch.setenv("WD_AUTOTUNE", "0")   # default shapes: the streamed direction-2 filter where it applies
    for off in ("0", "1"):
        monkeypatch.setenv("WD_LINE2D_OFF", off)
        g = wd.Grid(spec, wd.FP32, scheme)
        a, st = g.steps(gpu_params(wd, scheme, prm), g.as_field(phi0), 4, kind=0)
        b, _ = g.steps(gpu_params(wd, scheme, prm), g.as_field(np.zeros(spec.N)), 10, kind=1)
        out[off] = (to_np(a), to_np(b), st["res_l2"])
        g.close()
    np.testing.assert_allclose(out["0"][0], ref, atol=1e-5 * scale(ref), rtol=0)
    np.testing.assert_allclose(out["0"][1], refp, atol=1e-5 * scale(refp), rtol=0)
    assert out["0"][2] == pytest.approx(ost["res_l2"], rel=1e-2)
    np.testing.assert_allclose(out["0"][0], out["1"][0], atol=2e-6 * scale(ref), rtol=0)
    np.testing.assert_allclose(out["0"][1], out["1"][1], atol=2e-6 * scale(refp), rtol=0)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("name", ["duct64x40-E6-lad", "box96x40x24-walls-E6-std"])
def test_streamed_z_filter_matches_oracle(wd, oracle, monkeypatch, prec, name):
    """The filter along direction 2 fused with the commit and streamed along z (wd_zfilter.cu:
    a Thomas sweep per column, forward into scratch, backward with the Dirichlet reset, the
    commit and the change norms), which the grids whose rows are a multiple of 32 long take
    by default: 4 pseudo steps and 10 Poisson steps against the oracle at the step bars
    (1e-10 FP64, 1e-5 FP32), and the residual of the last step."""
    mk, per, scheme, eq = CASES[name]
    spec = mk()
    prm = base_params(scheme, equation=eq)
    og = oracle_grid(oracle, spec, scheme)
    phi0 = og.apply_bc(wall_distance(spec, per) + 0.02 * W.random_field(spec, 8))
    ref, ost = og.hj_steps(phi0, 4, **oracle_kw(scheme, prm))
    refp, _ = og.poisson_steps(np.zeros(spec.N), 10, **oracle_kw(scheme, prm))
    monkeypatch.setenv("WD_AUTOTUNE", "0")
    g = wd.Grid(spec, prec, scheme)
    out, st = g.steps(gpu_params(wd, scheme, prm), g.as_field(phi0), 4, kind=0)
    outp, _ = g.steps(gpu_params(wd, scheme, prm), g.as_field(np.zeros(spec.N)), 10, kind=1)
    g.close()
    tol = 1e-10 if prec == 0 else 1e-5
    np.testing.assert_allclose(to_np(out), ref, atol=tol * scale(ref), rtol=0)
    np.testing.assert_allclose(to_np(outp), refp, atol=tol * scale(refp), rtol=0)
    assert st["res_l2"] == pytest.approx(ost["res_l2"], rel=1e-8 if prec == 0 else 1e-2)
