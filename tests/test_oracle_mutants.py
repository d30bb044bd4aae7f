"""Planted mistakes in the oracle: each case copies the oracle's C source, plants one
plausible mistake (a wrong coefficient, a flipped sign, a transposed index, a swapped
operand, a dropped term), builds that copy apart from the real oracle, and runs the pins
that guard the planted line against it: at least one must fail.  This shows that the pins
constrain each part of the oracle they cover.  The oracle itself is never modified, and
the copies live in pytest's temporary directory."""
import importlib.util
import os
import shutil

import pytest

from tests import test_oracle_method as TM
from tests import test_oracle_operators as TO
from tests import test_oracle_rk4 as TR
from tests import test_oracle_star as TS
from tests import test_oracle_upwind as TU

ORACLE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), os.pardir, "oracle")

# (name, line as written in the oracle, the planted mistake, pins that must catch it)
MUTANTS = [
    ("E4 interior coefficient",
     "(2.0 / 3.0) * (F(i + 1) - F(i - 1)) - (1.0 / 12.0) * (F(i + 2) - F(i - 2));",
     "(2.0 / 3.0) * (F(i + 1) - F(i - 1)) - (1.0 / 6.0) * (F(i + 2) - F(i - 2));",
     [(TO.test_deriv_interior_polynomial_order, dict(name="E4"))]),
    ("C6 left coupling",
     "            a[i] = 1.0 / 3.0;\n",
     "            a[i] = 0.3;\n",
     [(TO.test_deriv_periodic_symbol, dict(name="C6"))]),
    ("one-sided boundary row",
     "return (-25.0 * f0 + 48.0 * f1 - 36.0 * f2 + 16.0 * f3 - 3.0 * f4) / 12.0;",
     "return (-25.0 * f0 + 48.0 * f1 - 36.0 * f2 + 16.0 * f3 - 4.0 * f4) / 12.0;",
     [(TO.test_deriv_boundary_rows, {})]),
    ("metric inverse transposed",
     "C->xi[(l * 3 + m) * N + p] = (l < nd && m < nd) ? Mi[l][m] : 0.0;",
     "C->xi[(l * 3 + m) * N + p] = (l < nd && m < nd) ? Mi[m][l] : 0.0;",
     [(TO.test_metrics_uniform_and_affine, {})]),
    ("filter coupling",
     "        a[i] = al;\n        c[i] = al;\n",
     "        a[i] = 0.5 * al;\n        c[i] = al;\n",
     [(TO.test_filter_transfer_function_periodic, {})]),
    ("fourth difference",
     "out[i] = f[m2] - 4.0 * f[m1] + 6.0 * f[c] - 4.0 * f[p1] + f[p2];",
     "out[i] = f[m2] - 4.0 * f[m1] + 5.0 * f[c] - 4.0 * f[p1] + f[p2];",
     [(TM.test_lad_vanishes_on_linear_and_sees_a_kink, {}), (TM.test_lad_closed_form_on_a_quartic, dict(lad_exp=3.0, c=0.2))]),
    ("LAD exponent",
     "lad[p] += q * q * d4[p] * pow(C->dx[(size_t)l * N + p], P->lad_exp);",
     "lad[p] += q * q * d4[p] * pow(C->dx[(size_t)l * N + p], P->lad_exp - 1.0);",
     [(TM.test_lad_closed_form_on_a_quartic, dict(lad_exp=3.0, c=0.2))]),
    ("LAD metric scale",
     "lad[p] += q * q * d4[p] * pow(C->dx[(size_t)l * N + p], P->lad_exp);",
     "lad[p] += q * d4[p] * pow(C->dx[(size_t)l * N + p], P->lad_exp);",
     [(TM.test_lad_closed_form_on_a_quartic, dict(lad_exp=4.0, c=0.2))]),
    ("LAD Gaussian weight",
     "static const double gw[5] = {3565.0 / 10368.0, 3091.0 / 12960.0, 1997.0 / 25920.0,",
     "static const double gw[5] = {3565.0 / 10368.0, 3091.0 / 12961.0, 1997.0 / 25920.0,",
     [(TM.test_lad_gaussian_removes_the_nyquist_mode, {})]),
    ("curvature velocity term",
     "v = 0.001 * (1.0 - gm) * (1.0 - gm);",
     "v = 0.002 * (1.0 - gm) * (1.0 - gm);",
     [(TM.test_rhs_curvature_velocity_term, {})]),
    ("Spalding root",
     "phi[p] = -sqrt(g2) + sqrt(arg > 0.0 ? arg : 0.0);",
     "phi[p] = sqrt(g2) + sqrt(arg > 0.0 ? arg : 0.0);",
     [(TM.test_spalding_channel_exact, dict(scheme=1))]),
    ("curvature correction sign",
     "r = 1.0 + (gam + v) * (lap[p] - corr) - a2;",
     "r = 1.0 + (gam + v) * (lap[p] + corr) - a2;",
     [(TM.test_rhs_circle_curvature_sign, {})]),
    ("standard diffusivity dropped",
     "if (P->equation == OR_HJ_STD) gam = P->eps * phip;",
     "if (P->equation == OR_HJ_STD) gam = 0.0;",
     [(TM.test_rhs_closed_form_quadratic, dict(scheme=1, equation=0))]),
    ("chain rule",
     "for (int l = 0; l < nd; l++) s += C->xi[(l * 3 + m) * N + p] * D[(size_t)l * N + p];",
     "for (int l = 0; l < nd; l++) s += C->xi[(l * 3 + m) * N + p] * D[(size_t)m * N + p];",
     [(TM.test_rhs_closed_form_quadratic, dict(scheme=1, equation=2)),
      (TM.test_rhs_linear_field_on_sheared_grid, dict(scheme=1))]),
    ("Poisson source sign",
     "R[p] = 1.0 + lap[p];",
     "R[p] = 1.0 - lap[p];",
     [(TM.test_poisson_fixed_point_and_convergence, {})]),
    ("local step: diffusive term dropped",
     "dt[p] = P->cfl / (metric_sum1(C, p) * a + (gam + v) * metric_sum2(C, p));",
     "dt[p] = P->cfl / (metric_sum1(C, p) * a);",
     [(TM.test_lad_vanishes_on_linear_and_sees_a_kink, {})]),
    ("Dirichlet values",
     "if (C->dmask[p]) phi[p] = poisson ? 0.0 : C->dval[p];",
     "if (C->dmask[p]) phi[p] = 0.0;",
     [(TM.test_bc_far_field_and_dirichlet, {})]),
    ("far-field extrapolation sign",
     "else phi[p] = phi[p + s] + rat[p] * (phi[p + s] - phi[p + 2 * s]);",
     "else phi[p] = phi[p + s] - rat[p] * (phi[p + s] - phi[p + 2 * s]);",
     [(TM.test_bc_far_field_and_dirichlet, {})]),
    ("change norm over all nodes",
     "*l2 = cnt ? sqrt(ss / cnt) : 0.0;",
     "*l2 = cnt ? sqrt(ss / C->N) : 0.0;",
     [(TM.test_step_norms_match_numpy, {})]),
    ("pseudo-step RK4 weight",
     "phi[p] = p0[p] + dt[p] / 6.0 * (K[0][p] + 2.0 * K[1][p] + 2.0 * K[2][p] + K[3][p]);",
     "phi[p] = p0[p] + dt[p] / 6.0 * (K[0][p] + 2.0 * K[1][p] + K[2][p] + 2.0 * K[3][p]);",
     [(TR.test_pseudo_step_is_classical_rk4, {})]),
    ("cyclic correction sign",
     "for (int i = 0; i < n; i++) x[i] -= f * z[i];",
     "for (int i = 0; i < n; i++) x[i] += f * z[i];",
     [(TO.test_tridiag_matches_dense_solve, dict(cyclic=True))]),
    ("filter coefficient of the 8th-order member",
     "a[2] = (-7.0 + 14.0 * al) / 32.0;",
     "a[2] = (-7.0 + 14.0 * al) / 31.0;",
     [(TO.test_filter_coefficients_solve_their_defining_conditions, dict(hw=4, al=0.49))]),
    ("filter order near an end",
     "            if (e < hw) hw = e;",
     "            if (e < hw) hw = e + 1 < 5 ? e + 1 : 5;",
     [(TO.test_filter_nonperiodic_ends, {})]),
    ("periodic metric shift dropped",
     "for (int p = 0; p < N; p++) A[(m * 3 + l) * N + p] = dtmp[p] + shift / (double)n;",
     "for (int p = 0; p < N; p++) A[(m * 3 + l) * N + p] = dtmp[p];",
     [(TO.test_metrics_periodic_shift, {})]),
    ("spacing with a transposed Jacobian",
     "for (int m = 0; m < nd; m++) s += M[m][l] * M[m][l];",
     "for (int m = 0; m < nd; m++) s += M[l][m] * M[l][m];",
     [(TO.test_metrics_uniform_and_affine, {})]),
    ("far-field spacing ratio inverted",
     "r[p] = dist_nodes(C, p, p1) / dist_nodes(C, p1, p2);",
     "r[p] = dist_nodes(C, p1, p2) / dist_nodes(C, p, p1);",
     [(TM.test_bc_far_field_and_dirichlet, {})]),
    ("time-step metric sum without the square root",
     "        s += sqrt(q);\n    }\n    return s;\n}\n\n/* sum_l sum_k",
     "        s += q;\n    }\n    return s;\n}\n\n/* sum_l sum_k",
     [(TM.test_local_time_step_special_case, {})]),
    ("Gershgorin cross terms dropped",
     "                q += C->xi[(l * 3 + m) * C->N + p] * C->xi[(k * 3 + m) * C->N + p];\n            s += fabs(q);",
     "                q += C->xi[(l * 3 + m) * C->N + p] * C->xi[(k * 3 + m) * C->N + p];\n            s += l == k ? fabs(q) : 0.0;",
     [(TM.test_local_time_step_special_case, {}), (TM.test_local_time_step_sheared_grid, {})]),
    ("level-set selection not mirrored for F < 0",
     "double sg = Fs < 0.0 ? -1.0 : 1.0;",
     "double sg = 1.0;",
     [(TU.test_levelset_negative_speed_shrinks, {})]),
    ("C4 coefficient",
     "d[i] = 1.5 * (f[ip] - f[im]) / 2.0;",
     "d[i] = 1.4 * (f[ip] - f[im]) / 2.0;",
     [(TO.test_deriv_periodic_symbol, dict(name="C4"))]),
    ("LAD cap as a maximum",
     "gam = a < b ? a : b;\n        } else gam = 0.0;",
     "gam = a > b ? a : b;\n        } else gam = 0.0;",
     [(TM.test_lad_closed_form_on_a_quartic, dict(lad_exp=3.0, c=0.2))]),
    ("LAD magnitude without the absolute value",
     "for (int p = 0; p < N; p++) lad[p] = P->C_lad * fabs(lad[p]);",
     "for (int p = 0; p < N; p++) lad[p] = P->C_lad * lad[p];",
     [(TM.test_lad_closed_form_on_a_quartic, dict(lad_exp=3.0, c=-0.2))]),
    ("Poisson far field kept as extrapolation",
     "            if (poisson) bc = OR_BC_NEUMANN;\n",
     "",
     [(TM.test_poisson_fixed_point_and_convergence, {}), (TM.test_poisson_far_field_is_neumann, {})]),
    ("level length: crossing interpolated from the wrong end",
     "t = np.where(h, V[a] / (V[a] - V[b]), 0.0)",
     "t = np.where(h, V[b] / (V[a] - V[b]), 0.0)",
     [(TS.test_level_length_straight_lines_exact, dict(a=1.0, b=-2.0, c=0.25, length=None))]),
    ("recede: floor as a ceiling",
     "dval = np.where(mask == 1, np.maximum(new, floor), 0.0)",
     "dval = np.where(mask == 1, np.minimum(new, floor), 0.0)",
     [(TS.test_recede_definition, {})]),
    ("Thomas forward elimination",
     "double m = b[i] - a[i] * cp[i - 1];",
     "double m = b[i] - c[i] * cp[i - 1];",
     [(TO.test_tridiag_matches_dense_solve, dict(cyclic=False))]),
    ("E6 third-neighbour coefficient",
     "+ (1.0 / 60.0) * (F(i + 3) - F(i - 3));",
     "+ (1.0 / 50.0) * (F(i + 3) - F(i - 3));",
     [(TO.test_deriv_interior_polynomial_order, dict(name="E6"))]),
    ("C6 right-hand side",
     "d[i] = (14.0 / 9.0) * (f[ip] - f[im]) / 2.0 + (1.0 / 9.0) * (f[ip2] - f[im2]) / 4.0;",
     "d[i] = (14.0 / 9.0) * (f[ip] - f[im]) / 2.0 + (1.0 / 9.0) * (f[ip2] - f[im2]) / 2.0;",
     [(TO.test_deriv_periodic_symbol, dict(name="C6"))]),
    ("Jacobian determinant term",
     "- A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])",
     "+ A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])",
     [(TO.test_metrics_uniform_and_affine, {})]),
    ("wall faces not Dirichlet",
     "                    C->dmask[p] = 1;\n                    C->dval[p] = 0.0;",
     "                    C->dval[p] = 0.0;",
     [(TM.test_flat_wall_linear_fixed_point, dict(scheme=1, equation=0, curv=0))]),
    ("upwind slope pairing as printed",
     "return n_im1 * B + n_ip1 * F;",
     "return n_im1 * F + n_ip1 * B;",
     [(TU.test_upwind_slope_is_godunov, {})]),
    ("upwind gradient with transposed metrics",
     "for (int k = 0; k < nd; k++) Um[m] += C->xi[(k * 3 + m) * N + p] * sl[k];",
     "for (int k = 0; k < nd; k++) Um[m] += C->xi[(m * 3 + k) * N + p] * sl[k];",
     [(TU.test_advection_of_linear_field_on_sheared_grid, dict(a=(0.7, 0.2)))]),
    ("upwind halves swapped",
     "a += 0.5 * (uh + fabs(uh)) * B[(size_t)l * N + p] + 0.5 * (uh - fabs(uh)) * F[(size_t)l * N + p];",
     "a += 0.5 * (uh + fabs(uh)) * F[(size_t)l * N + p] + 0.5 * (uh - fabs(uh)) * B[(size_t)l * N + p];",
     [(TU.test_advection_of_monotone_field_is_first_order_upwind, {})]),
    ("level-set speed sign",
     "K[k][p] = -Fs * gm[p];",
     "K[k][p] = Fs * gm[p];",
     [(TU.test_levelset_planar_front_speed, {})]),
    ("level-set RK4 stage from the wrong predecessor",
     "for (int p = 0; p < N; p++) s[p] = p0[p] + cst[k] * dt * K[k - 1][p];",
     "for (int p = 0; p < N; p++) s[p] = p0[p] + cst[k] * dt * K[0][p];",
     [(TR.test_levelset_step_is_classical_rk4, {})]),
    ("level-set faces not held",
     "                if (on_face(g, p, d, side)) phi[p] = phi[p + s];",
     "                if (on_face(g, p, d, side)) phi[p] = phi[p];",
     [(TU.test_levelset_planar_front_speed, {})]),
]


def _mutant(tmp_path, line, planted):
    """A copy of the oracle (C source, header and the Python wrapper) in tmp_path with the
    mistake planted in whichever file holds the line, loaded as a separate module."""
    target = None
    for f in ("wd_oracle.c", "__init__.py"):
        src = open(os.path.join(ORACLE_DIR, f)).read()
        if line in src:
            assert src.count(line) == 1 and target is None, f"the planting site must occur once: {line!r}"
            target = f
            src = src.replace(line, planted)
        (tmp_path / f).write_text(src)
    assert target, f"planting site not found: {line!r}"
    shutil.copy(os.path.join(ORACLE_DIR, "wd_oracle.h"), tmp_path / "wd_oracle.h")
    spec = importlib.util.spec_from_file_location("oracle_mutant", str(tmp_path / "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._lib = None
    mod.build(force=True)
    return mod


@pytest.mark.parametrize("name,line,planted,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, oracle, name, line, planted, pins):
    # the pins pass on the real oracle
    for fn, kw in pins:
        fn(oracle, **kw)
    mod = _mutant(tmp_path, line, planted)
    caught = []
    for fn, kw in pins:
        try:
            fn(mod, **kw)
        except (AssertionError, ValueError, FloatingPointError):
            caught.append(fn.__name__)
    assert caught, f"no pin caught the planted mistake '{name}'"
