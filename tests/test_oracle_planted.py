"""The oracle's pins against planted mistakes.  Each case compiles a copy of the
oracle with one plausible error (a flipped sign, a dropped term, a wrong
operand), loads it in a child process, and runs the committed pin tests that
should reject it: they must fail.  The unmodified oracle passes the same tests in
the main suite."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dg_oracle.c")
HDR = os.path.join(ROOT, "oracle", "dg_oracle.h")

# name: (exact source text, planted replacement, pin tests that must fail); several
# edits go in as a list of (text, replacement) pairs with None in the second place
PLANTED = {
    # eq:411 lift at the upper element's lower face with the wrong sign
    "lift_sign": ("R[(ep * 5 + v) * nn + qR] + lift0 * (Fs[v] - FR[v]);",
                  "R[(ep * 5 + v) * nn + qR] - lift0 * (Fs[v] - FR[v]);",
                  ["tests/test_oracle_scheme.py::test_discrete_conservation",
                   "tests/test_oracle_scheme.py::test_ne_smooth_wave_exact_and_order"]),
    # eq:HLL dissipation term with the wrong sign
    "hll_dissipation_sign": ("+ (cmin * cmax / den) * (uR[v] - uL[v]);",
                             "- (cmin * cmax / den) * (uR[v] - uL[v]);",
                             ["tests/test_oracle_physics.py::test_llf_equals_hll_for_symmetric_speeds",
                              "tests/test_oracle_scheme.py::test_ne_sod_table_loose"]),
    # con2prim: a term dropped from rho eps = tau - v^2 (E + p - D W/(W + 1))
    "c2p_dropped_term": ("const double rhoeps = tau - v2 * (Ep - D * W / (W + 1.0));",
                         "const double rhoeps = tau - v2 * Ep;",
                         ["tests/test_oracle_physics.py::test_c2p_round_trip_conditioned",
                          "tests/test_oracle_physics.py::test_c2p_matches_independent_z_root"]),
    # LGL weights 2/(N(N+1) P_N(x)^2) with the square dropped
    "lgl_weight_square": ("w[j] = 2.0 / (N * (N + 1.0) * P * P);",
                          "w[j] = 2.0 / (N * (N + 1.0) * P);",
                          ["tests/test_oracle_lgl.py::test_closed_forms",
                           "tests/test_oracle_lgl.py::test_quadrature_exact_to_degree_2N_minus_1"]),
    # eq:MinMod picking the largest positive slope instead of the smallest
    "minmod_max": ("if (a1 > 0.0 && a2 > 0.0 && a3 > 0.0) return fmin(a1, fmin(a2, a3));",
                   "if (a1 > 0.0 && a2 > 0.0 && a3 > 0.0) return fmax(a1, fmax(a2, a3));",
                   ["tests/test_oracle_limiter.py::test_minmod_hand_case",
                    "tests/test_oracle_limiter.py::test_tvd_in_the_means"]),
    # SR characteristic speed without the (1 - c_s^2) factor on v_a
    "sr_speed_factor": ("*lmax = (va * (1.0 - cs2) + root) / den;",
                        "*lmax = (va + root) / den;",
                        ["tests/test_oracle_physics.py::test_sr_speeds_limits"]),
    # SSP-RK3 second-stage weights swapped (3/4 U^n + 1/4 (...) -> 1/4 U^n + 3/4 (...))
    "rk3_weights_swapped": ([("const double ca[3] = {0.0, 0.75, 1.0 / 3.0};", "const double ca[3] = {0.0, 0.25, 1.0 / 3.0};"),
                             ("const double cb[3] = {1.0, 0.25, 2.0 / 3.0};", "const double cb[3] = {1.0, 0.75, 2.0 / 3.0};")],
                            None,
                            ["tests/test_oracle_scheme.py::test_rk3_temporal_order"]),
    # the element slope U_x = 2 c_1 / dx without its factor 2
    "limiter_slope_factor": ("minmodB(2.0 * Se[7 + a] / m->dx[a],", "minmodB(Se[7 + a] / m->dx[a],",
                             ["tests/test_oracle_limiter.py"]),
    # eq:411 volume term with the wrong sign
    "volume_sign": ("acc = acc + (2.0 / m->dx[a]) * s;", "acc = acc - (2.0 / m->dx[a]) * s;",
                    ["tests/test_oracle_scheme.py::test_ne_smooth_wave_exact_and_order"]),
    # limiter summaries: the upper face mean taken one node line inside the element
    "summary_face_index": ("S[2 + 2 * a] = ubar[n - 1];", "S[2 + 2 * a] = ubar[n - 2];",
                           ["tests/test_oracle_limiter.py::test_linear_data_not_limited"]),
    # limiter summaries: the element slope from the P2 instead of the P1 Legendre coefficient (Sec. 3.3.2)
    "summary_p1_row": ("for (int i = 0; i < n; ++i) c1 = c1 + m->Vinv[1 * n + i] * ubar[i];",
                       "for (int i = 0; i < n; ++i) c1 = c1 + m->Vinv[2 * n + i] * ubar[i];",
                       ["tests/test_oracle_limiter.py"]),
    # eq:Roe: the u - c wave weighted by |u + c|
    "roe_wave_speed": ("const double w1 = fabs(un - c) * al1,", "const double w1 = fabs(un + c) * al1,",
                       ["tests/test_oracle_physics.py::test_roe_flux_matches_eigendecomposition"]),
    # the energy flux (tau + p) v_a without its pressure work
    "energy_flux_work": ("F[4] = (u[4] + p) * va;", "F[4] = u[4] * va;",
                         ["tests/test_oracle_physics.py::test_flux_consistency",
                          "tests/test_oracle_sr_riemann.py::test_re_sod_st1_table_loose"]),
    # the momentum flux's pressure on the wrong diagonal entry
    "momentum_flux_pressure": ("F[1 + a] = F[1 + a] + p;", "F[1 + (a + 1) % 3] = F[1 + (a + 1) % 3] + p;",
                               ["tests/test_oracle_physics.py::test_flux_consistency"]),
    # con2prim's Newton derivative f'(p) = 1 - (g-1) v^2 (1 - D W / (E + p)) with the wrong sign
    # inside: the bracket keeps the root, the iteration count gives it away
    "c2p_derivative": ("r.df = 1.0 - (g - 1.0) * v2 * (1.0 - D * W / Ep);",
                       "r.df = 1.0 - (g - 1.0) * v2 * (1.0 + D * W / Ep);",
                       ["tests/test_oracle_physics.py::test_c2p_newton_converges_quadratically"]),
    # CFL: dx_min as the element half-width instead of the smallest LGL node gap (Sec. 3.4)
    "cfl_dxmin": ("double h = 0.5 * m->dx[a] * (m->x[1] - m->x[0]);", "double h = 0.5 * m->dx[a];",
                  ["tests/test_oracle_scheme.py::test_cfl_dt_closed_form",
                   "tests/test_oracle_scheme.py::test_ne_smooth_wave_exact_and_order"]),
    # eq:LLF with alpha from the left state only
    "llf_alpha_one_side": ("double al = fmax(fmax(fabs(lminL), fabs(lmaxL)), fmax(fabs(lminR), fabs(lmaxR)));",
                           "double al = fmax(fabs(lminL), fabs(lmaxL));",
                           ["tests/test_oracle_physics.py::test_numerical_flux_mirror_symmetry"]),
    # prim2con (stable form) with the p (W^2 - 1) term of tau dropped
    "prim2con_dropped_term": ("u[4] = rho * W * (W2v2 / (W + 1.0)) + rhoeps * W * W + p * W2v2;",
                              "u[4] = rho * W * (W2v2 / (W + 1.0)) + rhoeps * W * W;",
                              ["tests/test_oracle_physics.py"]),
    # the differentiation matrix's diagonal with the wrong sign (negative-sum trick)
    "dmat_diagonal_sign": ("D[i * n + i] = -s;", "D[i * n + i] = s;", ["tests/test_oracle_lgl.py"]),
    # MRS bound widening alpha h instead of alpha h^{3/2} (eq:MRSSol, Sec. 3.3.3)
    "mrs_width_exponent": ("const double wid = m->d.mrs_alpha * h * sqrt(h);", "const double wid = m->d.mrs_alpha * h;",
                           ["tests/test_oracle_limiter.py::test_mrs_theta_closed_form_for_an_isolated_bump"]),
    # the fix's momentum bound tau (tau + 2 D) with the factor 2 dropped
    "fix_bound": ("(1.0 - 1e-12) * (*tau * (*tau + 2.0 * *D));", "(1.0 - 1e-12) * (*tau * (*tau + *D));",
                  ["tests/test_oracle_limiter.py::test_fix_bounds"]),
}


@pytest.mark.parametrize("name", sorted(PLANTED))
def test_pins_reject_planted_mistake(name, tmp_path):
    old, new, pins = PLANTED[name]
    edits = old if new is None else [(old, new)]
    with open(SRC) as f:
        src = f.read()
    for o, n in edits:
        assert src.count(o) == 1, "the planted site must exist exactly once"
        src = src.replace(o, n)
    shutil.copy(HDR, tmp_path / "dg_oracle.h")
    (tmp_path / "dg_oracle.c").write_text(src)
    lib = tmp_path / "libdg_oracle_planted.so"
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
                    "-shared", str(tmp_path / "dg_oracle.c"), "-o", str(lib), "-lm"], check=True)
    env = dict(os.environ, DG_ORACLE_LIB=str(lib))
    for pin in pins:
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", pin], cwd=ROOT,
                           env=env, capture_output=True, text=True, timeout=900)
        # pytest exits 1 when tests ran and some failed (not 0, and not a collection error)
        assert r.returncode == 1 and " failed" in r.stdout, (pin, r.returncode, r.stdout[-1500:])
