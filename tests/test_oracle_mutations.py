"""Mutation check of the oracle's pins: each case plants one plausible
mistake (a dropped term, a wrong sign, coefficient or operand) in a copy of
the oracle source, rebuilds it on the CPU and runs the pin that should catch
it; the pin must fail. This shows the pins constrain every part of the
oracle rather than only re-deriving it."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "srhd_oracle.cpp")

MUTANTS = [
    ("tm_eos_coefficient", "return R(2.5) * T + a / (R(1.0) + sqrt(a + R(1.0)));",
     "return R(2.4) * T + a / (R(1.0) + sqrt(a + R(1.0)));",
     "test_oracle_eos.py::test_tm_is_taub_equality"),
    ("inverse_eos_coefficient", "R(18.0) * ht + R(25.0));\n  return num / den;",
     "R(16.0) * ht + R(25.0));\n  return num / den;",
     "test_oracle_eos.py::test_tm_T_htilde_round_trip"),
    ("sound_speed_term", "((R(5.0) * h - R(8.0) * T) / (h - T))",
     "((R(5.0) * h - R(7.0) * T) / (h - T))",
     "test_oracle_eos.py::test_sound_speed_from_thermodynamics"),
    ("f_dropped_m2", "T * T * hh / (hh + m2);", "T * T * hh / (hh);",
     "test_oracle_eos.py::test_transcendental_relation"),
    ("df_wrong_power", "R(2.0) * h * dT + num / (q * q);", "R(2.0) * h * dT + num / (q);",
     "test_oracle_eos.py::test_derivatives_by_central_differences"),
    ("E_D_operand", "U[4] = D * (s / (R(1.0) + sqrt(R(1.0) + s)));",
     "U[4] = D * (s / (R(1.0) + sqrt(R(1.0) + m2)));",
     "test_oracle_eos.py::test_prim2con_matches_definitions"),
    ("A_sign", "return eD * (eD + R(2.0)) - m2;", "return eD * (eD + R(2.0)) + m2;",
     "test_oracle_eos.py::test_round_trip_error_tracks_conditioning"),
    ("four_velocity_dropped_h", "R ux = U[1] / Dh,", "R ux = U[1] / D,",
     "test_oracle_scheme.py::test_uniform_state_unchanged"),
    ("van_leer_factor", "R vl = R(2.0) * dl * dr / (dl + dr);", "R vl = dl * dr / (dl + dr);",
     "test_oracle_scheme.py::test_limiter_properties"),
    ("energy_flux_dropped_p", ": (U[4] + W[4]) * v;", ": (U[4]) * v;",
     "test_oracle_scheme.py::test_riemann_consistency_and_upwinding"),
    ("pressure_wrong_index", "F[1 + d] = F[1 + d] + W[4];", "F[1] = F[1] + W[4];",
     "test_oracle_scheme.py::test_mirror_symmetry"),
    ("char_speed_transverse", "R b = sqrt(cs2) * sqrt(R(1.0) + up2 * omc);",
     "R b = sqrt(cs2) * sqrt(R(1.0) + u2 * omc);",
     "test_oracle_scheme.py::test_characteristic_speeds"),
    ("hllc_star_energy_sign", "Us[4] = (Uk[4] * a + ps * lam - p * v) / b;",
     "Us[4] = (Uk[4] * a + ps * lam + p * v) / b;",
     "test_oracle_scheme.py::test_riemann_consistency_and_upwinding"),
    ("hll_average_sign", "Uhll[v] = (sR * UR[v] - sL * UL[v] - FR[v] + FL[v]) / ds;",
     "Uhll[v] = (sR * UR[v] - sL * UL[v] - FR[v] - FL[v]) / ds;",
     "test_oracle_scheme.py::test_riemann_consistency_and_upwinding"),
    ("half_step_factor", "R half = R(0.5) * dt / dh;", "R half = dt / dh;",
     "test_oracle_scheme.py::test_shock_tube_converges_to_exact"),
    ("update_sign",
     "            int o = (k * n[1] + j) * n[0] + i;\n            R Un[5];\n"
     "            for (int v = 0; v < 5; ++v) {\n"
     "              Un[v] = in[(size_t)v * nc + c] - coef * div[v];",
     "            int o = (k * n[1] + j) * n[0] + i;\n            R Un[5];\n"
     "            for (int v = 0; v < 5; ++v) {\n"
     "              Un[v] = in[(size_t)v * nc + c] + coef * div[v];",
     "test_oracle_scheme.py::test_periodic_conservation"),
    ("vl_update_sign",
     "            const int o = (k * n[1] + j) * n[0] + i;\n            R Un[5];\n"
     "            for (int v = 0; v < 5; ++v) {\n"
     "              Un[v] = in[(size_t)v * nc + c] - coef * div[v];",
     "            const int o = (k * n[1] + j) * n[0] + i;\n            R Un[5];\n"
     "            for (int v = 0; v < 5; ++v) {\n"
     "              Un[v] = in[(size_t)v * nc + c] + coef * div[v];",
     "test_oracle_vl.py::test_mirror_symmetry_and_periodic_conservation"),
    ("cfl_sound_term", "R umax = gs * su + R(double(ndim)) * gamma * us;",
     "R umax = gs * su + gamma * us;", "test_oracle_scheme.py::test_cfl_limits"),
    ("taub_adiabat_sign", "(hd / rhod + K.h / K.rho) * (K.p - ps);",
     "(hd / rhod - K.h / K.rho) * (K.p - ps);",
     "test_oracle_exact.py::test_exact_table_mixed_limits"),
    ("isentrope_dropped_T", "std::pow(T * (h - T) / (K.T * (K.h - K.T)), 1.5);",
     "std::pow(T * (h) / (K.T * (K.h)), 1.5);",
     "test_oracle_exact.py::test_exact_table_mixed_limits"),
    ("original_scheme_A_sign", "if (ori) return (eD * eD - m2) - R(1.0);",
     "if (ori) return (eD * eD + m2) - R(1.0);",
     "test_oracle_scheme.py::test_original_scheme_round_trip_tracks_its_error_estimate"),
    ("original_scheme_flux_index", "F[4] = ori ? U[1 + d] :", "F[4] = ori ? U[1] :",
     "test_oracle_scheme.py::test_original_scheme_agrees_for_hot_gas_and_conserves"),
    ("retry_factor_compounded_twice",
     "    theta = theta * P.retry_factor;\n    if (theta < P.theta_floor * theta0) theta = 0.0;\n"
     "  }\n  if (retries_out) *retries_out = attempt;\n  if (flux_out) {",
     "    theta = theta * P.retry_factor * P.retry_factor;\n"
     "    if (theta < P.theta_floor * theta0) theta = 0.0;\n"
     "  }\n  if (retries_out) *retries_out = attempt;\n  if (flux_out) {",
     "test_oracle_retry.py::test_retry_count_matches_single_attempt_at_theta_k"),
    ("retry_floor_absolute",
     "    if (theta < P.theta_floor * theta0) theta = 0.0;\n"
     "  }\n  if (retries_out) *retries_out = attempt;\n  if (flux_out) {",
     "    if (theta < P.theta_floor) theta = 0.0;\n"
     "  }\n  if (retries_out) *retries_out = attempt;\n  if (flux_out) {",
     "test_oracle_retry.py::test_floor_gives_piecewise_constant_attempt"),
    ("retry_skips_an_attempt",
     "    ++attempt;\n    theta = theta * P.retry_factor;\n"
     "    if (theta < P.theta_floor * theta0) theta = 0.0;\n"
     "  }\n  if (retries_out) *retries_out = attempt;\n  if (flux_out) {",
     "    ++attempt;\n    theta = theta * P.retry_factor;\n"
     "    if (attempt == 3) theta = theta * P.retry_factor;\n"
     "    if (theta < P.theta_floor * theta0) theta = 0.0;\n"
     "  }\n  if (retries_out) *retries_out = attempt;\n  if (flux_out) {",
     "test_oracle_retry.py::test_retry_count_matches_single_attempt_at_theta_k"),
    ("cold_guess_coefficient", "R a = (R(43.0) * m2 + R(63.0)) / (R(125.0) * P);",
     "R a = (R(43.0) * m2 + R(60.0)) / (R(125.0) * P);",
     "test_oracle_eos.py::test_guess_threshold_is_crossing"),
]


@pytest.mark.parametrize("name,orig,repl,target", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(tmp_path, name, orig, repl, target):
    src = open(SRC).read()
    assert src.count(orig) == 1, f"mutation site not found or ambiguous: {name}"
    mpath = tmp_path / f"mut_{name}.cpp"
    mpath.write_text(src.replace(orig, repl))
    env = dict(os.environ, ORACLE_SRC=str(mpath), ORACLE_LIB=str(tmp_path / f"mut_{name}.so"))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", target)], env=env, capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 1, f"pin {target} did not catch {name}:\n{r.stdout[-2000:]}"
