"""The oracle's pins must fail when a plausible mistake is planted in the oracle.

Each case below plants one mistake (a dropped term, a wrong sign, index or weight)
in a copy of ``oracle/ffo.c``, compiles the copy into a temporary directory, and
runs the oracle pin suite against it in a subprocess (``FFO_LIB`` points the
wrapper at the broken build).  The suite has to fail for every case.  The real
source is never modified.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ffo.c")

MUTANTS = {
    "rk4_weight_k2": ("x[i] + (h / 6.0) * (k1[i] + 2.0 * k2[i]", "x[i] + (h / 6.0) * (k1[i] + 1.0 * k2[i]"),
    "rk4_stage4_point": ("xs[i] = x[i] + h * k3[i]", "xs[i] = x[i] + (h / 2.0) * k3[i]"),
    "euler_sign": ("x[i] = x[i] + h * k[i];", "x[i] = x[i] - h * k[i];"),
    "lorenz_y_sign": ("dx[1] = x[0] * (r - x[2]) - x[1];", "dx[1] = x[0] * (r - x[2]) + x[1];"),
    "lorenz_z_index": ("dx[2] = x[0] * x[1] - beta * x[2];", "dx[2] = x[0] * x[1] - beta * x[1];"),
    "lorenz_x_swap": ("dx[0] = sigma * (x[1] - x[0]);", "dx[0] = sigma * (x[0] - x[1]);"),
    "wc_inhibition_sign": ("double aE = wEE * E - wEI * I + P;", "double aE = wEE * E + wEI * I + P;"),
    "wc_swapped_inputs": ("double aI = wIE * E - wII * I + Q;", "double aI = wIE * I - wII * E + Q;"),
    "wc_gain_dropped": ("return 1.0 / (1.0 + exp(-gain * (a - thresh)));",
                        "return 1.0 / (1.0 + exp(-(a - thresh)));"),
    "wc_tau_swapped": ("dx[1] = (-I + wc_sigmoid(aI, gain, th)) / tauI;",
                       "dx[1] = (-I + wc_sigmoid(aI, gain, th)) / tauE;"),
    "hh_ring_not_all_to_all": ("if (j != i) s_others += x[5 * j + 4];\n        double I_L",
                               "if (j == (i + 2) % 3) s_others += x[5 * j + 4];\n        double I_L"),
    "hh_beta_m_scale": ("return 4.0 * exp(-(V + 65.0) / 18.0);", "return 4.0 * exp(-(V + 65.0) / 20.0);"),
    "hh_n_power": ("double I_K = gK * (n * n * n * n) * (EK - V);", "double I_K = gK * (n * n * n) * (EK - V);"),
    "hh_tau_swap": ("di[4] = act * (1.0 - s) / tau_r - s / tau_d;", "di[4] = act * (1.0 - s) / tau_d - s / tau_r;"),
    "hh_drive_index": ("di[0] = (I_L + I_Na + I_K + I_syn + p[9 + i]) / C;",
                       "di[0] = (I_L + I_Na + I_K + I_syn + p[9]) / C;"),
    "hh_vtrap_sign": ("return v / (-expm1(-v / 10.0));", "return v / (-expm1(v / 10.0));"),
    "hh_vtrap_limit": ("if (v == 0.0) return 10.0;", "if (v == 0.0) return 1.0;"),
    "hh_alpha_h_shift": ("return 0.07 * exp(-(V + 65.0) / 20.0);", "return 0.07 * exp(-(V + 60.0) / 20.0);"),
    "rng_counter_offset": ("uint64_t z = seed + n * 0x9E3779B97F4A7C15ULL;",
                           "uint64_t z = seed + (n + 1) * 0x9E3779B97F4A7C15ULL;"),
    "rng_draw_order": ("(uint64_t)j * (uint64_t)dim + (uint64_t)k + 1u",
                       "(uint64_t)k * (uint64_t)count + (uint64_t)j + 1u"),
    "seed_bits": ("double u = (double)(r >> 40) * (1.0 / 16777216.0);",
                  "double u = (double)(r >> 41) * (1.0 / 8388608.0);"),
    "linspace_denominator": ("(double)i / (double)(P - 1)", "(double)i / (double)(P)"),
    "pixel_round_half": ("float q = d * scale_f;", "float q = d * scale_f + 0.5f;"),
    "behind_camera_kept": ("if (!(cl[3] > 0.0f)) continue;\n        float nx = cl[0] / cl[3];\n        float ny = cl[1] / cl[3];\n        float c =",
                           "if (!(cl[3] != 0.0f)) continue;\n        float nx = cl[0] / cl[3];\n        float ny = cl[1] / cl[3];\n        float c ="),
    "mvp_row_major": ("Hf = (float)H;\n    for (int64_t i = 0; i < P; ++i) {\n        if (include && !include[i]) continue;\n        float cl[4];\n        for (int j = 0; j < 4; ++j) {\n            float a = m[0 + j] * x[i];",
                      "Hf = (float)H;\n    for (int64_t i = 0; i < P; ++i) {\n        if (include && !include[i]) continue;\n        float cl[4];\n        for (int j = 0; j < 4; ++j) {\n            float a = m[4 * j] * x[i];"),
    "sprite_mvp_row_major": ("inv_r2 = (float)(1.0 / ((double)R * (double)R));\n    for (int64_t i = 0; i < P; ++i) {\n        if (include && !include[i]) continue;\n        float cl[4];\n        for (int j = 0; j < 4; ++j) {\n            float a = m[0 + j] * x[i];",
                             "inv_r2 = (float)(1.0 / ((double)R * (double)R));\n    for (int64_t i = 0; i < P; ++i) {\n        if (include && !include[i]) continue;\n        float cl[4];\n        for (int j = 0; j < 4; ++j) {\n            float a = m[4 * j] * x[i];"),
    "rows_top_down": ("image[(int64_t)r * W + (int64_t)c] += 1u;\n    }\n}\n\n/* Soft-sprite",
                      "image[(int64_t)(H - 1 - (int)r) * W + (int64_t)c] += 1u;\n    }\n}\n\n/* Soft-sprite"),
    "reset_counter_block": ("uint64_t n = ((uint64_t)r * (uint64_t)count[i] + (uint64_t)j[i])",
                            "uint64_t n = ((uint64_t)(r - 1u) * (uint64_t)count[i] + (uint64_t)j[i])"),
    "reset_age_kept": ("            age[i] = 0u;\n            resets[i] = r;", "            resets[i] = r;"),
    "reset_schedule": ("if ((step0 + s + 1) % check_every != 0) continue;", "if ((step0 + s) % check_every != 0) continue;"),
    "reset_bound_strict": ("if (!(xf >= blo[k] && xf <= bhi[k])) out = 1;", "if (!(xf > blo[k] && xf < bhi[k])) out = 1;"),
    "reset_age_limit": ("if (max_age > 0 && age[i] >= max_age) out = 1;", "if (max_age > 0 && age[i] > max_age) out = 1;"),
    "jac_lorenz_sign": ("J[3] = r - x[2]; J[4] = -1.0; J[5] = -x[0];", "J[3] = x[2] - r; J[4] = -1.0; J[5] = -x[0];"),
    "jac_lorenz_param": ("Fp[2 * 3 + 2] = -x[2];", "Fp[2 * 3 + 2] = x[2];"),
    "jac_wc_gain": ("Fp[0 * 10 + 8] = SE * (1.0 - SE) * (aE - th) / tauE;", "Fp[0 * 10 + 8] = SE * (1.0 - SE) * aE / tauE;"),
    "jac_wc_cross": ("J[2] = (dSI * wIE) / tauI;", "J[2] = (dSI * wIE) / tauE;"),
    "jac_hh_leak_dropped": ("J[rV * dim + rV] = (-gL - gNa * m3h - gK * n4 - gsyn * s_others) / C;",
                            "J[rV * dim + rV] = (-gNa * m3h - gK * n4 - gsyn * s_others) / C;"),
    "jac_hh_m_power": ("J[rV * dim + rm] = 3.0 * gNa * m * m * h * (ENa - V) / C;",
                       "J[rV * dim + rm] = 3.0 * gNa * m * m * m * (ENa - V) / C;"),
    "jac_hh_syn_self": ("if (j != i) J[rV * dim + 5 * j + 4]", "if (j != (i + 1) % 3) J[rV * dim + 5 * j + 4]"),
    "jac_hh_C_sign": ("Fp[rV * np + 0] = -Itot / (C * C);", "Fp[rV * np + 0] = Itot / (C * C);"),
    "jac_hh_drive_index": ("Fp[rV * np + 9 + i] = 1.0 / C;", "Fp[rV * np + 9] = 1.0 / C;"),
    "jac_hh_beta_h_deriv": ("dbh = bh * (1.0 - bh) / 10.0;", "dbh = -bh * (1.0 - bh) / 10.0;"),
    "jac_hh_gate_diag": ("J[rn * dim + rn] = -(an + bn);", "J[rn * dim + rn] = -(an - bn);"),
    "jac_hh_theta_sign": ("Fp[rs * np + 15] = -sig * a1 * (1.0 - s) / tau_r;",
                          "Fp[rs * np + 15] = sig * a1 * (1.0 - s) / tau_r;"),
    "jac_hh_vtrap_series": ("return 0.5 + x * (1.0 / 6.0 + x2", "return 0.5 + x * (1.0 / 3.0 + x2"),
    "jac_hh_vtrap_closed": ("return (1.0 - e * (1.0 + x)) / (d * d);", "return (1.0 - e * (1.0 - x)) / (d * d);"),
    "sprite_falloff_linear": ("double a = (1.0 - (double)q) * (1.0 - (double)q);", "double a = (1.0 - (double)q);"),
    "sprite_pixel_corner": ("float dx = ((float)col + 0.5f) - pc;", "float dx = (float)col - pc;"),
    "sprite_radius_not_squared": ("(hi_v - lo_v));\n    float inv_r2 = (float)(1.0 / ((double)R * (double)R));",
                                  "(hi_v - lo_v));\n    float inv_r2 = (float)(1.0 / (double)R);"),
    "sprite_rim_inclusive": ("if (!(q < 1.0f)) continue;\n            double a", "if (!(q <= 1.0f)) continue;\n            double a"),
    "sprite_rows_top_down": ("int64_t at = ((int64_t)row * W + col) * 4;", "int64_t at = ((int64_t)(H - 1 - row) * W + col) * 4;"),
    "sprite_one_colour": ("colour + 4 * group[i]);\n    }\n}\n\n/* 3D soft", "colour);\n    }\n}\n\n/* 3D soft"),
    "sprite_channel": ("double c = gain * a * colour[k];", "double c = gain * a * colour[0];"),
    "sprite_3d_offset": ("float pc = (nx - -1.0f) * su;", "float pc = nx * su;"),
    "sprite_3d_behind": ("if (!(cl[3] > 0.0f)) continue;\n        float nx = cl[0] / cl[3];\n        float ny = cl[1] / cl[3];\n        float pc",
                         "if (!(cl[3] != 0.0f)) continue;\n        float nx = cl[0] / cl[3];\n        float ny = cl[1] / cl[3];\n        float pc"),
    "tangent_no_forcing": ("double s = Fp[i * np + q];", "double s = 0.0;"),
    "tangent_stage": ("for (int a = 0; a < n; ++a) ys[a] = y[a] + hh * k3[a];", "for (int a = 0; a < n; ++a) ys[a] = y[a] + hh * k2[a];"),
    "tangent_euler_step": ("for (int a = 0; a < n; ++a) y[a] = y[a] + hh * k1[a];", "for (int a = 0; a < n; ++a) y[a] = y[a] + (hh / 2.0) * k1[a];"),
    "escape_threshold": ("if (!(fabs(v) <= 1e30)) esc = 1;", "if (!(fabs(v) < 1e38)) esc = 1;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found or not unique"
    mutated = src.replace(old, new, 1)
    csrc = tmp_path / "ffo_mut.c"
    csrc.write_text(mutated)
    lib = tmp_path / "libffo_mut.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(lib),
                    str(csrc), "-lm"], check=True)
    env = dict(os.environ, FFO_LIB=str(lib))
    tests = sorted(os.path.join(ROOT, "tests", f) for f in os.listdir(os.path.join(ROOT, "tests"))
                   if f.startswith("test_oracle_") and f != "test_oracle_mutants.py")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *tests],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the oracle pins"
