"""Mutation test of the oracle's pins (no GPU).

Each case copies the oracle's C source, plants one plausible mistake (a
dropped term, a wrong sign, index or coefficient, an off-by-one comparison),
compiles the copy and requires at least one pin to fail on it.  The planted
mistakes live only in temporary copies; the oracle itself is not changed.
"""
import os

import pytest

import oracle_pins as P
from oracle import oracle as O

MUTANTS = {
    "far_g_sign": ("*g = -3.0 / (r2 * r2 * r);", "*g = 3.0 / (r2 * r2 * r);"),
    "inner_f_coeff": ("*f = (32.0 / 3.0 + u2 * (-192.0 / 5.0 + 32.0 * u)) / h3;",
                      "*f = (32.0 / 3.0 + u2 * (-192.0 / 5.0 + 30.0 * u)) / h3;"),
    "outer_g_term": ("*g = (-48.0 / u + 384.0 / 5.0 - 32.0 * u + 1.0 / (5.0 * u5)) / h5;",
                     "*g = (-48.0 / u + 384.0 / 5.0 - 32.0 * u) / h5;"),
    "outer_phi_coeff": ("*phi = (16.0 / 5.0 - 1.0 / (15.0 * u)",
                        "*phi = (16.0 / 5.0 - 1.0 / (5.0 * u)"),
    "self_term_kept": ("if (j == i) continue;\n            double d[3] = {pos[3 * j] - xi,",
                       ";\n            double d[3] = {pos[3 * j] - xi,"),
    "jerk_sign": ("nadd(&jk[c], m * (f * v[c] + g * dv * d[c]));",
                  "nadd(&jk[c], m * (f * v[c] - g * dv * d[c]));"),
    "jerk_dropped_term": ("nadd(&jk[c], m * (f * v[c] + g * dv * d[c]));",
                          "nadd(&jk[c], m * (f * v[c]));"),
    "tidal_index": ("nadd(&tt[4], -m * (g * d[0] * d[2]));", "nadd(&tt[4], -m * (g * d[0] * d[1]));"),
    "tidal_sign": ("nadd(&tt[1], -m * (f + g * d[1] * d[1]));", "nadd(&tt[1], m * (f + g * d[1] * d[1]));"),
    "d_transposed": ("double d[3] = {pos[3 * j] - xi,", "double d[3] = {xi - pos[3 * j],"),
    "vel_index": ("double v[3] = {vel[3 * j] - ui, vel[3 * j + 1] - vi,",
                  "double v[3] = {vel[3 * j] - ui, vel[3 * j + 1] - ui,"),
    "pot_sign": ("nadd(&ph, -m * phi);", "nadd(&ph, m * phi);"),
    "G_dropped": ("jerk[3 * t + c] = G * nval(&jk[c]);", "jerk[3 * t + c] = nval(&jk[c]);"),
    "dt_offdiag_once": ("s = s + 2.0 * (t6[3] * t6[3]);", "s = s + (t6[3] * t6[3]);"),
    "dt_norm_6": ("return sqrt(eta) / sqrt(sqrt(s / 6.0));", "return sqrt(eta) / sqrt(sqrt(s / 3.0));"),
    "due_strict": ("if (elapsed >= need) {", "if (elapsed > need) {"),
    "no_reset": ("            tf_ticks[i] = 0;\n        } else {", "        } else {"),
    "counter_one_tick": ("tf_ticks[i] += (int64_t)1 << (k_max - k);", "tf_ticks[i] += 1;"),
    "active_wrong_step": ("int64_t step = (int64_t)1 << (k_max - k);", "int64_t step = (int64_t)1 << k;"),
    "compact_off_by_one": ("if (flags[i]) idx[c++] = (int32_t)i;", "if (flags[i]) idx[c++] = (int32_t)i + 1;"),
    "predict_half": ("double inc = j_last[3 * i + c] * tau;", "double inc = j_last[3 * i + c] * tau * 0.5;"),
    "predict_due_too": ("        if (due[i]) {\n            for (int c = 0; c < 3; ++c) a_out[3 * i + c] = a_last[3 * i + c];\n            continue;\n        }\n", ""),
    "bin_round_up": ("if (mm > mi) k += 1;", "if (mm >= mi) k += 1;"),
    "bin_no_align": ("if (k < k_align) k = k_align;", ";"),
    "bin_hydro_ignored": ("if (dt_hydro && dt_hydro[i] < dt) dt = dt_hydro[i];", ";"),
    "poly_slope_sign": ("double diff = a_last[3 * i + c] - a_prev[3 * i + c];",
                        "double diff = a_prev[3 * i + c] - a_last[3 * i + c];"),
    "poly_gap_wrong": ("dt_prev[i] = (dt_grav[i] == 0.0) ? 0.0 : (double)elapsed_ticks[i] * dt_min;",
                       "dt_prev[i] = (dt_grav[i] == 0.0) ? 0.0 : (double)(elapsed_ticks[i] + 1) * dt_min;"),
    "elapsed_after_reset": ("            if (elapsed_ticks) elapsed_ticks[i] = tf_ticks[i];\n            tf_ticks[i] = 0;\n",
                            "            tf_ticks[i] = 0;\n            if (elapsed_ticks) elapsed_ticks[i] = tf_ticks[i];\n"),
    "poly_no_log": ("for (int c = 0; c < 3; ++c) a_prev[3 * i + c] = a_last[3 * i + c];", ";"),
    "periodic_floor": ("for (int c = 0; c < 3; ++c) d[c] -= box * nearbyint(d[c] / box);",
                       "for (int c = 0; c < 3; ++c) d[c] -= box * floor(d[c] / box);"),
    "periodic_half_up": ("for (int c = 0; c < 3; ++c) d[c] -= box * nearbyint(d[c] / box);",
                         "for (int c = 0; c < 3; ++c) d[c] -= box * floor(d[c] / box + 0.5);"),
    "periodic_two_axes": ("for (int c = 0; c < 3; ++c) d[c] -= box * nearbyint(d[c] / box);",
                          "for (int c = 0; c < 2; ++c) d[c] -= box * nearbyint(d[c] / box);"),
    "soft_corr_sign": ("fc = -0.5 * (zeta[i] * wri + zeta[j] * wrj) / r;",
                       "fc = 0.5 * (zeta[i] * wri + zeta[j] * wrj) / r;"),
    "soft_corr_drop_source": ("fc = -0.5 * (zeta[i] * wri + zeta[j] * wrj) / r;",
                              "fc = -0.5 * (zeta[i] * wri) / r;"),
    "soft_omega_one": ("double om = 1.0 + h * rho_h / (3.0 * rho);", "double om = 1.0;"),
    "soft_dh_drho": ("if (zeta) zeta[i] = -h * psi_h / (3.0 * rho * om);",
                     "if (zeta) zeta[i] = -h * psi_h / (2.0 * rho * om);"),
    "soft_rho_no_self": ("        nadd(&sr, mass[j] * w);",
                         "        if (j != i) nadd(&sr, mass[j] * w);"),
    "soft_psi_with_self": ("        if (j != i) nadd(&sp, mass[j] * ph);",
                           "        nadd(&sp, mass[j] * ph);"),
    "soft_sums_rho_h_sign": ("        nadd(&srh, mass[j] * wh);", "        nadd(&srh, -mass[j] * wh);"),
    "soft_sums_psi_h_kernel": ("        if (j != i) nadd(&sp, mass[j] * ph);",
                               "        if (j != i) nadd(&sp, mass[j] * wh);"),
    "soft_force_own_h": ("f = 0.5 * (fi + fj);", "f = fi;"),
    "soft_g_own_h": ("g = 0.5 * (gi + gj);", "g = gi;"),
    "soft_pot_own_h": ("phi = 0.5 * (pi_ + pj);", "phi = pi_;"),
    "soft_w_h_term": ("*w_h = -c * (3.0 * wu + u * dwu) / h;", "*w_h = -c * (3.0 * wu - u * dwu) / h;"),
    "soft_psi_h_power": ("*psi_h = -dup / (h * h);", "*psi_h = -dup / h;"),
    "tree_com_unweighted": ("                mx[c] = mx[c] + mj * t->pos[3 * j + c];",
                            "                mx[c] = mx[c] + t->pos[3 * j + c];"),
    "tree_vcom_dropped": ("double v[3] = {nd->vcom[0] - vi[0], nd->vcom[1] - vi[1], nd->vcom[2] - vi[2]};",
                          "double v[3] = {-vi[0], -vi[1], -vi[2]};"),
    "tree_half_side": ("double L = ldexp(t->ext, -nd->level);", "double L = ldexp(t->ext, -nd->level - 1);"),
    "tree_self_in_leaf": ("            if (j == i) continue;\n            double dj[3]", "            double dj[3]"),
    "tree_wrong_digit": ("int shift = 3 * (20 - nd->level);", "int shift = 3 * (21 - nd->level) % 63;"),
    "tree_key_axes": ("kv[i].key = (spread21(q[0]) << 2) | (spread21(q[1]) << 1) | spread21(q[2]);",
                      "kv[i].key = (spread21(q[2]) << 2) | (spread21(q[1]) << 1) | spread21(q[0]);"),
    "tree_rel_power": ("if (accept && rel > 0.0) accept = (G * nd->m) * L2 <= (rel * r2) * r2;",
                       "if (accept && rel > 0.0) accept = (G * nd->m) * L2 <= rel * r2;"),
    "cond_tidal_cross": ("st += m * sqrt(2.0 * f * f + e3 * e3);", "st += m * sqrt(3.0 * f * f + e3 * e3);"),
    "cond_jerk_sign": ("for (int c = 0; c < 3; ++c) jv[c] = f * v[c] + g * dv * d[c];",
                       "for (int c = 0; c < 3; ++c) jv[c] = f * v[c] - g * dv * d[c];"),
    "cond_self_kept": ("            if (j == i) continue;\n            double d[3], v[3];",
                       "            double d[3], v[3];"),
    "adj_mass_sign": ("nadd(&mb, -f * da);", "nadd(&mb, f * da);"),
    "adj_g_term": ("nadd(&xb[c], f * ab[c] + g * d[c] * da);", "nadd(&xb[c], f * ab[c]);"),
    "adj_tidal_transposed": ("ta[0] = t6[0] * ak[0] + t6[3] * ak[1] + t6[4] * ak[2];",
                             "ta[0] = t6[0] * ak[0] + t6[4] * ak[1] + t6[3] * ak[2];"),
    "adj_w_sign": ("px[c] -= w_bar * mass[k] * acc[3 * k + c];", "px[c] += w_bar * mass[k] * acc[3 * k + c];"),
    "adj_pot_dropped": ("pm += w_bar * pot[k];", ";"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(O._SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/present: {name}"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = O.load(O.build(force=True, src=str(path), out=str(tmp_path / "libmutant.so")))
    caught = []
    for pin in P.ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, ValueError, FloatingPointError):
            caught.append(pin.__name__)
            break
    assert caught, f"mutant {name} passed every pin"
