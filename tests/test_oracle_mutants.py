"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each case copies ``oracle.c``, plants one plausible mistake (a transposed
operand, a dropped term, a wrong index, sign or inclusivity), compiles the
copy into a temporary directory and runs the pins against it: at least one
pin has to fail.  The library is not involved.
"""
import os
import subprocess

import pytest

import oracle
from tests import oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTANTS = {
    "R_transposed": ("(double)R[3 * r] * x[0] + (double)R[3 * r + 1] * x[1] +\n"
                     "               (double)R[3 * r + 2] * x[2]",
                     "(double)R[r] * x[0] + (double)R[r + 3] * x[1] +\n"
                     "               (double)R[r + 6] * x[2]"),
    "t_dropped": (" + (double)vw->t[r];", ";"),
    "fy_for_u": ("double u = (double)vw->fx * qx", "double u = (double)vw->fy * qx"),
    "pixel_index_transposed": ("int64_t pix = (int64_t)iy * vw->W + ix;\n            if (pix_out)",
                               "int64_t pix = (int64_t)ix * vw->H + iy;\n            if (pix_out)"),
    "round_not_floor": ("*ix = (int)floor(u);", "*ix = (int)lround(u);"),
    "closed_frame": ("u < (double)vw->W", "u <= (double)vw->W"),
    "mask_dropped_from_W": ("Wsum += m * w;\n            Zsum += w;\n            if (i < 32)",
                            "Wsum += w;\n            Zsum += w;\n            if (i < 32)"),
    "depth_gate_exclusive": ("if (!(fabs(e) <= Delta)) continue;\n            double r = e / Delta;\n"
                             "            double w = exp(-pr->alpha1 * r * r);\n            Wsum += m * w;"
                             "\n            Zsum += w;\n            if (i < 32)",
                             "if (!(fabs(e) < Delta)) continue;\n            double r = e / Delta;\n"
                             "            double w = exp(-pr->alpha1 * r * r);\n            Wsum += m * w;"
                             "\n            Zsum += w;\n            if (i < 32)"),
    "weight_not_squared": ("double w = exp(-pr->alpha1 * r * r);\n            Wsum += m * w;"
                           "\n            Zsum += w;\n            if (i < 32)",
                           "double w = exp(-pr->alpha1 * fabs(r));\n            Wsum += m * w;"
                           "\n            Zsum += w;\n            if (i < 32)"),
    "gamma_ignored": ("double Delta = pr->gamma * hv;\n            double e",
                      "double Delta = hv;\n            double e"),
    "centre_offset": ("double c[3] = {origin[0] + (i + 0.5) * h",
                      "double c[3] = {origin[0] + (i + 1.0) * h"),
    "mask_gate_exclusive": ("*pass = *m >= pr->tau_m;\n    } else if",
                            "*pass = *m > pr->tau_m;\n    } else if"),
    "P_inverted": ("double P = Zsum > pr->eps ? Wsum / Zsum : 0.0;",
                   "double P = Zsum > pr->eps ? Zsum / (Wsum + 1e-300) : 0.0;"),
    "vmask_not_gated": ("vmask_out[a] = seg ? bits : 0u;", "vmask_out[a] = bits;"),
    "consensus_exclusive": ("int seg = P >= pr->tau_cons;", "int seg = P > pr->tau_cons;"),
    "view_bit_shifted": ("if (i < 32) bits |= 1u << i;", "if (i < 31) bits |= 1u << (i + 1);"),
    "z_near_dropped": ("if (!(p[2] > z_near)) return 0;", ""),
    "hv_linear_stretch": ("*hv = h / ((2.0 - rho) * (2.0 - rho));", "*hv = h / (2.0 - rho);"),
    "uncontract_wrong": ("double s = 1.0 / (rho * (2.0 - rho));", "double s = 1.0 / (2.0 - rho);"),
    "contract_wrong": ("double s = (2.0 - 1.0 / r) / r;", "double s = (2.0 - 1.0 / r);"),
    "label_closed_bound": ("s < (double)g", "s <= (double)g"),
    "grad_depth_sign": ("((mv[k] - P) / Zsum) * dwdD", "((P - mv[k]) / Zsum) * dwdD"),
    "grad_sigmoid_dropped": ("mv[k] * (1.0 - mv[k]) : 1.0", "mv[k] : 1.0"),
    "grad_Z_dropped": ("(wv[k] / Zsum) * dmdl", "wv[k] * dmdl"),
    "grad_alpha_dropped": ("wv[k] * 2.0 * pr->alpha1 * ev[k]", "wv[k] * 2.0 * ev[k]"),
    # depth-tuple mode
    "tuple_one_sided_abs": ("double lhs = front ? xd - dmin : fabs(xd - dmed);",
                            "double lhs = front ? fabs(xd - dmin) : fabs(xd - dmed);"),
    "tuple_no_tightening": ("double tdep = pr->gamma * hv / (1.0 + tp->beta * E);",
                            "double tdep = pr->gamma * hv;"),
    "tuple_layered_inclusive": ("if (d <= 0) return 0;\n    return (__int128)d * d > ",
                                "if (d < 0) return 0;\n    return (__int128)d * d >= "),
    "tuple_behind_margin_dropped": ("int behind_fail = xd > dsurf + tp->behind_margin * hv;",
                                    "int behind_fail = xd > dsurf;"),
    "tuple_coverage_over_area": ("(double)n_md >= tp->rho_cover * (double)n_depth",
                                 "(double)n_md >= tp->rho_cover * (double)A"),
    "tuple_ray_factor_dropped": ("double lo = dmin * ray, hi = dref * ray;",
                                 "double lo = dmin, hi = dref;"),
    "tuple_seethru_flipped": ("int seethru = dmed > tp->gamma_st * vw->d_cam;",
                              "int seethru = dmed < tp->gamma_st * vw->d_cam;"),
    "tuple_hw_not_halved": ("double dhw = fmax(0.5 * (dmax - dmin) * ray, pr->eps);",
                            "double dhw = fmax((dmax - dmin) * ray, pr->eps);"),
    "tuple_thin_denominator_t": ("if (t >= tp->tau_thin) {\n                Wsum += t;\n                Zsum += 1.0;",
                                 "if (t >= tp->tau_thin) {\n                Wsum += t;\n                Zsum += t;"),
    "tuple_dist_gate_dropped": (" &&\n                        d2 <= gate * gate)", ")"),
    "tuple_pi_ignored": ("double tau_sp = hv * pi_dg(vw, ix, iy, tp->k_dg);",
                         "double tau_sp = hv;"),
    "tuple_thin_trusted_dropped": ("int fr_q = (layered_exact(nq, A, S1, S2) || st_q) && tr_q;",
                                   "int fr_q = (layered_exact(nq, A, S1, S2) || st_q);"),
    # NeRF variant
    "nerf_lambda_range_dropped": ("double tau_sp = hv * pi_dg(vw, ix, iy, np->k_dg) +\n"
                                  "                                np->lambda_range * sqrt(k2) * (dmax - dmin);",
                                  "double tau_sp = hv * pi_dg(vw, ix, iy, np->k_dg);"),
    "nerf_delta_unclamped": ("double zc = zproj < dmin ? dmin : (zproj > dmax ? dmax : zproj);",
                             "double zc = zproj;"),
    "nerf_bonus_uncapped": ("double b = fmin(np->beta * (double)n, np->b_max);",
                            "double b = np->beta * (double)n;"),
    "nerf_thin_gamma_not_doubled": ("double tq = (2.0 * np->gamma + bq) * hv;",
                                    "double tq = (np->gamma + bq) * hv;"),
    "nerf_mmax_supportive_only": (
        "if (mq > m_max) m_max = mq;\n"
        "                    double bq = fmin(np->beta * (double)vw->n_samp[q], np->b_max);\n"
        "                    double tq = (2.0 * np->gamma + bq) * hv;\n"
        "                    double e = fabs(xd - (double)vw->d_med[q]);\n"
        "                    near_flag(e, tq, fabs(xd), &flags);\n"
        "                    if (hq && e <= tq) ++n_valid;",
        "double bq = fmin(np->beta * (double)vw->n_samp[q], np->b_max);\n"
        "                    double tq = (2.0 * np->gamma + bq) * hv;\n"
        "                    double e = fabs(xd - (double)vw->d_med[q]);\n"
        "                    near_flag(e, tq, fabs(xd), &flags);\n"
        "                    if (hq && e <= tq) { ++n_valid; if (mq > m_max) m_max = mq; }"),
    "nerf_coverage_exclusive": ("((double)n_valid >= np->rho_cover * (double)N)",
                                "((double)n_valid > np->rho_cover * (double)N)"),
    "nerf_weight_full_width": ("double hd = fmax(0.5 * (dmax - dmin), pr->eps);",
                               "double hd = fmax(dmax - dmin, pr->eps);"),
    "nerf_density_ignored": ("if (!check_thin || !eligible || !(rho_v >= np->rho_thin)) continue;",
                             "if (!check_thin || !eligible) continue;"),
    "nerf_thin_after_thick": ("if (!check_thin || !eligible || !(rho_v >= np->rho_thin)) continue;",
                              "if (!eligible || !(rho_v >= np->rho_thin)) continue;"),
    # near-boundary flags: bands wider than 1e-6 of the decision's scale, or none
    "flag_margin_widened": ("#define ORACLE_MARGIN 1e-6", "#define ORACLE_MARGIN 4e-6"),
    "flag_pixel_scale_dropped": ("dist_to_int(u) < ORACLE_MARGIN * su", "dist_to_int(u) < ORACLE_MARGIN"),
    "flag_depth_missing": ("if (fabs(fabs(e) - Delta) < ORACLE_MARGIN * sc) flags |= FLAG_DEPTH;", ""),
    "flag_tuple_distance_coordinate_scale": ("near_flag(sqrt(d2), gate, gate, &flags);",
                                             "near_flag(sqrt(d2), gate, 4.0 * (1.0 + fabs(x[2])), &flags);"),
    "flag_nerf_spatial_coordinate_scale": ("near_flag(delta, tau_sp, tau_sp, &flags);",
                                           "near_flag(delta, tau_sp, 4.0 * (1.0 + fabs(xd)), &flags);"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, (name, src.count(old))
    mut = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(mut)
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", str(c),
                    "-o", str(so), "-lm"], check=True)
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    orc = oracle.variant(_build(tmp_path, name, old, new))
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(orc)
        except AssertionError:
            caught.append(pin.__name__)
            break
    assert caught, f"no pin caught the planted mistake {name}"
