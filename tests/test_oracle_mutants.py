"""The pins must catch plausible slips in the oracle.  Each case plants one
mistake in a copy of part_oracle.c: a wrong sign, a dropped term or factor, a
transposed index, a wrong constant, a reversed order.  The copy is built like
the oracle, the wrappers are pointed at it, and the pin aimed at that part of
the oracle must then fail.  The same pins pass on the real oracle
(test_oracle_pins).  CPU only; mutant builds go to _build/oracle_mutants/."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

from oracle import oracle as O

import test_oracle_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "part_oracle.c")
OUT = os.path.join(ROOT, "_build", "oracle_mutants")

# name: (text in part_oracle.c, its replacement, pins that must fail[, which
# occurrence of the text, when it occurs more than once])
MUTANTS = {
    "boris_cross_product_sign": (
        "upl[0] = um[0] + (um[1] * t[2] - um[2] * t[1]);",
        "upl[0] = um[0] + (um[2] * t[1] - um[1] * t[2]);",
        [pins.test_boris_conserves_u_in_pure_B]),
    "boris_rotation_factor_dropped": (
        "s[a] = 2.0 * t[a] / (1.0 + t2);",
        "s[a] = t[a] / (1.0 + t2);",
        [pins.test_boris_conserves_u_in_pure_B]),
    "boris_second_half_kick_dropped": (
        "for (int a = 0; a < 3; ++a) u[a] = up[a] + h * E[a];",
        "for (int a = 0; a < 3; ++a) u[a] = up[a];",
        [pins.test_boris_exb_drift_second_order]),
    "tsc_centre_weight": (
        "if (a <= 0.5) return 0.75 - a * a;",
        "if (a <= 0.5) return 0.75 - 0.5 * a * a;",
        [lambda: pins.test_shape_partition_of_unity_and_first_moment(O.TSC)]),
    "gather_z_weight_dropped": (
        "double w = (wz * wy) * wx;\n        int64_t cell = cell_linear(g, nbr(g, 0, j[0] + kx), "
        "nbr(g, 1, j[1] + ky),\n                                   nbr(g, 2, j[2] + kz));\n"
        "        for (int c = 0; c < ncomp; ++c)",
        "double w = wy * wx;\n        int64_t cell = cell_linear(g, nbr(g, 0, j[0] + kx), "
        "nbr(g, 1, j[1] + ky),\n                                   nbr(g, 2, j[2] + kz));\n"
        "        for (int c = 0; c < ncomp; ++c)",
        [lambda: pins.test_gather_uniform_and_linear(O.TSC, 3)]),
    "deposit_index_transposed": (
        "int64_t cell = cell_linear(g, nbr(g, 0, j[0] + kx), nbr(g, 1, j[1] + ky),\n"
        "                                     nbr(g, 2, j[2] + kz));\n"
        "          for (int c = 0; c < 3; ++c) out",
        "int64_t cell = cell_linear(g, nbr(g, 0, j[0] + ky), nbr(g, 1, j[1] + kx),\n"
        "                                     nbr(g, 2, j[2] + kz));\n"
        "          for (int c = 0; c < 3; ++c) out",
        [lambda: pins.test_deposit_total_and_adjoint(O.TSC, 3)]),
    "sort_ties_reversed": (
        "return x->idx < y->idx ? -1 : (x->idx > y->idx);",
        "return x->idx > y->idx ? -1 : (x->idx < y->idx);",
        [pins.test_stable_sort_matches_python_sorted]),
    "rk2_corrector_average_dropped": (
        "x1[a] = or_wrap(g, a, x0[a] + dt * (0.5 * (v1[a] + v2[a])));",
        "x1[a] = or_wrap(g, a, x0[a] + dt * v2[a]);",
        [pins.test_lp_rk_orders_on_solid_rotation]),
    "spectrum_loss_sign": (
        "double s = A + C * e;",
        "double s = A - C * e;",
        [pins.test_spec_pure_synchrotron_closed_form]),
    "spectrum_chi_power": (
        "chi[(int64_t)i * n + p] = (chi[(int64_t)i * n + p] * (s * s)) / A;",
        "chi[(int64_t)i * n + p] = (chi[(int64_t)i * n + p] * s) / A;",
        [pins.test_spec_pure_adiabatic_closed_form]),
    "shock_kernel_exponent_sign": (
        "sum += c0 * pow(eng[i] / e0, 2.0 - q) * I;",
        "sum += c0 * pow(eng[i] / e0, q - 2.0) * I;",
        [pins.test_shock_convolution_of_a_power_law_is_exact]),
    "dsa_index_denominator": (
        "double or_dsa_index(double r) { return 3.0 * r / (r - 1.0); }",
        "double or_dsa_index(double r) { return 3.0 * r / (r + 1.0); }",
        [pins.test_rh_compression_and_slope_match_the_shock_test]),
    "compaction_holes_reversed": (
        "src[holes[k]] = i;",
        "src[holes[ndel - 1 - k]] = i;",
        [pins.test_compaction_invariants]),
    "philox_multiplier": (
        "uint64_t p0 = (uint64_t)0xD2511F53u * c0;",
        "uint64_t p0 = (uint64_t)0xD2511F52u * c0;",
        [pins.test_philox_known_answers]),
    "cell_key_bricks_transposed": (
        "int64_t brick = ((int64_t)(j[2] / b[2]) * nb1 + j[1] / b[1]) * nb0 + j[0] / b[0];",
        "int64_t brick = ((int64_t)(j[2] / b[2]) * nb1 + j[0] / b[0]) * nb0 + j[1] / b[1];",
        [pins.test_cell_key_is_brick_bijection]),
    "periodic_wrap_direction": (
        "if (x < g->xmin[axis]) x = x + L;",
        "if (x < g->xmin[axis]) x = x - L;",
        [pins.test_cell_coord_edges_and_wrap]),
    "force_weight_dropped": (
        "F_out[a * n + p] = wp * ((up[a] - u0[a]) / dt);",
        "F_out[a * n + p] = (up[a] - u0[a]) / dt;",
        [pins.test_boris_step_drift_and_force, pins.test_deposit_momentum_balance]),
    "rk3_final_stage_weight": (
        "x1[a] = or_wrap(g, a, x0[a] + dt * ((k1[a] + k2[a] + 4.0 * k3[a]) / 6.0));",
        "x1[a] = or_wrap(g, a, x0[a] + dt * ((k1[a] + k2[a] + 2.0 * k3[a]) / 6.0));",
        [pins.test_lp_rk3_uniform_velocity_exact]),
    "rk3_middle_stage_point": (
        "xb[a] = or_wrap(g, a, x0[a] + dt * (0.25 * (k1[a] + k2[a])));",
        "xb[a] = or_wrap(g, a, x0[a] + dt * (0.5 * (k1[a] + k2[a])));",
        [pins.test_lp_rk_orders_on_solid_rotation]),
    "lp_b2_start_sample_dropped": (                       # the RK2 step's copy (first)
        "b2m[p] = 0.5 * (bb0 + bb1);",
        "b2m[p] = bb1;",
        [pins.test_lp_samples_in_linear_fields], 0),
    "init_spectrum_norm_sign": (
        "double norm = N0 * (1.0 - p) / (pow(emax, 1.0 - p) - pow(emin, 1.0 - p));",
        "double norm = N0 * (p - 1.0) / (pow(emax, 1.0 - p) - pow(emin, 1.0 - p));",
        [pins.test_init_spectrum_power_law_and_norm]),
    "shock_convergence_sign": (
        "if (dv < 0.0) {",
        "if (dv > 0.0) {",
        [pins.test_shock_cells_on_the_rh_snapshot]),
    "cic_weight_slope": (
        "return a < 1.0 ? 1.0 - a : 0.0;",
        "return a < 1.0 ? 1.0 - 0.5 * a : 0.0;",
        [lambda: pins.test_shape_partition_of_unity_and_first_moment(O.CIC)]),
    "gather_index_transposed": (
        "int64_t cell = cell_linear(g, nbr(g, 0, j[0] + kx), nbr(g, 1, j[1] + ky),\n"
        "                                   nbr(g, 2, j[2] + kz));\n"
        "        for (int c = 0; c < ncomp; ++c)",
        "int64_t cell = cell_linear(g, nbr(g, 0, j[0] + ky), nbr(g, 1, j[1] + kx),\n"
        "                                   nbr(g, 2, j[2] + kz));\n"
        "        for (int c = 0; c < ncomp; ++c)",
        [lambda: pins.test_gather_uniform_and_linear(O.TSC, 3)]),
    "cell_start_off_by_one": (
        "while (p < n && (int64_t)sk[p] < c) ++p;",
        "while (p < n && (int64_t)sk[p] <= c) ++p;",
        [pins.test_stable_sort_matches_python_sorted]),
    "shock_applied_every_step": (
        "if (!state[p]) {",
        "if (1) {",
        [pins.test_lp_shock_applies_once_per_crossing]),
    "rh_compression_gamma": (
        "return (gamma + 1.0) * m2 / (2.0 + (gamma - 1.0) * m2);",
        "return (gamma - 1.0) * m2 / (2.0 + (gamma - 1.0) * m2);",
        [pins.test_rh_compression_and_slope_match_the_shock_test]),
    "maxwellian_radius": (
        "double rad0 = sqrt(-2.0 * log(u01(r1[0])));",
        "double rad0 = sqrt(-1.0 * log(u01(r1[0])));",
        [pins.test_init_particles_statistics]),
    "open_outside_lower_face": (
        "if (x[a] < g->xmin[a] || x[a] >= g->xmin[a] + L) return 1;",
        "if (x[a] >= g->xmin[a] + L) return 1;",
        [pins.test_open_axis_no_wrap_and_outside]),
    "upper_edge_tie_dropped": (
        "if (jj >= g->n[a]) jj = g->n[a] - 1;",
        ";",
        [pins.test_cell_coord_edges_and_wrap]),
    "spectrum_proper_time": (
        "double dtau = dt / gam[p];",
        "double dtau = dt * gam[p];",
        [pins.test_spec_pure_synchrotron_closed_form]),
    "spectrum_expm1_factor_dropped": (
        "double C = cr * dtau * (L == 0.0 ? 1.0 : expm1(L) / L);",
        "double C = cr * dtau;",
        [pins.test_spec_combined_integrating_factor]),
    "boris_drift_without_gamma": (
        "for (int a = 0; a < g->dim; ++a) xp[a] = or_wrap(g, a, xp[a] + dt * (up[a] / gam));",
        "for (int a = 0; a < g->dim; ++a) xp[a] = or_wrap(g, a, xp[a] + dt * up[a]);",
        [pins.test_boris_step_drift_and_force]),
    "init_spectrum_spacing": (
        "double e = nb > 1 ? exp(la + (lb - la) * ((double)i / (double)(nb - 1))) : emin;",
        "double e = nb > 1 ? exp(la + (lb - la) * ((double)i / (double)nb)) : emin;",
        [pins.test_init_spectrum_power_law_and_norm]),
    "shock_ratio_inverted": (
        "double ratio = hi / lo;",
        "double ratio = lo / hi;",
        [pins.test_shock_cells_on_the_rh_snapshot]),
    "kw_index_middle_term_sign": (
        "return (3.0 * beta_u - 2.0 * beta_u * beta_d * beta_d + beta_d * beta_d * beta_d) /",
        "return (3.0 * beta_u + 2.0 * beta_u * beta_d * beta_d + beta_d * beta_d * beta_d) /",
        [pins.test_kw_index_limits]),
    "kw_index_cubic_term_dropped": (
        "return (3.0 * beta_u - 2.0 * beta_u * beta_d * beta_d + beta_d * beta_d * beta_d) /",
        "return (3.0 * beta_u - 2.0 * beta_u * beta_d * beta_d) /",
        [pins.test_kw_index_limits]),
    "shock_speed_from_proper_density": (
        "double v_sh = (D_d * v_d - D_u * v_u) / (D_d - D_u);",
        "double v_sh = (rho_d * v_d - rho_u * v_u) / (rho_d - rho_u);",
        [pins.test_shock_frame_speeds_recover_a_boosted_shock]),
    "shock_frame_galilean": (
        "double bu = fabs((v_u - v_sh) / (1.0 - v_u * v_sh));",
        "double bu = fabs(v_u - v_sh);",
        [pins.test_shock_frame_speeds_recover_a_boosted_shock]),
    "shock_lorentz_tangential_dropped": (
        "double D_u = rho_u / sqrt(1.0 - s2_u);",
        "double D_u = rho_u / sqrt(1.0 - v_u * v_u);",
        [pins.test_shock_frame_speeds_recover_a_boosted_shock]),
    "slopes_upstream_side_fixed": (
        "int64_t un = dn == cp ? cm : cp;",
        "int64_t un = cm;",
        [pins.test_shock_slopes_on_a_relativistic_snapshot]),
    "slopes_normal_component_transposed": (
        "if (or_shock_frame_speeds(vel[axis * G + up], s2u, rho[up], vel[axis * G + down],",
        "if (or_shock_frame_speeds(vel[(1 - axis) * G + up], s2u, rho[up], vel[axis * G + down],",
        [pins.test_shock_slopes_on_a_relativistic_snapshot]),
    "lp_shock_ignores_cell_slope": (
        "double q = q_cell ? q_cell[c] : or_dsa_index(r);",
        "double q = or_dsa_index(r);",
        [pins.test_lp_shock_takes_the_cell_slope]),
    "open_axis_upper_clamp_dropped": (
        "if (s > (double)g->n[a]) s = (double)g->n[a];",
        ";",
        [lambda: pins.test_open_axis_uniform_field_everywhere(O.TSC)]),
}


def _build(name):
    old, new = MUTANTS[name][:2]
    nth = MUTANTS[name][3] if len(MUTANTS[name]) > 3 else None
    src = open(SRC).read()
    if nth is None:
        assert src.count(old) == 1, f"{name}: the text to mutate must occur exactly once"
        nth = 0
    at = -1
    for _ in range(nth + 1):
        at = src.index(old, at + 1)
    os.makedirs(OUT, exist_ok=True)
    path = os.path.join(OUT, f"{name}.c")
    with open(path, "w") as f:
        f.write(src[:at] + new + src[at + len(old):])
    return O.compile_source(path, os.path.join(OUT, f"lib{name}.so"))


@pytest.fixture(scope="module")
def mutant_libs():
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        return dict(zip(MUTANTS, ex.map(_build, MUTANTS)))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pin_catches_planted_mistake(name, mutant_libs):
    aimed = MUTANTS[name][2]
    for pin in aimed:
        pin()                                  # holds on the real oracle
    caught = False
    with O.using(mutant_libs[name]), np.errstate(all="ignore"):
        for pin in aimed:
            try:
                pin()
            except AssertionError:
                caught = True
    assert caught, f"no pin caught the planted mistake {name}"
