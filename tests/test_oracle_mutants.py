"""Planted mistakes in the oracle must make its pins fail.

Each entry plants one plausible slip (a dropped term, a wrong sign, index or
coefficient, a swapped operand, a wrong boundary rule) in a copy of
oracle/hgks_ref.c, builds the copy, and runs the pins named beside it
against the copy (through HGKS_REF_LIB): at least one of them must fail.
The original text has to occur exactly once in the oracle, so an edit of the
oracle that moves or rewrites a planted line shows up here.  Everything runs
on the CPU; nothing is planted in the CUDA path.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hgks_ref.c")

K = "tests/test_oracle_kinetic.py::"
W = "tests/test_oracle_weno.py::"
S = "tests/test_oracle_solver.py::"
D = "tests/test_decomp.py::"

# (name, original text, planted text, pins of which one must fail)
MUTANTS = [
    # velocity and internal-energy moments, primitives (Sec. 2)
    ("half_range_first_moment_sign", "m[1] = U * m[0] + e; }", "m[1] = U * m[0] - e; }",
     [K + "test_velocity_moments_against_quadrature"]),
    ("moment_recurrence_index", "(n + 1) / (2.0 * lam) * m[n]", "n / (2.0 * lam) * m[n]",
     [K + "test_velocity_moments_against_quadrature"]),
    ("xi4_moment", "K * (K + 2.0) / (4.0 * lam * lam)", "K * K / (4.0 * lam * lam)",
     [K + "test_internal_moments_against_quadrature"]),
    ("lambda_factor", "(K + 3.0) * rho / (4.0 * eint)", "(K + 3.0) * rho / (2.0 * eint)",
     [K + "test_primitive_lambda"]),
    ("psi4_without_xi", "        p_add(p, 0.5, extra_u, 0, 0, 1);\n", "",
     [K + "test_micro_slope_against_quadrature"]),
    ("slope_v_w_transposed", "p_add(p, s * a[2], e[0], e[1] + 1, e[2], e[3]);",
     "p_add(p, s * a[2], e[0], e[1], e[2] + 1, e[3]);", [K + "test_navier_stokes_limit"]),
    ("heat_weight_sign", "p_add(p, -1.5 * U0, 2, 0, 0, 0);", "p_add(p, 1.5 * U0, 2, 0, 0, 0);",
     [K + "test_uniform_state_gives_euler_flux"]),
    # micro-slopes, compatibility, time integration of the flux (Sec. 2)
    ("time_slope_sign", "b[i] = -moment2(&pp, &pau, g, R_FULL) / g->rho;",
     "b[i] = moment2(&pp, &pau, g, R_FULL) / g->rho;", [K + "test_point_flux_against_brute_force"]),
    ("compat_wrong_half_range", "moment2(&pp, one_poly(), gr, R_NEG);", "moment2(&pp, one_poly(), gr, R_POS);",
     [K + "test_compat_against_quadrature"]),
    ("time_coefficient_sign", "- tau * d - tau * d * e;", "- tau * d + tau * d * e;",
     [K + "test_time_coefficients_against_quadrature"]),
    ("time_fit_weight", "(4.0 * Ih[i] - If[i]) / dt", "(2.0 * Ih[i] - If[i]) / dt",
     [K + "test_time_fit_recovers_linear_flux"]),
    ("nonequilibrium_slope_sign", "- q[4] * B[4][i] - tau", "+ q[4] * B[4][i] - tau",
     [K + "test_navier_stokes_limit"]),
    ("equilibrium_time_slope_dropped", "+ q[2] * B[2][i] + q[3]", "+ q[3]",
     [K + "test_point_flux_against_brute_force"]),
    ("prandtl_fix_inverted", "(1.0 / gp->Pr - 1.0) * I[5]", "(gp->Pr - 1.0) * I[5]",
     [K + "test_navier_stokes_limit"]),
    ("collision_time_mu_over_rho", "viscosity(&gp->visc, T0) / p0", "viscosity(&gp->visc, T0) / W0[0]",
     [K + "test_point_flux_against_brute_force"]),
    # WENO-Z and the reconstructions (R-W, R-SL, R-EQ, R-T)
    ("weno_z_tau_index", "fabs(beta[0] - beta[2])", "fabs(beta[0] - beta[1])",
     [W + "test_weno_z_avoids_discontinuous_stencil"]),
    ("weno_z_weight_without_one", "P->lin[k] * (1.0 + tau5 / (beta[k] + eps))",
     "P->lin[k] * (tau5 / (beta[k] + eps))", [S + "test_free_stream_preserved_bitwise"]),
    ("smoothness_second_derivative_dropped", "return poly_int_cell(sq1, 3) + poly_int_cell(sq2, 1);",
     "return poly_int_cell(sq1, 3);", [W + "test_smoothness_indicators_jiang_shu"]),
    ("normal_slope_edges_swapped", "2.0 * lm_l + 4.0 * lm_r - 6.0 * X[c][2]", "4.0 * lm_l + 2.0 * lm_r - 6.0 * X[c][2]",
     [S + "test_shear_wave_viscous_decay"]),
    ("normal_slope_sign", "-4.0 * r_l - 2.0 * r_r + 6.0 * X[c][3]", "4.0 * r_l + 2.0 * r_r - 6.0 * X[c][3]",
     [S + "test_shear_wave_viscous_decay"]),
    ("equilibrium_slope_coefficient", "(15.0 * (X[c][3] - X[c][2])", "(16.0 * (X[c][3] - X[c][2])",
     [S + "test_shear_wave_viscous_decay"]),
    ("gauss_point_of_wrong_direction", "V[qi][c] = weno_z_at(X, gpt[n]);", "V[qi][c] = weno_z_at(X, gpt[m]);",
     [S + "test_tgv_reflection_symmetries"]),
    ("gauss_weight", "Fsum[c] += 0.25 * Fn[c];", "Fsum[c] += 0.5 * Fn[c];", [S + "test_shear_wave_viscous_decay"]),
    ("tangential_equilibrium_slope_dropped", "dQ0[1][c] = Dt1[2][c] / h1;", "dQ0[1][c] = 0.0;",
     [S + "test_tgv_swap_symmetry_approximate"]),
    ("second_tangential_slope_dropped", "dQl[2][c] = Dt2[0][c] / h2;", "dQl[2][c] = 0.0;",
     [S + "test_tgv_reflection_symmetries"]),
    ("tangential_cell_size_swapped", "dQ0[2][c] = Dt2[2][c] / h2;", "dQ0[2][c] = Dt2[2][c] / h1;",
     [S + "test_diagonal_shear_wave_viscous_decay"]),
    # mesh, boundaries, time step (R-MESH, R-BC, R-DT)
    ("z_face_area", "else area = dx_(h) * dy_cell(h, ijk[1]);", "else area = dx_(h) * dz_(h);",
     [S + "test_advection_across_stretched_mesh"]),
    ("stretch_metric", "return 0.5 * h->g.ly * b * (1.0 - th * th) / tanh(b) * ds;",
     "return 0.5 * h->g.ly * b * (1.0 - th * th) * ds;", [S + "test_wall_modes_decay"]),
    ("periodic_ghost_shift", "s = ((g % n) + n) % n;", "s = ((g % n) + n + 1) % n;",
     [S + "test_conservation_periodic"]),
    ("wall_slip", "double U = -W[1], V = -W[2], Wv = -W[3];", "double U = W[1], V = -W[2], Wv = -W[3];",
     [S + "test_channel_wall_shear_laminar"]),
    ("wall_adiabatic", "double Tg = 2.0 * Tw - T;", "double Tg = T;", [S + "test_wall_modes_decay"]),
    ("time_step_uniform_y", "double hd[3] = { dx_(h), dy_cell(h, j), dz_(h) };",
     "double hd[3] = { dx_(h), dx_(h), dz_(h) };", [S + "test_time_step_per_direction"]),
    ("time_step_normal_velocity", "double v = hd[d] / (fabs(W[1 + d]) + cs);", "double v = hd[d] / (fabs(W[1]) + cs);",
     [S + "test_time_step_per_direction"]),
    # S2O4 update and the body force (Eq. "two-stage", R-S2, R-F)
    ("two_stage_first_coefficient", "+ 0.125 * dt * dt * h->dL1", "+ 0.25 * dt * dt * h->dL1",
     [S + "test_convergence_order_1d"]),
    ("two_stage_second_weights", "(h->dL1[c * N + ci] + 2.0 * h->dL2[c * N + ci])",
     "(2.0 * h->dL1[c * N + ci] + h->dL2[c * N + ci])", [S + "test_convergence_order_1d"]),
    ("force_time_derivative_momentum_dropped", "for (int e = 0; e < 3; e++) dLc[1 + e] += h->G[e] * Lc[0];", "",
     [S + "test_body_force_source_and_its_time_derivative"]),
    ("force_time_derivative_energy_dropped", "dLc[4] += h->G[0] * Lc[1] + h->G[1] * Lc[2] + h->G[2] * Lc[3];", "",
     [S + "test_body_force_source_and_its_time_derivative"]),
    ("force_work_dropped", "Lc[4] += q[1 * S + p] * h->G[0] + q[2 * S + p] * h->G[1] + q[3 * S + p] * h->G[2];", "",
     [S + "test_body_force_source_and_its_time_derivative"]),
    # diagnostics and initial states (R-STAT, R-INIT, R-NOISE)
    ("enstrophy_factor", "ens += 0.5 * W[0] * w2 * vol;", "ens += W[0] * w2 * vol;",
     [S + "test_stats_vorticity_and_dilatation"]),
    ("dilatation_dropped", "eps += mu * (w2 + 4.0 / 3.0 * div * div) * vol;", "eps += mu * w2 * vol;",
     [S + "test_stats_vorticity_and_dilatation"]),
    ("vorticity_sign", "wy = gr[0][2] - gr[2][0]", "wy = gr[0][2] + gr[2][0]",
     [S + "test_stats_vorticity_and_dilatation"]),
    ("wall_shear_sign", "s += acc; walls++;", "s -= acc; walls++;", [S + "test_channel_wall_shear_laminar"]),
    ("tgv_pressure", "(C2x + C2y) * (C2z + 2.0)", "(C2x + C2y) * (C2z + 1.0)",
     [S + "test_tgv_initial_field_is_exact_cell_average"]),
    ("channel_profile", "double U = 1.5 * Ub * (1.0 - yn * yn);", "double U = Ub * (1.0 - yn * yn);",
     [S + "test_channel_wall_shear_laminar"]),
    ("splitmix_shift", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;", "z = (z ^ (z >> 28)) * 0x94D049BB133111EBull;",
     [S + "test_channel_noise_generator"]),
    ("density_wave_point_values", "if (kd[d] > 0) fac *= sin(PI * hs[d] / 2.0) / (PI * hs[d] / 2.0);", "",
     [S + "test_density_wave_initial_field_is_exact_cell_average"]),
    # reconstruction tables
    ("cell_average_of_power", "return (pow(c + 0.5, n + 1) - pow(c - 0.5, n + 1)) / (n + 1);",
     "return (pow(c + 0.5, n + 1) - pow(c - 0.5, n + 1)) / n;", [W + "test_linear_weights_at_faces"]),
    ("fit_derivative_power", "else s[n] = (n == 0) ? 0.0 : n * pow(sigma, n - 1);",
     "else s[n] = (n == 0) ? 0.0 : pow(sigma, n - 1);", [W + "test_quartic_value_and_derivative"]),
    ("gauss_abscissa", "const double g = sqrt(3.0) / 6.0;", "const double g = sqrt(3.0) / 3.0;",
     [S + "test_convergence_order_2d_diagonal"]),
    ("edge_points_swapped", "build_weno_point(&wp[WP_RIGHT], 0.5);", "build_weno_point(&wp[WP_RIGHT], -0.5);",
     [S + "test_shear_wave_viscous_decay"]),
    ("tangential_slope_from_value_weights", "Dt1[qi][c] = dot5(gpt[n]->qv, X);", "Dt1[qi][c] = dot5(gpt[n]->qd, X);",
     [S + "test_tgv_reflection_symmetries"]),
    # sweep geometry: rotation, tangential order, metrics, areas, volumes
    ("rotation_of_y_sweep", "{ 0, 2, 1, 3, 4 }", "{ 0, 2, 3, 1, 4 }", [S + "test_tgv_reflection_symmetries"]),
    ("tangential_order_of_z_sweep", "static const int tdir[3][2] = { { 1, 2 }, { 0, 2 }, { 0, 1 } };",
     "static const int tdir[3][2] = { { 1, 2 }, { 0, 2 }, { 1, 0 } };", [S + "test_tgv_reflection_symmetries"]),
    ("normal_metric_at_centre", "double hn = metric(h, d, (double)f);", "double hn = metric(h, d, f + 0.5);",
     [S + "test_channel_wall_shear_laminar"]),
    ("tangential_metric_at_centre", "double h1 = metric(h, tdir[d][0], a + 0.5 + gpt[m]->sigma);",
     "double h1 = metric(h, tdir[d][0], a + 0.5);", [S + "test_face_stress_uses_metric_at_gauss_points"]),
    ("x_face_area", "if (d == 0) area = dy_cell(h, ijk[1]) * dz_(h);", "if (d == 0) area = dx_(h) * dz_(h);",
     [S + "test_body_force_source_and_its_time_derivative"]),
    ("cell_volume", "double vol = dx_(h) * dy_cell(h, j) * dz_(h);\n                /* face indices",
     "double vol = dx_(h) * dx_(h) * dz_(h);\n                /* face indices", [S + "test_shear_wave_viscous_decay"]),
    ("mesh_map_without_normalisation", "return h->g.y0 + 0.5 * h->g.ly * (1.0 + tanh(b * (s - 1.0)) / tanh(b));",
     "return h->g.y0 + 0.5 * h->g.ly * (1.0 + tanh(b * (s - 1.0)));", [S + "test_time_step_per_direction"]),
    # ghosts and walls
    ("ghost_fill_order", "if (e < d) { lo[e] = -NG; hi[e] = n_of(h, e) + NG; }",
     "if (e > d) { lo[e] = -NG; hi[e] = n_of(h, e) + NG; }", [S + "test_free_stream_preserved_bitwise"]),
    ("wall_mirror_offset", "else s = side == 0 ? m : n - 1 - m;", "else s = side == 0 ? m + 1 : n - 1 - m;",
     [S + "test_wall_modes_decay"]),
    ("wall_ghost_density", "double rho = p / Tg;", "double rho = W[0];", [S + "test_wall_modes_decay"]),
    ("wall_ghost_kinetic_energy_interior_density",
     "dst[4] = p / (h->gas.gamma - 1.0) + 0.5 * rho * (U * U + V * V + Wv * Wv);",
     "dst[4] = p / (h->gas.gamma - 1.0) + 0.5 * W[0] * (U * U + V * V + Wv * Wv);",
     [S + "test_wall_ghost_face_conditions"]),
    ("wall_shear_normalisation", "h->wall_shear = walls ? s / (walls * h->g.lx * h->g.lz) : 0.0;",
     "h->wall_shear = walls ? s / (walls * h->g.lx) : 0.0;", [S + "test_channel_wall_shear_laminar"]),
    # S2O4, gas model, kinetic weights
    ("second_stage_uses_stage_two_rhs", "h->qn[c * S + p] = h->q[c * S + p] + dt * h->L1[c * N + ci]",
     "h->qn[c * S + p] = h->q[c * S + p] + dt * h->L2[c * N + ci]", [S + "test_advection_across_stretched_mesh"]),
    ("viscosity_exponent", "return v->mu_ref * pow(T / v->T_ref, v->omega);",
     "return v->mu_ref * pow(T / v->T_ref, 1.0 - v->omega);", [K + "test_power_law_viscosity_in_shear_stress"]),
    ("kinetic_energy_factor", "double eint = Q[4] - 0.5 * rho * (U * U + V * V + Wv * Wv);",
     "double eint = Q[4] - rho * (U * U + V * V + Wv * Wv);", [K + "test_primitive_lambda"]),
    ("heat_weight_cross_sign", "double cc[3] = { 0.5, -C, 0.5 * C * C };", "double cc[3] = { 0.5, C, 0.5 * C * C };",
     [K + "test_point_flux_against_brute_force"]),
    # initial states and diagnostics
    ("tgv_sin_squared_average", "avs[d][3][i] = 0.5 - 0.5 * avs[d][2][i];", "avs[d][3][i] = 0.5 + 0.5 * avs[d][2][i];",
     [S + "test_tgv_initial_field_is_exact_cell_average"]),
    ("noise_scaled_by_bulk_velocity", "U + noise_amp * U * r0", "U + noise_amp * Ub * r0",
     [S + "test_channel_noise_recipe"]),
    ("noise_cell_index", "uint64_t idx = ((uint64_t)k * h->g.ny + j) * h->g.nx + i;",
     "uint64_t idx = ((uint64_t)j * h->g.nz + k) * h->g.nx + i;", [S + "test_channel_noise_recipe"]),
    ("stats_uniform_y_metric", "double hb = (b == 0) ? dx_(h) : (b == 1 ? dy_dj(h, j + 0.5) : dz_(h));",
     "double hb = (b == 0) ? dx_(h) : (b == 1 ? dx_(h) : dz_(h));", [S + "test_stats_on_stretched_wall_mesh"]),
    ("stats_difference_coefficient", "(uu[0][a] - 8.0 * uu[1][a] + 8.0 * uu[2][a] - uu[3][a]) / (12.0 * hb)",
     "(uu[0][a] - 8.0 * uu[1][a] + 8.0 * uu[2][a] - uu[3][a]) / (6.0 * hb)", [S + "test_stats_vorticity_and_dilatation"]),
    ("kinetic_energy_not_per_rho0", "o->Ek = ek / (h->rho_ref * vol_tot);", "o->Ek = ek / vol_tot;",
     [S + "test_diagnostics_normalised_by_rho0"]),
    # state transfer, totals, bookkeeping
    ("set_state_transposed",
     "h->q[c * h->ncell_pad + pidx(h, i, j, k)] = hq[c * h->ncell + iidx(h, i, j, k)];",
     "h->q[c * h->ncell_pad + pidx(h, i, j, k)] = hq[c * h->ncell + iidx(h, j % h->g.nx, i % h->g.ny, k)];",
     [S + "test_shear_wave_viscous_decay"]),
    ("mass_without_volume", "mass += Q[0] * vol;", "mass += Q[0];", [S + "test_totals_on_stretched_grid"]),
    ("energy_total_component", "en += Q[4] * vol;", "en += Q[3] * vol;", [S + "test_conservation_periodic"]),
    ("momentum_total_component", "for (int a = 0; a < 3; a++) mom[a] += Q[1 + a] * vol;",
     "for (int a = 0; a < 3; a++) mom[a] += Q[1] * vol;", [S + "test_channel_wall_shear_laminar"]),
    ("max_mach_isothermal_sound", "double cs = sqrt(h->gas.gamma * pr / W[0]);\n                if (sqrt(u2) / cs > mmax)",
     "double cs = sqrt(pr / W[0]);\n                if (sqrt(u2) / cs > mmax)", [S + "test_stats_vorticity_and_dilatation"]),
    ("wall_shear_top_wall_dropped", "            s += acc; walls++;\n", "            walls++;\n",
     [S + "test_channel_wall_shear_laminar"]),
    ("time_not_advanced", "    h->t += dt;\n", "", [S + "test_time_and_step_bookkeeping"]),
    # initial states
    ("tgv_origin_ignored", "if (d == 0) { xl = h->g.x0 + i * dx_(h); xr = xl + dx_(h); }",
     "if (d == 0) { xl = i * dx_(h); xr = xl + dx_(h); }", [S + "test_tgv_initial_field_with_origin_offset"]),
    ("tgv_cos_z_average", "double Cz = avs[2][1][k], C2z = avs[2][2][k], ccz = avs[2][4][k];",
     "double Cz = avs[2][0][k], C2z = avs[2][2][k], ccz = avs[2][4][k];",
     [S + "test_tgv_initial_field_is_exact_cell_average"]),
    ("density_wave_velocity_not_momentum", "for (int d = 0; d < 3; d++) h->q[(1 + d) * S + pp] = rho * kd[d];",
     "for (int d = 0; d < 3; d++) h->q[(1 + d) * S + pp] = kd[d];", [S + "test_density_wave_initial_field_is_exact_cell_average"]),
    ("channel_wall_temperature", "const double Tw = Ub * Ub / (h->gas.gamma * Ma_b * Ma_b);",
     "const double Tw = Ub * Ub / (Ma_b * Ma_b);", [S + "test_channel_wall_shear_laminar"]),
    ("channel_profile_centre", "const double ymid = h->g.y0 + 0.5 * h->g.ly, hh = 0.5 * h->g.ly;",
     "const double ymid = h->g.y0, hh = 0.5 * h->g.ly;", [S + "test_channel_noise_recipe"]),
    # time loop
    ("step_without_ghost_fill",
     "    for (int s = 0; s < nsteps; s++) {\n        ghost_fill(h, h->q);\n        double m = dt_limit(h, h->q);",
     "    for (int s = 0; s < nsteps; s++) {\n        double m = dt_limit(h, h->q);", [S + "test_conservation_periodic"]),
    ("stage_two_without_ghost_fill", "    ghost_fill(h, h->qs);\n    /* stage 2 on Q* */", "    /* stage 2 on Q* */",
     [S + "test_conservation_periodic"]),
    # sampled-cell right-hand side (must equal the full one)
    ("sampled_face_offset", "face_flux_local(h, h->q, d, f + 1, a, b, dt, Fp, dFp);",
     "face_flux_local(h, h->q, d, f + 1, a, b + (d == 0), dt, Fp, dFp);", [S + "test_sampled_rhs_matches_full_rhs"]),
    ("sampled_cell_volume", "        double vol = dx_(h) * dy_cell(h, j) * dz_(h);\n        double Lc[5], dLc[5];",
     "        double vol = dx_(h) * dy_dj(h, j + 0.5) * dz_(h);\n        double Lc[5], dLc[5];",
     [S + "test_sampled_rhs_matches_full_rhs"]),
    # kinetic weights and time coefficients
    ("time_coefficient_q4_decay", "q[4] = 2.0 * tau * tau * (1.0 - e) - tau * d * e;",
     "q[4] = 2.0 * tau * tau * (1.0 - e) - tau * d;", [K + "test_time_coefficients_against_quadrature"]),
    ("time_coefficient_q3", "q[3] = tau * (1.0 - e);", "q[3] = tau * e;", [K + "test_time_coefficients_against_quadrature"]),
    ("heat_weight_without_xi", "p_add(p, 0.5, 1, 0, 0, 1);", "p_add(p, 0.5, 1, 0, 0, 0);",
     [K + "test_uniform_state_gives_euler_flux"]),
    ("slope_energy_without_xi", "p_add(p, s * 0.5 * a[4], e[0], e[1], e[2], e[3] + 1);",
     "p_add(p, s * 0.5 * a[4], e[0], e[1], e[2], e[3]);", [K + "test_navier_stokes_limit"]),
    # moment engine internals
    ("maxwellian_v_from_w", "moments_1d(W[2], W[4], R_FULL, 8, g->mu[1]);", "moments_1d(W[3], W[4], R_FULL, 8, g->mu[1]);",
     [K + "test_micro_slope_against_quadrature"]),
    ("psi_v_component", "case 2: p_add(p, 1.0, extra_u, 1, 0, 0); break;", "case 2: p_add(p, 1.0, extra_u, 0, 1, 0); break;",
     [K + "test_micro_slope_against_quadrature"]),
    ("psi_energy_w_as_v", "        p_add(p, 0.5, extra_u, 0, 2, 0);\n", "        p_add(p, 0.5, extra_u, 2, 0, 0);\n",
     [K + "test_micro_slope_against_quadrature"]),
    ("half_ranges_swapped", "const double *mu = (range == R_FULL) ? g->mu[0] : (range == R_POS ? g->mpos : g->mneg);",
     "const double *mu = (range == R_FULL) ? g->mu[0] : (range == R_POS ? g->mneg : g->mpos);",
     [K + "test_compat_against_quadrature"]),
    ("internal_moment_index", "return mu[e[0]] * g->mu[1][e[1]] * g->mu[2][e[2]] * g->mxi[e[3]];",
     "return mu[e[0]] * g->mu[1][e[1]] * g->mu[2][e[2]] * g->mxi[e[3] > 0 ? e[3] - 1 : 0];",
     [K + "test_micro_slope_against_quadrature"]),
    ("slope_rhs_not_per_density", "for (int i = 0; i < 5; i++) b[i] = dQ[i] / g->rho;\n    gauss_solve(5, M, b, a);",
     "for (int i = 0; i < 5; i++) b[i] = dQ[i];\n    gauss_solve(5, M, b, a);", [K + "test_micro_slope_against_quadrature"]),
    # point-flux assembly
    ("equilibrium_term_with_left_slopes", "B[1][i] = moment2(&wgt, &au_0, &g0, R_FULL);",
     "B[1][i] = moment2(&wgt, &au_l, &g0, R_FULL);", [K + "test_point_flux_against_brute_force"]),
    ("equilibrium_time_slope_of_left_state", "time_slope_solve(&g0, a0, A0);", "time_slope_solve(&gl, a0, A0);",
     [K + "test_point_flux_against_brute_force"]),
    ("right_side_slope_term_range",
     "B[4][i] = moment2(&wgt, &au_l, &gl, R_POS) + moment2(&wgt, &au_r, &gr, R_NEG);",
     "B[4][i] = moment2(&wgt, &au_l, &gl, R_POS) + moment2(&wgt, &au_r, &gr, R_POS);",
     [K + "test_point_flux_against_brute_force"]),
    ("collision_temperature_of_left_state", "double T0 = 1.0 / (2.0 * W0[4]);", "double T0 = 1.0 / (2.0 * Wl[4]);",
     [K + "test_point_flux_against_brute_force"]),
    ("time_fit_slope_factor", "dFn[i] = 4.0 * (If[i] - 2.0 * Ih[i]) / (dt * dt);",
     "dFn[i] = 2.0 * (If[i] - 2.0 * Ih[i]) / (dt * dt);", [K + "test_time_fit_recovers_linear_flux"]),
    # sweeps, divergence, diagnostics
    ("z_metric_from_x", "if (d == 2) return dz_(h);", "if (d == 2) return dx_(h);",
     [S + "test_advection_across_stretched_mesh"]),
    ("normal_reconstruction_right_stencil", "const double *sl = &X[c][0], *sr = &X[c][1];",
     "const double *sl = &X[c][0], *sr = &X[c][0];", [S + "test_shear_wave_viscous_decay"]),
    ("tangential_values_linear", "T1V[kk][qi][c] = weno_z_at(X, gpt[m]);", "T1V[kk][qi][c] = dot5(gpt[m]->qv, X);",
     [S + "test_tangential_values_non_oscillatory_at_a_step"]),
    ("face_records_transposed", "size_t fi = ((size_t)(b + kk) * e1 + (size_t)(a + jj)) * (nd + 1) + f;",
     "size_t fi = ((size_t)(b + jj) * e1 + (size_t)(a + kk)) * (nd + 1) + f;",
     [S + "test_diagonal_shear_wave_viscous_decay"]),
    ("y_face_index_order", "size_t fy = ((size_t)k * nx + i) * (ny + 1) + j;",
     "size_t fy = ((size_t)i * nz + k) * (ny + 1) + j;", [S + "test_tgv_reflection_symmetries"]),
    ("z_divergence_sign", "double sz = h->F[2][c * nf[2] + fz + 1] - h->F[2][c * nf[2] + fz];",
     "double sz = h->F[2][c * nf[2] + fz] - h->F[2][c * nf[2] + fz + 1];",
     [S + "test_diagonal_shear_wave_viscous_decay"]),
    ("wall_shear_wrong_row",
     "for (int i = 0; i < nx; i++) acc += h->F[1][1 * nf[1] + ((size_t)k * nx + i) * (ny + 1) + 0];",
     "for (int i = 0; i < nx; i++) acc += h->F[1][1 * nf[1] + ((size_t)k * nx + i) * (ny + 1) + 1];",
     [S + "test_wall_shear_is_the_wall_face_flux"]),
    ("stats_uniform_cell_volume", "double vol = dx_(h) * dy_cell(h, j) * dz_(h);\n                double Q[5], W[5];",
     "double vol = dx_(h) * (h->g.ly / h->g.ny) * dz_(h);\n                double Q[5], W[5];",
     [S + "test_stats_on_stretched_wall_mesh"]),
    ("noise_w_from_r1", "noise_amp * Ub * r1, noise_amp * Ub * r2, p);", "noise_amp * Ub * r1, noise_amp * Ub * r1, p);",
     [S + "test_channel_noise_recipe"]),
    # linear algebra, fitting, smoothness
    ("pivot_without_rhs_swap", "            double t = b[c]; b[c] = b[p]; b[p] = t;\n", "",
     [K + "test_micro_slope_against_quadrature"]),
    ("elimination_factor", "double f = A[r * n + c] / A[c * n + c];", "double f = A[r * n + c] / A[c * n + c] * 0.5;",
     [K + "test_micro_slope_against_quadrature"]),
    ("smoothness_first_derivative", "double d1[2] = { c[1], 2.0 * c[2] };", "double d1[2] = { c[1], c[2] };",
     [W + "test_smoothness_indicators_jiang_shu"]),
    ("cell_integral_odd_terms", "if (k % 2 == 0) s += c[k] * 2.0 * pow(0.5, k + 1) / (k + 1);",
     "s += c[k] * 2.0 * pow(0.5, k + 1) / (k + 1);", [W + "test_smoothness_indicators_jiang_shu"]),
    ("linear_weights_fit_slopes", "for (int j = 0; j < 5; j++) rhs[a] += P->cand[a][j] * P->qv[j];",
     "for (int j = 0; j < 5; j++) rhs[a] += P->cand[a][j] * P->qd[j];", [W + "test_linear_weights_at_faces"]),
    # heat-flux weight (Prandtl correction)
    ("heat_linear_coefficient", "p_add(p, 1.5 * U0 * U0, 1, 0, 0, 0);", "p_add(p, 0.5 * U0 * U0, 1, 0, 0, 0);",
     [K + "test_uniform_state_gives_euler_flux"]),
    ("heat_constant_sign", "p_add(p, -0.5 * U0 * U0 * U0, 0, 0, 0, 0);", "p_add(p, 0.5 * U0 * U0 * U0, 0, 0, 0, 0);",
     [K + "test_uniform_state_gives_euler_flux"]),
    ("heat_xi_shift_sign", "p_add(p, -0.5 * U0, 0, 0, 0, 1);", "p_add(p, 0.5 * U0, 0, 0, 0, 1);",
     [K + "test_uniform_state_gives_euler_flux"]),
    ("heat_cross_shift_sign", "p_add(p, -U0 * cc[q], 0, ev, ew, 0);", "p_add(p, U0 * cc[q], 0, ev, ew, 0);",
     [K + "test_uniform_state_gives_euler_flux"]),
    # gas constants, time step, initial states, diagnostics
    ("internal_degrees_of_freedom", "h->gas.K = (5.0 - 3.0 * gamma) / (gamma - 1.0);",
     "h->gas.K = (3.0 - gamma) / (gamma - 1.0);", [S + "test_time_step_per_direction"]),
    ("time_step_isothermal_sound", "double cs = sqrt(h->gas.gamma * pr / W[0]);\n                double hd[3]",
     "double cs = sqrt(pr / W[0]);\n                double hd[3]", [S + "test_time_step_per_direction"]),
    ("point_value_energy", "h->q[4 * S + pp] = p / (h->gas.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);",
     "h->q[4 * S + pp] = p / h->gas.gamma + 0.5 * rho * (u * u + v * v + w * w);", [S + "test_channel_noise_recipe"]),
    ("tgv_mean_pressure", "const double p0 = rho0 * U0 * U0 / (h->gas.gamma * Ma * Ma);",
     "const double p0 = rho0 * U0 / (h->gas.gamma * Ma * Ma);", [S + "test_tgv_initial_field_with_origin_offset"]),
    ("density_wave_energy", "h->q[4 * S + pp] = 1.0 / (h->gas.gamma - 1.0) + 0.5 * rho * (kd[0] + kd[1] + kd[2]);",
     "h->q[4 * S + pp] = 1.0 / (h->gas.gamma - 1.0) + 0.5 * (kd[0] + kd[1] + kd[2]);",
     [S + "test_density_wave_initial_field_is_exact_cell_average"]),
    ("divergence_sign", "double div = gr[0][0] + gr[1][1] + gr[2][2];", "double div = gr[0][0] - gr[1][1] + gr[2][2];",
     [S + "test_stats_vorticity_and_dilatation"]),
    # entry points, hooks and the step's bookkeeping
    ("rhs_without_ghost_fill", "    ghost_fill(h, h->q);\n    eval_rhs(h, h->q, dt, L, dL, 0);",
     "    eval_rhs(h, h->q, dt, L, dL, 0);", [S + "test_sampled_rhs_matches_full_rhs"]),
    ("step_ignores_cfl_hook", "        if (h->min_hook) m = h->min_hook(h->hook_user, m);\n        double dt = cfl * m;",
     "        double dt = cfl * m;", [S + "test_cfl_minimum_hook_applies_to_steps_and_compute_dt"]),
    ("compute_dt_ignores_cfl_hook",
     "    double m = dt_limit(h, h->q);\n    if (h->min_hook) m = h->min_hook(h->hook_user, m);\n    *dt = cfl * m;",
     "    double m = dt_limit(h, h->q);\n    *dt = cfl * m;", [S + "test_cfl_minimum_hook_applies_to_steps_and_compute_dt"]),
    ("halo_hook_not_called", "    if (h->halo_hook) h->halo_hook(h->hook_user, q);\n", "",
     [D + "test_split_equals_unsplit"]),
    ("state_not_swapped", "    double *t = h->q; h->q = h->qn; h->qn = t;\n", "", [S + "test_shear_wave_viscous_decay"]),
    ("last_dt_not_recorded", "    h->dt_last = dt;\n    return HGKS_REF_OK;", "    return HGKS_REF_OK;",
     [S + "test_time_and_step_bookkeeping"]),
    ("first_stage_full_step", "h->qs[c * S + p] = h->q[c * S + p] + 0.5 * dt * h->L1[c * N + ci]",
     "h->qs[c * S + p] = h->q[c * S + p] + dt * h->L1[c * N + ci]", [S + "test_convergence_order_1d"]),
    ("wall_shear_from_second_stage", "    eval_rhs(h, h->qs, dt, h->L2, h->dL2, 0);",
     "    eval_rhs(h, h->qs, dt, h->L2, h->dL2, 1);", [S + "test_wall_shear_is_the_wall_face_flux"]),
    ("get_state_component_shift",
     "hq[c * h->ncell + iidx(h, i, j, k)] = h->q[c * h->ncell_pad + pidx(h, i, j, k)];",
     "hq[c * h->ncell + iidx(h, i, j, k)] = h->q[((c + 1) % 5) * h->ncell_pad + pidx(h, i, j, k)];",
     [S + "test_free_stream_preserved_bitwise"]),
    ("stats_density_not_from_tgv", "    h->rho_ref = rho0;\n", "", [S + "test_diagnostics_normalised_by_rho0"]),
    ("step_counter_increment", "    h->step += 1;\n", "    h->step += 2;\n", [S + "test_time_and_step_bookkeeping"]),
    # uniform-mesh branches, defaults, small helpers
    ("uniform_metric_length", "double ds = 2.0 / h->g.ny;\n    if (!stretched(h)) return h->g.ly / h->g.ny;",
     "double ds = 2.0 / h->g.ny;\n    if (!stretched(h)) return h->g.lz / h->g.ny;", [S + "test_shear_wave_viscous_decay"]),
    ("uniform_cell_height", "static double dy_cell(const hgks_ref_t h, int j)\n{\n    if (!stretched(h)) return h->g.ly / h->g.ny;",
     "static double dy_cell(const hgks_ref_t h, int j)\n{\n    if (!stretched(h)) return h->g.lz / h->g.ny;",
     [S + "test_shear_wave_viscous_decay"]),
    ("uniform_y_map", "if (!stretched(h)) return h->g.y0 + 0.5 * s * h->g.ly;", "if (!stretched(h)) return h->g.y0 + s * h->g.ly;",
     [S + "test_channel_noise_recipe"]),
    ("noise_range_halved", "* (1.0 / 4503599627370496.0) - 1.0;", "* (1.0 / 9007199254740992.0) - 1.0;",
     [S + "test_channel_noise_recipe"]),
    ("default_reference_density", "    h->rho_ref = 1.0;\n    h->np[0]", "    h->rho_ref = 2.0;\n    h->np[0]",
     [S + "test_stats_vorticity_and_dilatation"]),
    ("density_wave_in_single_cell_directions", "double kd[3] = { h->g.nx > 1, h->g.ny > 1, h->g.nz > 1 };",
     "double kd[3] = { 1, 1, 1 };", [S + "test_convergence_order_1d"]),
    ("density_wave_y_spacing", "double hs[3] = { dx_(h), h->g.ly / h->g.ny, dz_(h) };",
     "double hs[3] = { dx_(h), dx_(h), dz_(h) };", [S + "test_density_wave_initial_field_is_exact_cell_average"]),
    ("stats_z_spacing", "(b == 1 ? dy_dj(h, j + 0.5) : dz_(h))", "(b == 1 ? dy_dj(h, j + 0.5) : dx_(h))",
     [S + "test_stats_vorticity_and_dilatation"]),
]


def _plant_and_run(name, original, planted, pins, workdir):
    from oracle.build import compile_oracle
    with open(SRC) as f:
        src = f.read()
    if src.count(original) != 1:
        return "original text occurs %d times" % src.count(original)
    cpath = os.path.join(workdir, name + ".c")
    with open(cpath, "w") as f:
        f.write(src.replace(original, planted))
    so = compile_oracle(cpath, os.path.join(workdir, name + ".so"))
    env = dict(os.environ, HGKS_REF_LIB=so, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "--tb=no", "-p", "no:cacheprovider"] + pins,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    if r.returncode == 1:
        return None  # a pin failed: the mistake is caught
    if r.returncode == 0:
        return "survived: every pin passed"
    return "pytest exit %d: %s" % (r.returncode, r.stdout[-400:])


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    workdir = str(tmp_path_factory.mktemp("planted"))
    workers = max(1, min(16, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        # the convergence-order and brute-force pins take longest: start them first
        slow = ("convergence", "brute_force", "decomp")
        order = sorted(MUTANTS, key=lambda m: not any(k in p for p in m[3] for k in slow))
        futs = {m[0]: ex.submit(_plant_and_run, *m, workdir) for m in order}
        return {k: f.result() for k, f in futs.items()}


def test_mutant_names_unique():
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(outcomes, name):
    assert outcomes[name] is None, "%s: %s" % (name, outcomes[name])
