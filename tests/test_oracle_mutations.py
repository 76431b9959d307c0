"""Planted mistakes in a copy of the oracle (CPU only).

Each case compiles a copy of the oracle's C source with one plausible
mistake (a dropped term, a wrong sign, a transposed operand, a wrong weight,
factor or boundary rule), loads it as a separate instance of the `oracle` package and runs
one of the pins of test_oracle_pins.py against it: the pin must fail.  The
oracle itself is not modified.
"""
import importlib.util
import os
import shutil

import pytest

import oracle
import test_oracle_pins as pins

# (what, text in ehd_oracle.c, its mistaken form, a pin that must fail)
MUTATIONS = [
    ("Eq. 53: the -u^2 / (2 cs2) term of r_i(u) dropped",
     "return w9[i] * (cu / cs2 + cu * cu / (2.0 * cs2 * cs2) - uu / (2.0 * cs2));",
     "return w9[i] * (cu / cs2 + cu * cu / (2.0 * cs2 * cs2));",
     "test_p2_equilibrium_moments"),
    ("Eq. 54: sign of the cs2 u.grad(rho) part of the tensor term",
     "double tens = uc * gc - cs2 * ugr;",
     "double tens = uc * gc + cs2 * ugr;",
     "test_p4_momentum_and_ion_sources_exact_for_any_rates"),
    ("Eq. 59: c_x in place of c_y in the y gradient",
     "sy += w9[i] * cy9[i] * v;",
     "sy += w9[i] * cx9[i] * v;",
     "test_p5_stencil_exact_on_low_degree_polynomials"),
    ("Eq. 25: a diagonal weight 1/18 instead of 1/36",
     "1.0 / 9.0,  1.0 / 36.0,\n",
     "1.0 / 9.0,  1.0 / 18.0,\n",
     "test_p2_equilibrium_moments"),
    ("Eq. 32: sign of the sharpening flux",
     "double vx = dphiux + cs2 * lam * nx;",
     "double vx = dphiux - cs2 * lam * nx;",
     "test_p12_static_droplet_obeys_laplace_law"),
    ("Eq. 38: sign of the advective part of the ion equilibrium",
     "out[i] = w5[i] * c * (1.0 + (cx5[i] * ux + cy5[i] * uy) / cs2);",
     "out[i] = w5[i] * c * (1.0 - (cx5[i] * ux + cy5[i] * uy) / cs2);",
     "test_p2_equilibrium_moments"),
    ("Eq. 5: (k + 2) in place of (k + 1) in the series of I1",
     "term *= y / ((double)k * (double)(k + 1));",
     "term *= y / ((double)k * (double)(k + 2));",
     "test_p6_onsager_full_form_matches_bessel_i1"),
    ("Eq. 47: vartheta times cs2 in tau_g",
     "c->tau_g = 0.5 + P->vartheta / cs2; /* Eq. 47 */",
     "c->tau_g = 0.5 + P->vartheta * cs2; /* Eq. 47 */",
     "test_p9_uniform_charge_gives_the_poisson_parabola"),
    ("Eq. 50: tau_g dropped from E_x",
     "*Ex = sx / (cs2 * tau_g);",
     "*Ex = sx / cs2;",
     "test_p9_field_is_minus_grad_psi_for_a_charge_wave"),
    ("Eq. 14: sign of the x part of -1/2 |E|^2 grad eps",
     "double Fx = mu_phi * gx + P->Kq * q * Ex - 0.5 * E2 * dex;",
     "double Fx = mu_phi * gx + P->Kq * q * Ex + 0.5 * E2 * dex;",
     "test_polarization_force_across_a_tangential_field"),
    ("Eq. 39: cs2 dropped from the L source",
     "out[i] = wq[i] * R + (L_term ? wq[i] * cF * c / cs2 : 0.0);",
     "out[i] = wq[i] * R + (L_term ? wq[i] * cF * c : 0.0);",
     "test_p15_ion_sources_carry_R_and_c_F"),
    ("Eq. 57: the 1/2 u.grad rho term dropped",
     "return cs2 / (1.0 - w9[0]) * (s_ne0 + 0.5 * (ux * grx + uy * gry) + rho * r_u(0, ux, uy));",
     "return cs2 / (1.0 - w9[0]) * (s_ne0 + rho * r_u(0, ux, uy));",
     "test_p14_pressure_of_eq57_round_trips_with_forcing"),
    ("Eq. 56: the half force dropped from u",
     "double ux = (jx + 0.5 * Fx) / rho;",
     "double ux = (jx) / rho;",
     "test_p12_static_droplet_obeys_laplace_law"),
    ("Eq. 13: sign of the kappa laplacian in the chemical potential",
     "double mu_phi = 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) - kappa * lap;",
     "double mu_phi = 4.0 * beta * phi * (phi - 1.0) * (phi - 0.5) + kappa * lap;",
     "test_p12_static_droplet_obeys_laplace_law"),
    ("Eq. 43: sign of the recombination in R",
     "*R = k_d * F - k_r * (*cp) * (*cm);",
     "*R = k_d * F + k_r * (*cp) * (*cm);",
     "test_p7_reaction_satisfies_eq41_with_eq5"),
    ("Eq. 34: sign of the cation drift",
     "c->ps[Q * k + i] = pp[i] - aq[i] + bq[i] - cq[i];   /* Eq. 34 */",
     "c->ps[Q * k + i] = pp[i] - aq[i] + bq[i] + cq[i];   /* Eq. 34 */",
     "test_ion_drift_moves_the_centroid_at_mobility_times_field"),
    ("Eq. 64: a wall link returning the same population instead of the opposite",
     "                    out[k * 9 + i] = post[k * 9 + opp9[i]];\n                else",
     "                    out[k * 9 + i] = post[k * 9 + i];\n                else",
     "test_p8_sum_phi_conserved_with_electrodes_and_walls"),
    ("Eq. 64: sign of the anti-bounce-back at the electrodes",
     "out[k * 5 + i] = mode == 0 ? -a + 2.0 * w5[i] * v : a;",
     "out[k * 5 + i] = mode == 0 ? a + 2.0 * w5[i] * v : a;",
     "test_p9_linear_potential_between_electrodes"),
    ("Eq. 30: M_phi times cs2 in tau_h",
     "double tau_h = 0.5 + P->M_phi / cs2; /* Eq. 30 */",
     "double tau_h = 0.5 + P->M_phi * cs2; /* Eq. 30 */",
     "test_p11_flat_interface_relaxes_to_tanh"),
    ("Eq. 2: 2 in place of 4 in lambda",
     "double lam = 4.0 * phi * (1.0 - phi) / W;",
     "double lam = 2.0 * phi * (1.0 - phi) / W;",
     "test_p11_flat_interface_relaxes_to_tanh"),
    ("Eq. 49: psi without the 1/(1 - w0) of the non-rest sum",
     "    return s / (1.0 - w5[0]);",
     "    return s;",
     "test_p9_linear_potential_between_electrodes"),
    ("Eq. 44: the source not divided by eps",
     "double rho_t = (P->Kq * c->q[k] - (dex * Ex + dey * Ey)) / eps;",
     "double rho_t = (P->Kq * c->q[k] - (dex * Ex + dey * Ey));",
     "test_polarization_force_sets_the_pressure_jump"),
    ("Eq. 7: sign of the grad eps . E part of the source",
     "double rho_t = (P->Kq * c->q[k] - (dex * Ex + dey * Ey)) / eps;",
     "double rho_t = (P->Kq * c->q[k] + (dex * Ex + dey * Ey)) / eps;",
     "test_polarization_force_sets_the_pressure_jump"),
    ("Eq. 6: the linear Onsager form with b^2 for 2 b^2",
     "if (form == 1) return 1.0 + 2.0 * b * b;",
     "if (form == 1) return 1.0 + b * b;",
     "test_p6_onsager_full_form_matches_bessel_i1"),
    ("Eq. 52: the rest population with w0 instead of w0 - 1",
     "double a = (i == 0) ? (w9[0] - 1.0) * p / cs2 : w9[i] * p / cs2;",
     "double a = (i == 0) ? w9[0] * p / cs2 : w9[i] * p / cs2;",
     "test_p2_equilibrium_moments"),
    ("Eq. 45: the rest population with w0 instead of w0 - 1",
     "out[i] = (i == 0) ? (w5[0] - 1.0) * psi : w5[i] * psi;",
     "out[i] = (i == 0) ? w5[0] * psi : w5[i] * psi;",
     "test_p2_equilibrium_moments"),
    ("Eq. 38 on D2Q9: sign of the advective part",
     "out[i] = w9[i] * c * (1.0 + (cx9[i] * ux + cy9[i] * uy) / cs2);",
     "out[i] = w9[i] * c * (1.0 - (cx9[i] * ux + cy9[i] * uy) / cs2);",
     "test_d2q9_ion_equilibrium_moments"),
    ("Eq. 32: cs2 dropped from the interface source",
     "out[i] = w9[i] * (cx9[i] * vx + cy9[i] * vy) / cs2;",
     "out[i] = w9[i] * (cx9[i] * vx + cy9[i] * vy);",
     "test_p11_flat_interface_relaxes_to_tanh"),
    ("Eq. 31: cs2 dropped from the advective part of h_eq",
     "out[i] = w9[i] * phi * (1.0 + (cx9[i] * ux + cy9[i] * uy) / cs2);",
     "out[i] = w9[i] * phi * (1.0 + (cx9[i] * ux + cy9[i] * uy));",
     "test_p2_equilibrium_moments"),
    ("the Laplacian stencil without its factor 2",
     "sl += 2.0 * w9[i] * (v - c0);",
     "sl += w9[i] * (v - c0);",
     "test_p5_stencil_exact_on_low_degree_polynomials"),
    ("Eq. 64: the ghost row below the lattice mirrored from row 1",
     "if (yn < 0) yn = 0;          /* mirror ghost row: zero normal */",
     "if (yn < 0) yn = 1;          /* mirror ghost row: zero normal */",
     "test_p5_stencil_periodic_x_and_mirror_rows"),
    ("Eq. 64 on D2Q9 ions: D2Q5 weights in the electrode anti-bounce-back",
     "out[k * 9 + i] = mode == 0 ? -a + 2.0 * w9[i] * v : a;",
     "out[k * 9 + i] = mode == 0 ? -a + 2.0 * w5[i % 5] * v : a;",
     "test_uniform_ions_stay_uniform_at_zero_gradient_electrodes_and_side_walls"),
    ("Eq. 64 on D2Q9 ions: sign of the electrode anti-bounce-back",
     "out[k * 9 + i] = mode == 0 ? -a + 2.0 * w9[i] * v : a;",
     "out[k * 9 + i] = mode == 0 ? a + 2.0 * w9[i] * v : a;",
     "test_ions_decay_in_the_slowest_mode_between_absorbing_electrodes"),
    ("Eq. 64 on D2Q9 ions: anti-bounce-back instead of bounce-back at a side wall",
     "                } else if (walls && (sx < 0 || sx >= c->nx)) {\n                    out[k * 9 + i] = post[k * 9 + opp9[i]];",
     "                } else if (walls && (sx < 0 || sx >= c->nx)) {\n                    out[k * 9 + i] = -post[k * 9 + opp9[i]];",
     "test_uniform_ions_stay_uniform_at_zero_gradient_electrodes_and_side_walls"),
    ("Eq. 64 on D2Q5: a side-wall link keeping its own direction",
     "                if (walls && (sx < 0 || sx >= c->nx)) {\n                    out[k * 5 + i] = post[k * 5 + opp5[i]];",
     "                if (walls && (sx < 0 || sx >= c->nx)) {\n                    out[k * 5 + i] = post[k * 5 + i];",
     "test_side_walls_potential_equals_the_mirrored_periodic_lattice"),
    ("Eq. 64: f and h periodic through the side walls",
     "if (sy < 0 || sy >= c->ny || (walls && (sx < 0 || sx >= c->nx)))",
     "if (sy < 0 || sy >= c->ny)",
     "test_side_walls_and_electrode_walls_act_alike_on_the_fluid"),
    ("Eq. 50: tau_g dropped from E_y",
     "*Ey = sy / (cs2 * tau_g);",
     "*Ey = sy / cs2;",
     "test_p9_linear_potential_between_electrodes"),
    ("Eq. 63: the y weights of the bilinear sampler swapped",
     "    return a * (1 - fy) + b * fy;",
     "    return a * fy + b * (1 - fy);",
     "test_deformation_sampler_is_exact_for_bilinear_fields"),
    ("Eq. 63: the wrong end of the crossing interval in the interpolation",
     "end = prev_t + (tt - prev_t) * (prev_v - 0.5) / (prev_v - v);",
     "end = prev_t + (tt - prev_t) * (0.5 - v) / (prev_v - v);",
     "test_deformation_factor_of_ellipses"),
    ("the MRT source factor (I - S) instead of (I - S/2)",
     "for (int k = 0; k < Q; ++k) m[k] *= (1.0 - 0.5 * s[k]);",
     "for (int k = 0; k < Q; ++k) m[k] *= (1.0 - s[k]);",
     "test_p4_momentum_and_ion_sources_exact_for_any_rates"),
    ("Eq. 43: the other root of the quadratic for B < 0",
     "c = (-B + disc) / (2.0 * lam0);",
     "c = (-B - disc) / (2.0 * lam0);",
     "test_p7_reaction_satisfies_eq41_with_eq5"),
    ("the sweep residual without its square root",
     "r = sp > 0.0 ? sqrt(sd / sp) : sqrt(sd);",
     "r = sp > 0.0 ? sd / sp : sqrt(sd);",
     "test_p9_linear_potential_between_electrodes"),
    ("Eq. 32: eps instead of eps^2 in the regularised normal",
     "double den = sqrt(gx * gx + gy * gy + eps * eps);",
     "double den = sqrt(gx * gx + gy * gy + eps);",
     "test_regularised_normal_is_the_unit_normal_away_from_flat_regions"),
    ("Sec. 2.2: cation diffusivity without the Einstein scaling",
     "double Dp = P->einstein_D ? P->D * mup / P->mu_v : P->D;",
     "double Dp = P->D;",
     "test_ion_diffusivities_follow_the_mobilities_inside_the_drop_phase"),
    ("Eq. 61: the mobility interpolated with 1 - phi",
     "double mup = P->mu_v * (1.0 + (P->mu_r - 1.0) * phi);",
     "double mup = P->mu_v * (1.0 + (P->mu_r - 1.0) * (1.0 - phi));",
     "test_ion_diffusivities_follow_the_mobilities_inside_the_drop_phase"),
    ("anion mobility without the ratio m",
     "double mum = P->m * mup;",
     "double mum = mup;",
     "test_ion_drift_moves_the_centroid_at_mobility_times_field"),
    ("Eq. 58: sign of the Euler derivative of phi u",
     "double dpux = phi * ux - c->phiu_prev[2 * k];",
     "double dpux = c->phiu_prev[2 * k] - phi * ux;",
     "test_side_walls_and_electrode_walls_act_alike_on_the_fluid"),
    ("Eq. 37: the ion relaxation time without 1/cs2",
     "rates_ion(P, Q, 0.5 + Dp / cs2, sqp);",
     "rates_ion(P, Q, 0.5 + Dp, sqp);",
     "test_ion_drift_moves_the_centroid_at_mobility_times_field"),
    ("Eq. 37: the first-moment ion rates set to 1",
     "    s[1] = s[2] = 1.0 / tau;\n}\n\n/* One",
     "    s[1] = s[2] = 1.0;\n}\n\n/* One",
     "test_ions_decay_in_the_slowest_mode_between_absorbing_electrodes"),
    ("Eq. 61: the density interpolated with 1 - phi",
     "        double rho = 1.0 + (P->rho_ratio - 1.0) * phi;\n",
     "        double rho = 1.0 + (P->rho_ratio - 1.0) * (1.0 - phi);\n",
     "test_shear_wave_inside_the_drop_phase_decays_at_eta_over_rho"),
    ("Eq. 61: the viscosity interpolated with 1 - phi",
     "double eta = eta_v * (1.0 + (P->eta_ratio - 1.0) * phi);",
     "double eta = eta_v * (1.0 + (P->eta_ratio - 1.0) * (1.0 - phi));",
     "test_shear_wave_inside_the_drop_phase_decays_at_eta_over_rho"),
    ("Eq. 55: the local tau_f without rho",
     "double tau_f = 0.5 + eta / (rho * cs2);",
     "double tau_f = 0.5 + eta / cs2;",
     "test_shear_wave_inside_the_drop_phase_decays_at_eta_over_rho"),
    ("Eq. 54: d rho / dy taken from d phi / dx",
     "double grx = (P->rho_ratio - 1.0) * gx, gry = (P->rho_ratio - 1.0) * gy;",
     "double grx = (P->rho_ratio - 1.0) * gx, gry = (P->rho_ratio - 1.0) * gx;",
     "test_flat_interface_translates_with_a_uniform_flow_along_it"),
    ("Eq. 55: cs2 dropped from the viscosity",
     "const double eta_v = cs2 * (P->tau_f - 0.5);",
     "const double eta_v = (P->tau_f - 0.5);",
     "test_shear_wave_decays_at_the_viscosity_of_tau_f"),
]


# arguments of the parametrised pins
PIN_ARGS = {"test_p15_ion_sources_carry_R_and_c_F": dict(q=5),
            "test_ions_decay_in_the_slowest_mode_between_absorbing_electrodes": dict(q=9),
            "test_uniform_ions_stay_uniform_at_zero_gradient_electrodes_and_side_walls": dict(q=9)}


def run_pin(pin):
    getattr(pins, pin)(**PIN_ARGS.get(pin, {}))


def mutant(tmp_path, old, new):
    """A separate instance of the oracle package built from the mutated source."""
    with open(oracle.SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    d = str(tmp_path)
    with open(os.path.join(d, "ehd_oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    shutil.copy(os.path.join(oracle.HERE, "ehd_oracle.h"), d)
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{tmp_path.name}",
                                                  os.path.join(oracle.HERE, "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.HERE, mod.SRC, mod.LIB = d, os.path.join(d, "ehd_oracle.c"), os.path.join(d, "libehd_oracle.so")
    return mod


@pytest.mark.parametrize("what,old,new,pin", MUTATIONS, ids=[m[3] + "/" + str(i) for i, m in enumerate(MUTATIONS)])
def test_planted_mistake_fails_a_pin(what, old, new, pin, tmp_path, monkeypatch):
    monkeypatch.setattr(pins, "O", mutant(tmp_path, old, new))
    with pytest.raises(AssertionError):
        run_pin(pin)


def test_the_unmutated_copy_passes_the_same_pins(tmp_path, monkeypatch):
    # the machinery itself: a copy built the same way without a mistake passes
    monkeypatch.setattr(pins, "O", mutant(tmp_path, "/* Eq. 52 */", "/* Eq. 52 */"))
    for pin in sorted({m[3] for m in MUTATIONS}):
        run_pin(pin)
