"""Do the oracle's pins catch plausible mistakes?  Each case plants one mistake in a copy of
the oracle source (a dropped term, a wrong sign, index or constant, a transposed operand),
builds it on the CPU and requires that at least one pin fails against it."""
import os
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
from paper_2409_06404_gb300 import synth
from conftest import P_ATM
import test_oracle_thermo as th
import test_oracle_rates as rt
import test_oracle_transport as tr
import test_oracle_derivs as dv
import test_oracle_rhs as rh
import test_oracle_diffusion as df
import test_oracle_reactor as rx
import test_oracle_rhs_jacobian as rj

SRC = open(os.path.join(os.path.dirname(oracle.__file__), "nkoracle.cpp")).read()

MUTATIONS = {
    "h_coefficient": ("hRT = S(a[0]) + S(a[1]) * T / S(2.0)", "hRT = S(a[0]) + S(a[1]) * T / S(3.0)"),
    "s_drops_a7": ("S(a[4]) * T4 / S(4.0) + S(a[6]);", "S(a[4]) * T4 / S(4.0);"),
    "nasa_range_swapped": ("(re(T) <= m.T_mid[k])", "(re(T) > m.T_mid[k])"),
    "Kc_sign": ("S Kc = exp(-sum_nu_g)", "S Kc = exp(sum_nu_g)"),
    "standard_pressure": ("const double P0 = 101325.0;", "const double P0 = 100000.0;"),
    "third_body_not_applied": ("        fwd = fwd * M;\n        rev = rev * M;\n", ""),
    "troe_0.14": ("S(0.14)", "S(0.15)"),
    "troe_n_slope": ("S(0.75) - S(1.27) * lFc", "S(0.75) - S(1.17) * lFc"),
    "troe_T2_sign": ("Fcent += exp(S(-T2) / T);", "Fcent += exp(S(T2) / T);"),
    "troe_weights_swapped": ("S(1.0 - a) * exp(-T / S(T3)) + S(a) * exp(-T / S(T1))",
                             "S(a) * exp(-T / S(T3)) + S(1.0 - a) * exp(-T / S(T1))"),
    "product_scatter_sign": ("omega[m.prod_sp[i]] += S((double)m.prod_nu[i]) * o.q;",
                             "omega[m.prod_sp[i]] -= S((double)m.prod_nu[i]) * o.q;"),
    "arrhenius_missing_R": ("exp(S(-Ea) / (S(RU) * T))", "exp(S(-Ea) / T)"),
    "arrhenius_beta_sign": ("pow(T, beta)", "pow(T, -beta)"),
    "density": ("mx.rho = S(p) * mx.Wbar / (S(RU) * T);", "mx.rho = S(p) / mx.Wbar / (S(RU) * T);"),
    "concentration_missing_W": ("mx.C[k] = mx.rho * Y[k] / S(m.W[k]);", "mx.C[k] = mx.rho * Y[k];"),
    "hrr_sign": ("hrr -= h * omega[k];", "hrr += h * omega[k];"),
    "wilke_quarter_power": ("pow(S(m.W[j] / m.W[k]), 0.25)", "pow(S(m.W[k] / m.W[j]), 0.25)"),
    "mathur_harmonic": ("lam = S(0.5) * (s1 + S(1.0) / s2);", "lam = S(0.5) * (s1 + S(1.0) * s2);"),
    "diffusion_pressure": ("* S(m.p_ref / p)", "* S(p / m.p_ref)"),
    "diffusion_numerator": ("num += mx.X[j] * S(m.W[j]);", "num += mx.X[j];"),
    "rhs_missing_W": ("fY[k] = S(m.W[k]) * w[k] / mx.rho;", "fY[k] = w[k] / mx.rho;"),
    "rhs_cp_molar": ("cp += Y[k] * S(RU) * cpR / S(m.W[k]);", "cp += Y[k] * S(RU) * cpR;"),
    "rhs_T_sign": ("fT = hrr / (mx.rho * cp);", "fT = -hrr / (mx.rho * cp);"),
    "diffusion_correction_sign": ("        Vc[c] = -sum;\n", "        Vc[c] = sum;\n"),
    "diffusion_mole_mass_ratio": ("yv[k] = -y_over_x * D[k] * gradX[c * K + k];", "yv[k] = -D[k] * gradX[c * K + k];"),
    "diffusion_flux_without_rho": ("j[c * K + k] = mx.rho * (yv[k] + Y[k] * Vc[c]);",
                                   "j[c * K + k] = (yv[k] + Y[k] * Vc[c]);"),
    "reactor_step_sign": ("G[k + 1] = x[k + 1] - x0[k + 1] - dt * fY[k].real();",
                          "G[k + 1] = x[k + 1] - x0[k + 1] + dt * fY[k].real();"),
    "reactor_jacobian_sign": ("(j == k + 1 ? 1.0 : 0.0) - dt * fY[k].imag() / hstep",
                              "(j == k + 1 ? 1.0 : 0.0) + dt * fY[k].imag() / hstep"),
    "rhs_jacobian_transposed": ("Ji[(size_t)(k + 1) * N + j] = f[k].imag() / hstep;",
                                "Ji[(size_t)j * N + k + 1] = f[k].imag() / hstep;"),
    "Kc_pressure_factor_inverted": ("ipow(S(P0) / (S(RU) * T), sum_nu)", "ipow(S(RU) * T / S(P0), sum_nu)"),
    "third_body_factor_on_troe": ("    if (m.rtype[r] == 1) {\n        fwd = fwd * M;",
                                  "    if (m.rtype[r] != 0) {\n        fwd = fwd * M;"),
    "troe_Pr_inverted": ("S Pr = k0 * M / kf;", "S Pr = kf * M / k0;"),
    "efficiencies_ignored": ("M += S(m.eff[(size_t)r * K + k]) * C[k];", "M += C[k];"),
    "cp_T2_term": ("S(a[2]) * T2 + S(a[3]) * T3", "S(a[2]) * T3 + S(a[3]) * T3"),
    "mole_fraction_inverted": ("mx.X[k] = Y[k] * mx.Wbar / S(m.W[k]);", "mx.X[k] = Y[k] * S(m.W[k]) / mx.Wbar;"),
    "rhs_jacobian_T_row_column_shift": ("            Ji[j] = ft.imag() / hstep;",
                                        "            Ji[j > 0 ? j - 1 : 0] = ft.imag() / hstep;"),
    "powers_of_magnitudes": ("    for (int i = 0; i < m; ++i) r = r * x;",
                             "    for (int i = 0; i < m; ++i) r = r * (re(x) < 0.0 ? -x : x);"),
}


def _pins():
    m9, m53, m120 = (synth.mechanism(n) for n in ("h2_9sp_21rx", "ch4_53sp_325rx", "big_120sp_700rx"))
    return [
        lambda: th.test_cp_is_dh_dT_and_ds_dT_is_cp_over_T(m53),
        lambda: th.test_continuity_at_T_mid(m53, m9),
        th.test_constant_cp_ideal_gas,
        lambda: th.test_pure_species_and_binary_mixture_state(m9),
        lambda: th.test_mixture_properties_are_mass_weighted(m53),
        lambda: th.test_heat_capacity_stays_on_the_fitted_curve(m53, m120),
        lambda: rt.test_mass_and_element_conservation("h2_9sp_21rx"),
        lambda: rt.test_zero_net_rates_at_equilibrium("h2_9sp_21rx", 2000.0, 5 * P_ATM),
        lambda: rt.test_zero_net_rates_at_equilibrium("ch4_53sp_325rx", 2500.0, P_ATM),
        lambda: rt.test_de_donder_relation("h2_9sp_21rx"),
        rt.test_arrhenius_special_values,
        rt.test_third_body_concentration,
        rt.test_negative_concentrations_enter_as_plain_powers,
        rt.test_troe_lindemann_limit,
        rt.test_troe_centre_and_limits,
        lambda: rt.test_enthalpy_shift_invariance("h2_9sp_21rx"),
        lambda: rt.test_heat_release_is_minus_sum_h_omega(m53),
        lambda: rt.test_species_relabelling(m53),
        tr.test_power_law_fits_and_pure_species_limits,
        tr.test_wilke_binary_hand_values,
        tr.test_mathur_binary_hand_value,
        lambda: tr.test_diffusion_pressure_scaling(m53),
        lambda: tr.test_hirschfelder_curtiss_textbook_form(m9),
        lambda: tr.test_mixture_values_within_species_bounds(m53),
        lambda: dv.test_jacobian_matches_central_differences("h2_9sp_21rx"),
        lambda: dv.test_grad_lnA_closed_form_and_fd("h2_9sp_21rx"),
        lambda: rh.test_mass_conservation("h2_9sp_21rx"),
        lambda: rh.test_enthalpy_conservation_at_constant_pressure("h2_9sp_21rx"),
        rh.test_pressure_scaling,
        rh.test_exothermic_reaction_heats,
        lambda: df.test_fluxes_sum_to_zero("h2_9sp_21rx"),
        df.test_binary_reduces_to_fick_in_mass_fractions,
        df.test_trace_species_and_uniform_composition,
        rx.test_isomerization_closed_form,
        rx.test_equilibrium_is_a_fixed_point,
        lambda: rj.test_columns_match_central_differences("h2_9sp_21rx"),
        lambda: rj.test_enthalpy_balance_ties_the_temperature_row("h2_9sp_21rx"),
        rj.test_isomerization_closed_form,
    ]


@pytest.fixture(scope="module")
def variants(tmp_path_factory):
    d = tmp_path_factory.mktemp("oracle_mutants")

    def make(item):
        name, (old, new) = item
        assert SRC.count(old) == 1, f"mutation {name}: snippet must occur exactly once"
        return name, oracle.build_variant(SRC.replace(old, new), str(d / f"lib_{name}.so"))

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return dict(ex.map(make, MUTATIONS.items()))


def test_unmutated_oracle_passes_every_pin():
    for pin in _pins():
        pin()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(variants, name):
    caught = 0
    with oracle.use_library(variants[name]):
        for pin in _pins():
            try:
                pin()
            except (AssertionError, ValueError, FloatingPointError):
                caught += 1
    assert caught >= 1, f"no pin fails for the planted mistake {name}"
