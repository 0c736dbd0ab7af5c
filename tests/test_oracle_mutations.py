"""The pins catch plausible mistakes.

Each case plants one mistake in a private copy of the oracle source (on the
CPU, in a temporary directory), compiles it, and checks that at least one pin
of tests/test_oracle_pins.py fails against it.  The oracle itself is never
modified.
"""
import os

import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_spectrum as spec

MUTATIONS = {
    "mu_star_sign": ("double mus = -mu;   /* Malik sign", "double mus = mu;   /* Malik sign"),
    "drop_planck_gradient": ("S_up = Pi * (Bt * (chi + xi) - psi * Bb + Bp * Theta);",
                             "S_up = Pi * (Bt * (chi + xi) - psi * Bb + 0.0 * Theta);"),
    "swap_psi_xi_in_block_A": ("a[0] = -r->psi;", "a[0] = -r->xi;"),
    "e_fit_cross_term_sign": ("+ 0.2351 * w0 * g0", "- 0.2351 * w0 * g0"),
    "beer_law_scale": ("exp(w->tau[i] / mus)", "exp(w->tau[i] / (2.0 * mus))"),
    "back_substitution_sign": ("X[2 * i] = Dp[2 * i] - cx[0];", "X[2 * i] = Dp[2 * i] + cx[0];"),
    "big_pi_denominator": ("OR_PI * (1.0 - w0) / (E - w0)", "OR_PI * (1.0 - w0) / E"),
    "g_factor_tail_sign": ("*Gp = 0.5 * (lead * (mus + 1.0 / (2.0 * E * one_m_wg)) + tail);",
                           "*Gp = 0.5 * (lead * (mus + 1.0 / (2.0 * E * one_m_wg)) - tail);"),
    "transmission_exponent": ("double T = exp(-2.0 * sqrt(", "double T = exp(-1.0 * sqrt("),
    "etau_fallback_off": ("if (dtau < (double)1e-4f) {", "if (dtau < 0.0) {"),
    "boa_drops_beam": ("d[0] = F_BOA + w->Fb[0];", "d[0] = F_BOA;"),
    "spectral_sum_drops_beam": ("sum_dn[i] += wg * (fd[lev] + fb[lev]);", "sum_dn[i] += wg * fd[lev];"),
    "heating_sign": ("(net[l + 1] - net[l]) / (p[l + 1] - p[l])", "(net[l] - net[l + 1]) / (p[l + 1] - p[l])"),
    "planck_wien": ("nu * nu * nu / expm1(x);", "nu * nu * nu / exp(x);"),
    "zeta_minus_sign": ("c->zeta_m = 0.5 * (1.0 - c->k);", "c->zeta_m = 0.5 * (1.0 + c->k);"),
    "sublayer_full_depth": ("w->dtau_s[2 * j + h] = 0.5 * d;", "w->dtau_s[2 * j + h] = d;"),
    "toa_spectrum_at_boa": ("toa_b += wg * fu[cfg->isothermal ? L : 2 * L];", "toa_b += wg * fu[0];"),
    "explicit_edge_shift": ("lo = cfg->wn_edges[b];", "lo = cfg->wn_edges[b > 0 ? b - 1 : 0];"),
}


def battery(orc):
    """Run the pins against ``orc``; return the names of those that fail."""
    checks = [
        ("planck_sum", lambda: pins.test_planck_bins_sum_to_sigma_T4_over_pi(orc, 800.0)),
        ("dense_lu", lambda: pins.test_block_thomas_matches_dense_lu(orc, False, 3)),
        ("ode_noniso", lambda: pins.test_column_matches_two_stream_ode(orc, False, True, 30.0)),
        ("ode_iso", lambda: pins.test_column_matches_two_stream_ode(orc, True, True, 60.0)),
        ("ode_regular", lambda: pins.test_column_matches_two_stream_ode(orc, False, False, 0.0)),
        ("ode_thin", lambda: pins.test_column_matches_ode_with_thin_sublayers(orc)),
        ("beer", lambda: pins.test_pure_absorption_beam_is_beer_law(orc, False)),
        ("conservation", lambda: pins.test_pure_scattering_conserves_net_flux(orc, False)),
        ("batch", lambda: pins.test_batch_matches_ode_and_quadrature(orc, False)),
        ("telescoping", lambda: pins.test_heating_telescopes_to_boundary_net_fluxes(orc)),
        ("toa_opaque", lambda: spec.test_opaque_isothermal_column_emits_pi_B_per_bin(orc, False)),
        ("toa_transparent", lambda: spec.test_transparent_column_passes_the_boa_spectrum(orc)),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_battery():
    assert battery(oracle.get()) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = os.path.join(tmp_path, "rt_oracle_mut.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = oracle.build(path, os.path.join(tmp_path, "libmut.so"))
    failed = battery(oracle.Oracle(lib))
    assert failed, f"planted mistake {name} went unnoticed"


# The iterative method (Sec. 2.2.2) has its own pins (tests/test_oracle_sweeps.py).
SWEEP_MUTATIONS = {
    "sweep_xi_sign": ("dn[s] = (r->S_dn + r->psi * dn[s + 1] - r->xi * up[s]) / r->chi;",
                      "dn[s] = (r->S_dn + r->psi * dn[s + 1] + r->xi * up[s]) / r->chi;"),
    "sweep_boa_drops_beam": ("up[0] = dn[0] + F_BOA + w->Fb[0];", "up[0] = dn[0] + F_BOA;"),
    "sweep_wrong_level": ("up[s + 1] = (r->S_up + r->psi * up[s] - r->xi * dn[s + 1]) / r->chi;",
                          "up[s + 1] = (r->S_up + r->psi * up[s] - r->xi * dn[s]) / r->chi;"),
    "sweep_drops_toa": ("dn[n] = cfg->F_toa;", "dn[n] = 0.0;"),
    "sweep_psi_for_chi": ("dn[s] = (r->S_dn + r->psi * dn[s + 1] - r->xi * up[s]) / r->chi;",
                          "dn[s] = (r->S_dn + r->chi * dn[s + 1] - r->xi * up[s]) / r->psi;"),
}


def sweep_battery(orc):
    import test_oracle_sweeps as sw
    checks = [
        ("no_scattering", lambda: sw.test_one_sweep_is_exact_without_scattering(orc, False)),
        ("fixed_point", lambda: sw.test_block_solution_is_a_fixed_point(orc, False)),
        ("gauss_seidel", lambda: sw.test_sweeps_are_gauss_seidel_on_the_block_rows(orc, True, 2)),
        ("converge", lambda: sw.test_sweeps_converge_to_the_block_solution(orc, False)),
    ]
    failed = []
    for name, fn in checks:
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_sweep_battery():
    assert sweep_battery(oracle.get()) == []


@pytest.mark.parametrize("name", sorted(SWEEP_MUTATIONS))
def test_planted_sweep_mistake_is_caught(tmp_path, name):
    old, new = SWEEP_MUTATIONS[name]
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    path = os.path.join(tmp_path, "rt_oracle_mut.c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    lib = oracle.build(path, os.path.join(tmp_path, "libmut.so"))
    failed = sweep_battery(oracle.Oracle(lib))
    assert failed, f"planted mistake {name} went unnoticed"
