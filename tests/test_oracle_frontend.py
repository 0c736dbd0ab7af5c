"""Pins of the oracle's input front end (k-table interpolation, gas and cloud
mixing of Sec. 2.1.3, H2/He Rayleigh scattering of App. C), and a check that
plausible mistakes planted in a private copy of it fail at least one pin."""
import sys
import types

import numpy as np
import pytest

import oracle.frontend as FE
import rt_synth

GRAV = 47.0


def table(fe, lk_value=None, f_cloud=1e-17, x_h2=0.85, x_he=0.15, NB=6, NG=3, seed=2):
    kt = rt_synth.ktable(n_bins=NB, n_g=NG, seed=seed)
    lk = kt["log10_kappa"] if lk_value is None else np.full_like(kt["log10_kappa"], lk_value)
    return fe.KTable(T_grid=kt["T_grid"], log10p_grid=kt["log10p_grid"], log10_kappa=lk,
                     sigma_scat_cloud=kt["sigma_scat_cloud"], sigma_abs_cloud=kt["sigma_abs_cloud"],
                     g0_cloud=kt["g0_cloud"], f_cloud=f_cloud, x_h2=x_h2, x_he=x_he,
                     mbar_amu=kt["mbar_amu"]), kt["edges"]


def state(NB=6, NG=3, L=7, n=2, seed=4):
    return rt_synth.state_columns(n, L, NB, NG, seed)


# -- pins, each taking the front-end module so that mutants can be checked --

def pin_grid_nodes(fe):
    kt, _ = table(fe)
    for i, j in ((0, 0), (7, 13), (59, 27), (30, 1)):
        got = fe.log10_kappa_at(kt, kt.T_grid[i], 10.0 ** kt.log10p_grid[j])
        np.testing.assert_allclose(got, kt.log10_kappa[i, j], rtol=0, atol=1e-9)


def pin_cell_centre_is_corner_mean(fe):
    kt, _ = table(fe)
    i, j = 11, 5
    T = 0.5 * (kt.T_grid[i] + kt.T_grid[i + 1])
    p = 10.0 ** (0.5 * (kt.log10p_grid[j] + kt.log10p_grid[j + 1]))
    want = 0.25 * (kt.log10_kappa[i, j].astype(np.float64) + kt.log10_kappa[i + 1, j]
                   + kt.log10_kappa[i, j + 1] + kt.log10_kappa[i + 1, j + 1])
    np.testing.assert_allclose(fe.log10_kappa_at(kt, T, p), want, rtol=0, atol=1e-9)
    # one third of the way in T only: linear in T
    T3 = kt.T_grid[i] + (kt.T_grid[i + 1] - kt.T_grid[i]) / 3.0
    p0 = 10.0 ** kt.log10p_grid[j]
    want = (2 * kt.log10_kappa[i, j].astype(np.float64) + kt.log10_kappa[i + 1, j]) / 3.0
    np.testing.assert_allclose(fe.log10_kappa_at(kt, T3, p0), want, rtol=0, atol=1e-9)


def pin_clamped_outside_the_grid(fe):
    kt, _ = table(fe)
    np.testing.assert_allclose(fe.log10_kappa_at(kt, 1.0, 1e-12), kt.log10_kappa[0, 0], atol=1e-9)
    np.testing.assert_allclose(fe.log10_kappa_at(kt, 1e5, 1e12), kt.log10_kappa[-1, -1], atol=1e-9)


def pin_rayleigh_textbook_limit(fe):
    # n -> 1: ((n^2 - 1) / (n^2 + 2))^2 -> (2 (n - 1) / 3)^2, the textbook
    # 32 pi^3 (n - 1)^2 / (3 N^2 lambda^4) for a dilute gas
    for lam_um in (0.4, 1.0, 5.0):
        lam = lam_um * 1e-6
        n = fe.n_r_h2(lam_um)
        want = 32 * np.pi ** 3 * (n - 1) ** 2 / (3 * fe.N_REF_H2 ** 2 * lam ** 4)
        got = fe.sigma_rayleigh(lam, n, fe.N_REF_H2)
        assert abs(got / want - 1) < 3 * (n - 1)
        # transparent gases disperse normally: the index falls with wavelength
        assert fe.n_r_h2(lam_um) > fe.n_r_h2(2 * lam_um) > 1.0
        # the mixture: each gas with its own index and reference density
        for x_h2, x_he in ((1.0, 0.0), (0.0, 1.0), (0.85, 0.15)):
            nh, ne = fe.n_r_h2(lam_um), fe.n_r_he(lam_um)
            want = 32 * np.pi ** 3 / (3 * lam ** 4) * (x_h2 * (nh - 1) ** 2 / fe.N_REF_H2 ** 2
                                                       + x_he * (ne - 1) ** 2 / fe.N_REF_HE ** 2)
            assert abs(fe.sigma_gas(1e4 / lam_um, x_h2, x_he) / want - 1) < 3 * (nh - 1)


def pin_rayleigh_inverse_fourth_power(fe):
    # He's index is flat in the far infrared, so sigma ~ lambda^-4
    wn = 500.0
    r = fe.sigma_gas(wn, 0.0, 1.0) / fe.sigma_gas(wn / 2, 0.0, 1.0)
    assert abs(r - 16.0) < 1e-6
    r = fe.sigma_gas(wn, 1.0, 0.0) / fe.sigma_gas(wn / 2, 1.0, 0.0)
    assert abs(r - 16.0) < 16 * 5e-4          # H2's index still varies a little


def pin_bin_average(fe):
    # far infrared, He: sigma = C nu^4, so the bin mean is C (b^5 - a^5) / (5 (b - a))
    a, b = 100.0, 400.0
    C = fe.sigma_gas(250.0, 0.0, 1.0) / 250.0 ** 4
    want = C * (b ** 5 - a ** 5) / (5 * (b - a))
    got = fe.sigma_gas_bins(np.array([a, b]), 0.0, 1.0)[0]
    assert abs(got / want - 1) < 1e-8
    # a narrow bin's mean is the value at its centre
    got = fe.sigma_gas_bins(np.array([20000.0, 20000.02]), 0.85, 0.15)[0]
    assert abs(got / fe.sigma_gas(20000.01, 0.85, 0.15) - 1) < 1e-9


def pin_column_mass(fe):
    # a flat table, no scatterers: sum of dtau = kappa (p_bot - p_top) / g
    kt, edges = table(fe, lk_value=-2.0, f_cloud=0.0, x_h2=0.0, x_he=0.0)
    cols = state()
    o = fe.optics(kt, cols, edges, GRAV)
    L, NB, NG = 7, 6, 3
    d = o["dtau"].reshape(2, L, NB, NG)
    for c in range(2):
        p = cols.p_iface[c * (L + 1):(c + 1) * (L + 1)]
        np.testing.assert_allclose(d[c].sum(axis=0), 1e-2 * (p[-1] - p[0]) / GRAV, rtol=1e-12)
    assert np.all(o["w0"] == 0.0) and np.all(o["g0"] == 0.0)


def pin_scattering_depth_independent_of_kappa(fe):
    # dtau w0 is the scattering optical depth: it does not see kappa; the
    # absorption depth dtau (1 - w0) grows by exactly the kappa change
    cols = state()
    kt1, edges = table(fe, lk_value=-3.0)
    kt2, _ = table(fe, lk_value=-3.0 + np.log10(5.0))
    o1, o2 = fe.optics(kt1, cols, edges, GRAV), fe.optics(kt2, cols, edges, GRAV)
    np.testing.assert_allclose(o1["dtau"] * o1["w0"], o2["dtau"] * o2["w0"], rtol=1e-10)
    dp = np.concatenate([np.repeat(np.diff(cols.p_iface[c * 8:(c + 1) * 8]), 18) for c in range(2)])
    absorb = lambda o: o["dtau"] * (1 - o["w0"])
    k1 = 10.0 ** float(kt1.log10_kappa.flat[0])        # the float32 table values, widened
    k2 = 10.0 ** float(kt2.log10_kappa.flat[0])
    np.testing.assert_allclose(absorb(o2) - absorb(o1), (k2 - k1) * dp / GRAV, rtol=1e-8)
    np.testing.assert_array_equal(o1["g0"], o2["g0"])


def pin_cloud_only_and_gas_only(fe):
    cols = state()
    # no gas scattering, negligible gas absorption: the cloud's own albedo and g0
    kt, edges = table(fe, lk_value=-40.0, f_cloud=1e-17, x_h2=0.0, x_he=0.0)
    o = fe.optics(kt, cols, edges, GRAV)
    w = kt.sigma_scat_cloud / (kt.sigma_scat_cloud + kt.sigma_abs_cloud)
    np.testing.assert_allclose(o["w0"].reshape(-1, 6, 3), np.broadcast_to(w[:, None], (14, 6, 3)), rtol=1e-12)
    np.testing.assert_allclose(o["g0"].reshape(-1, 6, 3), np.broadcast_to(kt.g0_cloud[:, None], (14, 6, 3)),
                               rtol=1e-12)
    # gas only: conservative Rayleigh scattering, isotropic
    kt, edges = table(fe, lk_value=-60.0, f_cloud=0.0)
    o = fe.optics(kt, cols, edges, GRAV)
    np.testing.assert_allclose(o["w0"], 1.0, rtol=1e-12)
    assert np.all(o["g0"] == 0.0)


PINS = [pin_grid_nodes, pin_cell_centre_is_corner_mean, pin_clamped_outside_the_grid,
        pin_rayleigh_textbook_limit, pin_rayleigh_inverse_fourth_power, pin_bin_average,
        pin_column_mass, pin_scattering_depth_independent_of_kappa, pin_cloud_only_and_gas_only]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_frontend_pin(pin):
    pin(FE)


MUTATIONS = {
    "weight_flipped": ("w = (v - grid[i]) / (grid[i + 1] - grid[i])",
                       "w = (grid[i + 1] - v) / (grid[i + 1] - grid[i])"),
    "kappa_per_particle_drops_mbar": ("ext = scat[:, None] + kappa * mbar + absc[:, None]",
                                      "ext = scat[:, None] + kappa + absc[:, None]"),
    "w0_drops_cloud_scattering": ("scat = sg + kt.f_cloud * kt.sigma_scat_cloud",
                                  "scat = sg"),
    "rayleigh_lambda_squared": ("(n_ref ** 2 * lam_m ** 4)", "(n_ref ** 2 * lam_m ** 2)"),
    "g0_not_weighted": ("kt.f_cloud * kt.sigma_scat_cloud / scat * kt.g0_cloud",
                        "kt.g0_cloud + 0.0 * scat"),
    "he_reference_density": ("sigma_rayleigh(lam_m, n_r_he(lam_um), N_REF_HE)",
                             "sigma_rayleigh(lam_m, n_r_he(lam_um), N_REF_H2)"),
    "h2_index_dispersion_sign": ("(1.0 + 7.52e-3 / lam_um ** 2)", "(1.0 - 7.52e-3 / lam_um ** 2)"),
    "dtau_drops_gravity": ("(p_bot - p_top) / grav", "(p_bot - p_top)"),
}


def mutant(old, new):
    src = open(FE.__file__).read()
    assert src.count(old) == 1, old
    m = types.ModuleType("frontend_mutant")
    sys.modules["frontend_mutant"] = m          # dataclasses look their module up
    try:
        exec(compile(src.replace(old, new), "frontend_mutant", "exec"), m.__dict__)
    finally:
        del sys.modules["frontend_mutant"]
    return m


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name):
    m = mutant(*MUTATIONS[name])
    failed = []
    for pin in PINS:
        try:
            pin(m)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutation {name} passed every pin"
