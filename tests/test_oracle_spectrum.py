"""Pins of the oracle's explicit bin edges and per-bin TOA spectrum (the
post-processing shape of Sec. 2.1.3: R = 500 opacity sampling, one g-point
per bin), and of the isothermal extension above the model top (Sec. 3 run
protocol) in the input generator.

The per-bin TOA values are checked against closed forms that do not go
through the oracle's own Planck routine: an opaque isothermal column emits
pi B(T) in every bin and a transparent one passes pi B(T_int) through, with
B integrated by scipy's adaptive quadrature over the bin's own edges.
"""
import numpy as np
import pytest
from scipy import integrate

import oracle
import rt_synth

H, C, KB = 6.62607015e-34, 299792458.0, 1.380649e-23


def planck_quad(T, lo, hi):
    """Integral of B_nu over [lo, hi] cm^-1 (W m^-2 sr^-1), adaptive quadrature."""
    f = lambda nu: 2 * H * C ** 2 * nu ** 3 / np.expm1(H * C * nu / (KB * T))
    v, _ = integrate.quad(f, lo * 100.0, hi * 100.0, epsabs=0.0, epsrel=1e-13, limit=200)
    return v


def uniform_column_batch(edges, L, n_g, T, dtau, T_int, mu=0.0, w0=0.0):
    NB = len(edges) - 1
    n = L * NB * n_g
    gx, gw = rt_synth.gauss_legendre_01(n_g)
    consts = dict(rt_synth._consts(), wn_edges=np.asarray(edges, np.float64), T_int=T_int)
    return rt_synth.Columns(
        n_layers=np.array([L], np.int32), n_bins=np.array([NB], np.int32), n_g=n_g,
        g_weights=gw, dtau=np.full(n, dtau, np.float32), w0=np.full(n, w0, np.float32),
        g0=np.zeros(n, np.float32), T_center=np.full(L, T), T_iface=np.full(L + 1, T),
        p_iface=np.geomspace(1.0, 1e7, L + 1), mu_star=np.array([mu]),
        F_star=np.zeros(NB), consts=consts)


def solve(orc, cols, **kw):
    cfg = oracle.OracleConfig(T_int=cols.consts["T_int"], wn_edges=cols.consts.get("wn_edges"), **kw)
    return orc.solve_columns(cfg, cols)


EDGES = np.array([50.0, 61.0, 400.0, 1234.5, 1250.0, 5000.0, 12000.0, 33333.0])


@pytest.mark.parametrize("iso", [False, True])
def test_opaque_isothermal_column_emits_pi_B_per_bin(orc, iso):
    T = 1100.0
    cols = uniform_column_batch(EDGES, 3, 2, T, 60.0, T_int=100.0)
    out = solve(orc, cols, isothermal=iso)
    want = np.array([np.pi * planck_quad(T, a, b) for a, b in zip(EDGES[:-1], EDGES[1:])])
    np.testing.assert_allclose(out["F_up_toa"], want, rtol=1e-11)


def test_transparent_column_passes_the_boa_spectrum(orc):
    T_int = 1500.0
    cols = uniform_column_batch(EDGES, 4, 3, 20.0, 1e-9, T_int=T_int)
    out = solve(orc, cols)
    want = np.array([np.pi * planck_quad(T_int, a, b) for a, b in zip(EDGES[:-1], EDGES[1:])])
    np.testing.assert_allclose(out["F_up_toa"], want, rtol=1e-7)


def test_uniform_edges_given_explicitly_reproduce_the_uniform_bins(orc):
    cols = rt_synth.generate([6, 9], [5, 5], 3, seed=31, optics="ktable")
    base = orc.solve_columns(oracle.OracleConfig(), cols)
    edges = np.linspace(rt_synth.WN_MIN, rt_synth.WN_MAX, 6)
    expl = orc.solve_columns(oracle.OracleConfig(wn_edges=edges), cols)
    for k in ("F_up", "F_down", "F_net", "Q", "F_up_toa"):
        np.testing.assert_allclose(expl[k], base[k], rtol=1e-12, atol=1e-12 * np.abs(base[k]).max())


def test_toa_spectrum_adds_up_to_the_toa_flux(orc):
    cols = rt_synth.generate([7, 3, 12], [4, 9, 2], 5, seed=32, optics="ktable")
    out = orc.solve_columns(oracle.OracleConfig(), cols)
    o = cols.offsets()
    for c in range(cols.n_cols):
        s = out["F_up_toa"][o["bins"][c]:o["bins"][c + 1]].sum()
        assert abs(s - out["F_up"][o["iface"][c]]) <= 1e-13 * abs(s)


def test_toa_spectrum_is_the_weighted_sum_of_the_systems(orc):
    cols = rt_synth.generate([5, 8], [3, 6], 4, seed=33, optics="ktable")
    out = orc.solve_columns(oracle.OracleConfig(), cols, per_system=True)
    o = cols.offsets()
    k = 0
    for c in range(cols.n_cols):
        L, NB, G = int(cols.n_layers[c]), int(cols.n_bins[c]), cols.n_g
        base = int(((cols.n_layers[:c].astype(np.int64) + 1) * cols.n_bins[:c]).sum()) * G
        top = out["sys_up"][base:base + NB * G].reshape(NB, G)     # interface 0 = TOA
        want = top @ cols.g_weights
        np.testing.assert_allclose(out["F_up_toa"][o["bins"][c]:o["bins"][c + 1]], want, rtol=1e-14)
        k += NB
    assert k == out["F_up_toa"].size


def test_explicit_edges_must_match_the_bin_count(orc):
    cols = rt_synth.generate([4], [5], 2, seed=34)
    with pytest.raises(ValueError):
        orc.solve_columns(oracle.OracleConfig(wn_edges=np.linspace(50, 100, 5)), cols)


def test_postproc_grid_is_R500_log_spaced():
    e = rt_synth.postproc_edges()
    assert e.size == 3256 and e[0] == pytest.approx(rt_synth.WN_MIN) and e[-1] == pytest.approx(rt_synth.WN_MAX)
    lam = 1e4 / e
    R = lam[:-1] / (lam[:-1] - lam[1:])
    assert np.allclose(R, R[0]) and 495.0 < R[0] < 505.0


def test_isothermal_extension_above_the_model_top():
    rng = np.random.default_rng(7)
    p_if, Tc, Ti = rt_synth.column_profile(rng, 10, 1e-3)
    p2, Tc2, Ti2, n = rt_synth.extend_isothermal(p_if, Tc, Ti, 1e-6, 4)
    assert n == 12 and p2.size == p_if.size + n and Tc2.size == Tc.size + n
    assert p2[0] == pytest.approx(1e-6 * 1e5) and np.all(np.diff(p2) > 0)
    np.testing.assert_array_equal(p2[n:], p_if)
    np.testing.assert_array_equal(Tc2[n:], Tc)
    np.testing.assert_array_equal(Ti2[n:], Ti)
    assert np.all(Tc2[:n] == Tc[0]) and np.all(Ti2[:n] == Tc[0])
    # a column already reaching 1 ubar is left as it is
    p_if, Tc, Ti = rt_synth.column_profile(rng, 10, 1e-7)
    p3, _, _, n3 = rt_synth.extend_isothermal(p_if, Tc, Ti, 1e-6, 4)
    assert n3 == 0 and p3 is p_if
