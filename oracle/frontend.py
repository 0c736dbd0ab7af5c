"""FP64 oracle of the input front end: k-table interpolation and the mixing
of gas and cloud optics into (dtau, w0, g0) per layer, bin and g-point.

TEST INFRASTRUCTURE ONLY.  The product library never imports or calls this
module; only the test suite, the smoke check and the benchmark's CPU leg do.
It shares no code with the CUDA path.

What it computes (Deitrick et al., arXiv 2203.02293):
  * the premixed absorption opacity kappa(T, p) per bin and g-point is read
    from a k-table on a (T, log p) grid (Sec. 2.1.3: 60 temperatures, 28
    pressures log-spaced).  The paper does not say how the GCM interpolates
    the table; this oracle (and the CUDA path) take bilinear interpolation of
    log10 kappa in (T, log10 p), with T and p clamped to the grid;
  * the layer's temperature is its centre temperature and its pressure the
    geometric mean of its interface pressures (a reading: the GCM's own
    layer-centre pressure is not an input of the solver);
  * gas scattering is Rayleigh scattering by H2 and He (App. C), the number-
    fraction-weighted sum of the two cross sections, averaged over the bin
    in wavenumber (Sec. 2.1.3: per-bin averages when k-tables are used);
  * w0 and g0 follow Eqs. 17-18 (Sec. 2.1.3): extinction per gas particle
    sigma_scat,gas + kappa mbar + f_cloud (sigma_abs,cloud +
    sigma_scat,cloud); gas scatters isotropically; kappa is the premixed
    opacity of Eq. 16, already summed over species in the table;
  * the layer optical depth is that extinction per unit mass times the layer
    column mass dp / g.
Where the scattering cross section is zero, g0 is 0 (no scatterers).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy import integrate

AMU = 1.66053906660e-27          # kg (CODATA 2018)
N_REF_H2 = 2.68678e19 * 1.0e6    # m^-3 (App. C)
N_REF_HE = 2.546899e19 * 1.0e6   # m^-3 (App. C)


def n_r_h2(lam_um):
    """Real refractive index of H2 (App. C), lambda in um."""
    return 1.358e-4 * (1.0 + 7.52e-3 / lam_um ** 2) + 1.0


def n_r_he(lam_um):
    """Real refractive index of He (App. C), lambda in um."""
    return 1.0e-8 * (2283.0 + 1.8102e13 / (1.5342e10 - lam_um ** -2)) + 1.0


def sigma_rayleigh(lam_m, n_r, n_ref, king=1.0):
    """Rayleigh cross section per molecule (m^2), App. C."""
    f = (n_r ** 2 - 1.0) / (n_r ** 2 + 2.0)
    return 24.0 * np.pi ** 3 / (n_ref ** 2 * lam_m ** 4) * f * f * king


def sigma_gas(wn_cm, x_h2, x_he):
    """Number-fraction-weighted H2 + He Rayleigh cross section at wavenumber wn (cm^-1)."""
    lam_m = 1.0e-2 / wn_cm
    lam_um = 1.0e4 / wn_cm
    return (x_h2 * sigma_rayleigh(lam_m, n_r_h2(lam_um), N_REF_H2)
            + x_he * sigma_rayleigh(lam_m, n_r_he(lam_um), N_REF_HE))


def sigma_gas_bins(edges_cm, x_h2, x_he):
    """Bin averages (in wavenumber) of the gas scattering cross section."""
    out = np.empty(len(edges_cm) - 1)
    for b in range(out.size):
        lo, hi = float(edges_cm[b]), float(edges_cm[b + 1])
        v, _ = integrate.quad(sigma_gas, lo, hi, args=(x_h2, x_he), epsabs=0.0, epsrel=1e-12,
                              limit=200)
        out[b] = v / (hi - lo)
    return out


@dataclass
class KTable:
    """A premixed k-table with the per-bin cloud and gas data."""
    T_grid: np.ndarray            # [nT] K, increasing
    log10p_grid: np.ndarray       # [nP] log10(p / Pa), increasing
    log10_kappa: np.ndarray       # [nT, nP, NB, NG] log10 (m^2 kg^-1), float32 values
    sigma_scat_cloud: np.ndarray  # [NB] m^2 per cloud particle
    sigma_abs_cloud: np.ndarray   # [NB]
    g0_cloud: np.ndarray          # [NB]
    f_cloud: float = 1e-17        # cloud-to-gas number ratio (Sec. 2.1.3)
    x_h2: float = 0.85
    x_he: float = 0.15
    mbar_amu: float = 2.34        # Table 3


def bracket(grid, v):
    """Lower index i and weight w with v = (1 - w) grid[i] + w grid[i + 1], v clamped."""
    n = len(grid)
    v = min(max(v, grid[0]), grid[-1])
    i = int(np.searchsorted(grid, v, side="right")) - 1
    i = min(max(i, 0), n - 2)
    w = (v - grid[i]) / (grid[i + 1] - grid[i])
    return i, w


def log10_kappa_at(kt: KTable, T, p):
    """Bilinear interpolation of log10 kappa at (T, log10 p): [NB, NG]."""
    i, wt = bracket(kt.T_grid, T)
    j, wp = bracket(kt.log10p_grid, np.log10(p))
    tab = kt.log10_kappa.astype(np.float64)
    return ((1 - wt) * (1 - wp) * tab[i, j] + (1 - wt) * wp * tab[i, j + 1]
            + wt * (1 - wp) * tab[i + 1, j] + wt * wp * tab[i + 1, j + 1])


def optics(kt: KTable, cols, edges_cm, grav):
    """dtau, w0, g0 (FP64) in the cube layout [column][layer][bin][g].

    ``cols`` carries n_layers, n_bins, T_center and p_iface (the column
    state); ``edges_cm`` are the bin edges shared by every column."""
    sg = sigma_gas_bins(edges_cm, kt.x_h2, kt.x_he)
    mbar = kt.mbar_amu * AMU
    scat = sg + kt.f_cloud * kt.sigma_scat_cloud                    # [NB] per gas particle
    absc = kt.f_cloud * kt.sigma_abs_cloud
    with np.errstate(invalid="ignore", divide="ignore"):
        g0b = np.where(scat > 0, kt.f_cloud * kt.sigma_scat_cloud / scat * kt.g0_cloud, 0.0)
    out = {k: [] for k in ("dtau", "w0", "g0")}
    lay = 0
    iface = 0
    for c in range(len(cols.n_layers)):
        L = int(cols.n_layers[c])
        NB = int(cols.n_bins[c])
        for l in range(L):
            T = float(cols.T_center[lay + l])
            p_top, p_bot = float(cols.p_iface[iface + l]), float(cols.p_iface[iface + l + 1])
            kappa = 10.0 ** log10_kappa_at(kt, T, np.sqrt(p_top * p_bot))   # [NB, NG]
            ext = scat[:, None] + kappa * mbar + absc[:, None]              # per gas particle
            out["dtau"].append((ext / mbar * (p_bot - p_top) / grav).ravel())
            out["w0"].append((scat[:, None] / ext).ravel())
            out["g0"].append(np.broadcast_to(g0b[:, None], ext.shape).ravel())
            assert NB == kappa.shape[0]
        lay += L
        iface += L + 1
    return {k: np.concatenate(v) for k, v in out.items()}
