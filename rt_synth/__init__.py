"""Seeded synthetic inputs for the column radiative-transfer solver.

This module only draws inputs.  It holds none of the solver's arithmetic and
is the one piece of code that the oracle side and the CUDA side share.

The paper's WASP-43b opacities (HELIOS-K k-tables, Sec. 2.1.3) and PHOENIX
stellar template (Sec. 2.1.5) are not available, so seeded random inputs with
the paper's shapes stand in for them:

* 2562 columns (icosahedral g_level = 4, Sec. 2.1.1), 40 layers, 30 bins
  uniform in wavenumber over 0.3-200 um, 20 Gauss points per bin (Sec. 2.1.3);
* pressure log-spaced from 1e-6 to 100 bar (layer 0 at the top);
* T linear in log p from 800 K (top) to 2000 K (bottom) plus N(0, 50 K) per
  layer centre; interface T linear in log p between centres, extrapolated at
  the ends (Sec. 2.2.1);
* cos(theta*) uniform in [0.1, 1] per column;
* g = 47 m s^-2, c_P = 12436 J kg^-1 K^-1, eps2 = 2/3, T_int = 100 K
  (Table 3, Sec. 3.1);
* stellar flux per bin: a 4798 K blackbody (Table 3) evaluated at the bin
  centre times the bin width, times pi (R*/a)^2 -- a crude stand-in for the
  bin-averaged PHOENIX template.

Layout: cubes are float32 ``[column][layer][bin][g]`` with g fastest, columns
packed back to back; per-column arrays are float64.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field, replace

import numpy as np

WN_MIN = 50.0            # cm^-1  (200 um)
WN_MAX = 1.0e4 / 0.3     # cm^-1  (0.3 um)
GRAV = 47.0
CP = 12436.0
EPS2 = 2.0 / 3.0
T_INT = 100.0
T_STAR = 4798.0
R_STAR = 4.64e8
A_ORBIT = 2.28e9
P_TOP_BAR = 1e-6
P_BOT_BAR = 100.0

_H, _C, _KB = 6.62607015e-34, 299792458.0, 1.380649e-23


@dataclass
class Columns:
    """A packed batch of atmospheric columns (host arrays)."""
    n_layers: np.ndarray        # int32 [C]
    n_bins: np.ndarray          # int32 [C]
    n_g: int
    g_weights: np.ndarray       # float64 [n_g], sum = 1
    dtau: np.ndarray            # float32 [sum L_c*NB_c*n_g]
    w0: np.ndarray              # float32, same layout
    g0: np.ndarray              # float32, same layout
    T_center: np.ndarray        # float64 [sum L_c]
    T_iface: np.ndarray         # float64 [sum (L_c+1)]
    p_iface: np.ndarray         # float64 [sum (L_c+1)], Pa
    mu_star: np.ndarray         # float64 [C]
    F_star: np.ndarray          # float64 [sum NB_c], W m^-2 normal to the beam
    consts: dict = field(default_factory=dict)
    name: str = ""

    @property
    def n_cols(self) -> int:
        return int(self.n_layers.size)

    @property
    def n_systems(self) -> int:
        return int((self.n_bins.astype(np.int64) * self.n_g).sum())

    def offsets(self):
        L = self.n_layers.astype(np.int64)
        NB = self.n_bins.astype(np.int64)
        z = lambda a: np.concatenate([[0], np.cumsum(a)])
        return dict(cube=z(L * NB * self.n_g), lay=z(L), iface=z(L + 1), bins=z(NB))

    def subset(self, idx) -> "Columns":
        """The columns ``idx`` (in that order) as a new packed batch."""
        idx = np.asarray(idx, dtype=np.int64)
        o = self.offsets()
        cat = lambda a, key: np.concatenate([a[o[key][i]:o[key][i + 1]] for i in idx]) \
            if idx.size else a[:0]
        return replace(self, n_layers=self.n_layers[idx].copy(), n_bins=self.n_bins[idx].copy(),
                       dtau=cat(self.dtau, "cube"), w0=cat(self.w0, "cube"),
                       g0=cat(self.g0, "cube"), T_center=cat(self.T_center, "lay"),
                       T_iface=cat(self.T_iface, "iface"), p_iface=cat(self.p_iface, "iface"),
                       mu_star=self.mu_star[idx].copy(), F_star=cat(self.F_star, "bins"),
                       name=self.name + f"[{idx.size} cols]")

    @property
    def nbytes_inputs(self) -> int:
        return sum(a.nbytes for a in (self.dtau, self.w0, self.g0, self.T_center,
                                      self.T_iface, self.p_iface, self.mu_star, self.F_star))


def gauss_legendre_01(n: int):
    """Gauss-Legendre nodes and weights on [0, 1]; weights sum to 1."""
    if n == 1:
        return np.array([0.5]), np.array([1.0])
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def stellar_flux_bins(n_bins: int, wn_min: float = WN_MIN, wn_max: float = WN_MAX):
    """Stand-in stellar spectrum per bin, W m^-2 normal to the beam."""
    edges = np.linspace(wn_min, wn_max, n_bins + 1) * 100.0    # m^-1
    mid = 0.5 * (edges[1:] + edges[:-1])
    width = np.diff(edges)
    x = _H * _C * mid / (_KB * T_STAR)
    b_mid = 2.0 * _H * _C ** 2 * mid ** 3 / np.expm1(x)
    return np.pi * b_mid * width * (R_STAR / A_ORBIT) ** 2


def _profile(rng, L: int, p_top_bar: float = P_TOP_BAR):
    """Pressure grid (Pa) and temperatures of one column, layer 0 at the top."""
    lp = np.linspace(np.log(p_top_bar), np.log(P_BOT_BAR), L + 1)
    p_if = np.exp(lp) * 1.0e5
    lpc = 0.5 * (lp[1:] + lp[:-1])
    frac = (lpc - lp[0]) / (lp[-1] - lp[0])
    Tc = 800.0 + 1200.0 * frac + rng.normal(0.0, 50.0, L)
    Ti = np.empty(L + 1)
    if L == 1:
        Ti[:] = Tc[0]
    else:
        Ti[1:L] = Tc[:-1] + (Tc[1:] - Tc[:-1]) * (lp[1:L] - lpc[:-1]) / (lpc[1:] - lpc[:-1])
        Ti[0] = Tc[0] + (Tc[1] - Tc[0]) * (lp[0] - lpc[0]) / (lpc[1] - lpc[0])
        Ti[L] = Tc[-2] + (Tc[-1] - Tc[-2]) * (lp[L] - lpc[-2]) / (lpc[-1] - lpc[-2])
    Ti = np.maximum(Ti, 10.0)
    Tc = np.maximum(Tc, 10.0)
    return p_if, Tc, Ti


def _consts():
    return dict(T_int=T_INT, grav=GRAV, cp=CP, eps2=EPS2, wn_min=WN_MIN, wn_max=WN_MAX)


def generate(n_layers, n_bins, n_g: int, seed: int, optics: str = "uniform",
             name: str = "", mu_range=(0.1, 1.0)) -> Columns:
    """Draw a packed batch.

    optics:
      "uniform"  dtau ~ logU[1e-6, 10], w0 ~ U[0, 0.95], g0 ~ U[0, 0.8]
      "ktable"   k ~ logU[1e-8, 1] m^2/kg sorted ascending over g within each
                 (column, layer, bin); dtau = k dp / g; w0, g0 as "uniform"
      "stress"   dtau ~ logU[1e-8, 1e4], w0 ~ U[0.99, 1-1e-6], g0 ~ U[0.5, 0.95]
    """
    rng = np.random.default_rng(seed)
    n_layers = np.asarray(n_layers, dtype=np.int32)
    n_bins = np.asarray(n_bins, dtype=np.int32)
    C = n_layers.size
    gx, gw = gauss_legendre_01(n_g)
    Tc_all, Ti_all, p_all, Fs_all = [], [], [], []
    cubes = {k: [] for k in ("dtau", "w0", "g0")}
    mu = rng.uniform(mu_range[0], mu_range[1], C)
    fs_cache = {}
    for c in range(C):
        L, NB = int(n_layers[c]), int(n_bins[c])
        p_if, Tc, Ti = _profile(rng, L)
        shape = (L, NB, n_g)
        if optics == "uniform":
            dtau = np.exp(rng.uniform(np.log(1e-6), np.log(10.0), shape))
            w0 = rng.uniform(0.0, 0.95, shape)
            g0 = rng.uniform(0.0, 0.8, shape)
        elif optics == "ktable":
            k = np.sort(rng.uniform(np.log(1e-8), np.log(1.0), shape), axis=-1)
            dp = np.diff(p_if)[:, None, None]
            dtau = np.exp(k) * dp / GRAV
            w0 = rng.uniform(0.0, 0.95, shape)
            g0 = rng.uniform(0.0, 0.8, shape)
        elif optics == "stress":
            dtau = np.exp(rng.uniform(np.log(1e-8), np.log(1e4), shape))
            w0 = rng.uniform(0.99, 1.0 - 1e-6, shape)
            g0 = rng.uniform(0.5, 0.95, shape)
        else:
            raise ValueError(optics)
        cubes["dtau"].append(dtau.astype(np.float32).ravel())
        cubes["w0"].append(w0.astype(np.float32).ravel())
        cubes["g0"].append(g0.astype(np.float32).ravel())
        Tc_all.append(Tc); Ti_all.append(Ti); p_all.append(p_if)
        if NB not in fs_cache:
            fs_cache[NB] = stellar_flux_bins(NB)
        Fs_all.append(fs_cache[NB])
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
    return Columns(n_layers=n_layers, n_bins=n_bins, n_g=n_g, g_weights=gw,
                   dtau=cat(cubes["dtau"], np.float32), w0=cat(cubes["w0"], np.float32),
                   g0=cat(cubes["g0"], np.float32), T_center=cat(Tc_all, np.float64),
                   T_iface=cat(Ti_all, np.float64), p_iface=cat(p_all, np.float64),
                   mu_star=mu, F_star=cat(Fs_all, np.float64), consts=_consts(), name=name)


def generate_fast(n_cols: int, L: int, NB: int, n_g: int, seed: int, optics: str,
                  name: str = "") -> Columns:
    """Uniform-shape batch drawn with whole-array numpy calls (large configs)."""
    rng = np.random.default_rng(seed)
    gx, gw = gauss_legendre_01(n_g)
    prof = [_profile(rng, L) for _ in range(n_cols)]
    p_if = np.stack([p[0] for p in prof])
    Tc = np.stack([p[1] for p in prof])
    Ti = np.stack([p[2] for p in prof])
    mu = rng.uniform(0.1, 1.0, n_cols)
    shape = (n_cols, L, NB, n_g)
    if optics == "ktable":
        k = rng.uniform(np.log(1e-8), np.log(1.0), shape).astype(np.float32)
        k.sort(axis=-1)
        dp = (np.diff(p_if, axis=1) / GRAV).astype(np.float32)[:, :, None, None]
        dtau = (np.exp(k) * dp).astype(np.float32)
        del k
        w0 = rng.uniform(0.0, 0.95, shape).astype(np.float32)
        g0 = rng.uniform(0.0, 0.8, shape).astype(np.float32)
    elif optics == "stress":
        dtau = np.exp(rng.uniform(np.log(1e-8), np.log(1e4), shape)).astype(np.float32)
        w0 = rng.uniform(0.99, 1.0 - 1e-6, shape).astype(np.float32)
        g0 = rng.uniform(0.5, 0.95, shape).astype(np.float32)
    elif optics == "uniform":
        dtau = np.exp(rng.uniform(np.log(1e-6), np.log(10.0), shape)).astype(np.float32)
        w0 = rng.uniform(0.0, 0.95, shape).astype(np.float32)
        g0 = rng.uniform(0.0, 0.8, shape).astype(np.float32)
    else:
        raise ValueError(optics)
    return Columns(n_layers=np.full(n_cols, L, np.int32), n_bins=np.full(n_cols, NB, np.int32),
                   n_g=n_g, g_weights=gw, dtau=dtau.ravel(), w0=w0.ravel(), g0=g0.ravel(),
                   T_center=Tc.ravel(), T_iface=Ti.ravel(), p_iface=p_if.ravel(),
                   mu_star=mu, F_star=np.tile(stellar_flux_bins(NB), n_cols),
                   consts=_consts(), name=name)


# ----------------------------------------------------------------------
# The five workloads.
# ----------------------------------------------------------------------

# The workloads' shapes, distributions and seeds (configs.json); the
# functions below take their defaults from it.
with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "configs.json")) as _f:
    CONFIGS = json.load(_f)


def config0(seed: int | None = None) -> Columns:
    """Plain FP64 case: 64 x 40 layers x 30 bins x 1 g-point, seed 0."""
    c = CONFIGS["config0"]
    n, L, NB = c["n_cols"], c["layers"], c["bins"]
    return generate([L] * n, [NB] * n, c["g_points"], c["seed"] if seed is None else seed, c["optics"],
                    name=f"config0 {n}x{L}x{NB}x{c['g_points']}")


def config1(n_cols: int | None = None, seed: int | None = None) -> Columns:
    """GCM-shaped: 2562 x 40 x 30 x 20 Gauss points, k-table optical depths."""
    c = CONFIGS["config1"]
    n = c["n_cols"] if n_cols is None else n_cols
    return generate_fast(n, c["layers"], c["bins"], c["g_points"], c["seed"] if seed is None else seed,
                         c["optics"], name=f"config1 {n}x{c['layers']}x{c['bins']}x{c['g_points']}")


def config2(n_cols: int | None = None, seed: int | None = None) -> Columns:
    """Precision stress: w0 in [0.99, 1-1e-6], dtau in [1e-8, 1e4], g0 in [0.5, 0.95]."""
    c = CONFIGS["config2"]
    n = c["n_cols"] if n_cols is None else n_cols
    return generate_fast(n, c["layers"], c["bins"], c["g_points"], c["seed"] if seed is None else seed,
                         c["optics"], name=f"config2 {n}x{c['layers']}x{c['bins']}x{c['g_points']}")


def uneven_shapes(n_cols: int, seed: int, L_range=None, NB_range=None):
    """Per-column layer and bin counts, uniform integers over the ranges
    (config 3's by default)."""
    c = CONFIGS["config3"]
    L_range = tuple(c["layers"]) if L_range is None else L_range
    NB_range = tuple(c["bins"]) if NB_range is None else NB_range
    rng = np.random.default_rng(seed + c["shape_seed_offset"])
    L = rng.integers(L_range[0], L_range[1] + 1, n_cols).astype(np.int32)
    NB = rng.integers(NB_range[0], NB_range[1] + 1, n_cols).astype(np.int32)
    return L, NB


def config3(n_cols: int | None = None, seed: int | None = None) -> Columns:
    """Uneven batch: L_c ~ U{20..200}, NB_c ~ U{30..300}, 20 g-points, optics as config 0."""
    c = CONFIGS["config3"]
    n = c["n_cols"] if n_cols is None else n_cols
    sd = c["seed"] if seed is None else seed
    L, NB = uneven_shapes(n, sd)
    return generate(L, NB, c["g_points"], sd, c["optics"], name=f"config3 {n} uneven")


# ----------------------------------------------------------------------
# Large batches drawn directly in device memory (torch's Philox generator),
# for the uneven and serving workloads whose cubes do not fit comfortably in
# host memory.  Per-column profiles are small and drawn on the host.
# ----------------------------------------------------------------------

class DeviceColumns:
    """A packed batch whose cubes live in device memory.

    Same fields as ``Columns`` except that dtau/w0/g0 (and the per-column
    arrays) are torch tensors on ``device``.  ``host_subset(idx)`` copies
    chosen columns back as a ``Columns`` for the oracle."""

    def __init__(self, n_layers, n_bins, n_g, g_weights, tensors: dict, consts: dict, name: str):
        self.n_layers = np.asarray(n_layers, dtype=np.int32)
        self.n_bins = np.asarray(n_bins, dtype=np.int32)
        self.n_g = int(n_g)
        self.g_weights = g_weights
        self.consts = consts
        self.name = name
        for k, v in tensors.items():
            setattr(self, k, v)

    @property
    def n_cols(self):
        return int(self.n_layers.size)

    @property
    def n_systems(self):
        return int((self.n_bins.astype(np.int64) * self.n_g).sum())

    def offsets(self):
        L = self.n_layers.astype(np.int64)
        NB = self.n_bins.astype(np.int64)
        z = lambda a: np.concatenate([[0], np.cumsum(a)])
        return dict(cube=z(L * NB * self.n_g), lay=z(L), iface=z(L + 1), bins=z(NB))

    def column_range(self, a: int, b: int) -> "DeviceColumns":
        """Columns [a, b) as a packed batch of views into the same device
        memory (no copy): one rank's contiguous share of a sharded batch."""
        o = self.offsets()
        t = {}
        for k, key in (("dtau", "cube"), ("w0", "cube"), ("g0", "cube"), ("T_center", "lay"),
                       ("T_iface", "iface"), ("p_iface", "iface"), ("F_star", "bins")):
            t[k] = getattr(self, k)[int(o[key][a]):int(o[key][b])]
        t["mu_star"] = self.mu_star[a:b]
        return DeviceColumns(self.n_layers[a:b].copy(), self.n_bins[a:b].copy(), self.n_g, self.g_weights, t,
                             self.consts, f"{self.name}[{a}:{b}]")

    def host_subset(self, idx) -> Columns:
        idx = np.asarray(idx, dtype=np.int64)
        o = self.offsets()

        def cat(t, key):
            parts = [t[int(o[key][i]):int(o[key][i + 1])].cpu().numpy() for i in idx]
            return np.concatenate(parts)
        return Columns(n_layers=self.n_layers[idx].copy(), n_bins=self.n_bins[idx].copy(),
                       n_g=self.n_g, g_weights=self.g_weights,
                       dtau=cat(self.dtau, "cube"), w0=cat(self.w0, "cube"), g0=cat(self.g0, "cube"),
                       T_center=cat(self.T_center, "lay"), T_iface=cat(self.T_iface, "iface"),
                       p_iface=cat(self.p_iface, "iface"),
                       mu_star=self.mu_star[torch_index(idx, self.mu_star)].cpu().numpy(),
                       F_star=cat(self.F_star, "bins"), consts=self.consts,
                       name=f"{self.name}[{idx.size} cols]")


def torch_index(idx, like):
    import torch
    return torch.as_tensor(idx, dtype=torch.long, device=like.device)


def _device_uniform(n, lo, hi, gen, device, log=False, chunk=1 << 28):
    import torch
    out = torch.empty(n, dtype=torch.float32, device=device)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        t = out[a:b]
        if log:
            t.uniform_(float(np.log(lo)), float(np.log(hi)), generator=gen)
            t.exp_()
        else:
            t.uniform_(lo, hi, generator=gen)
    return out


def device_generate(n_layers, n_bins, n_g: int, seed: int, device="cuda", name="") -> DeviceColumns:
    """Optics as config 0 (dtau ~ logU[1e-6, 10], w0 ~ U[0, 0.95], g0 ~
    U[0, 0.8]) drawn on the device; profiles, mu and F* as ``generate``."""
    import torch
    rng = np.random.default_rng(seed)
    n_layers = np.asarray(n_layers, dtype=np.int32)
    n_bins = np.asarray(n_bins, dtype=np.int32)
    C = n_layers.size
    gx, gw = gauss_legendre_01(n_g)
    mu = rng.uniform(0.1, 1.0, C)
    prof = [_profile(rng, int(L)) for L in n_layers]
    fs_cache = {}
    Fs = []
    for NB in n_bins:
        NB = int(NB)
        if NB not in fs_cache:
            fs_cache[NB] = stellar_flux_bins(NB)
        Fs.append(fs_cache[NB])
    n_cube = int((n_layers.astype(np.int64) * n_bins * n_g).sum())
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    t = dict(dtau=_device_uniform(n_cube, 1e-6, 10.0, gen, device, log=True),
             w0=_device_uniform(n_cube, 0.0, 0.95, gen, device),
             g0=_device_uniform(n_cube, 0.0, 0.8, gen, device))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
    t["T_center"] = dev(np.concatenate([p[1] for p in prof]))
    t["T_iface"] = dev(np.concatenate([p[2] for p in prof]))
    t["p_iface"] = dev(np.concatenate([p[0] for p in prof]))
    t["mu_star"] = dev(mu)
    t["F_star"] = dev(np.concatenate(Fs))
    return DeviceColumns(n_layers, n_bins, n_g, gw, t, _consts(), name)


def config3_device(n_cols: int | None = None, seed: int | None = None, device="cuda") -> DeviceColumns:
    """Uneven batch on the device: L_c ~ U{20..200}, NB_c ~ U{30..300}, 20 g."""
    c = CONFIGS["config3"]
    n = c["n_cols"] if n_cols is None else n_cols
    sd = c["seed"] if seed is None else seed
    L, NB = uneven_shapes(n, sd)
    return device_generate(L, NB, c["g_points"], sd, device, name=f"config3 {n} uneven (device)")


# ----------------------------------------------------------------------
# Post-processing workload (Sec. 2.1.3 and the run protocol of Sec. 3):
# after the GCM run the radiative transfer is repeated once on a
# high-resolution spectral grid -- opacity sampling at R = lambda / dlambda (Eq. 1) =
# 500, 3255 wavelength points log-spaced over 0.3-200 um, one g-point per
# bin -- on columns whose top is extended to 1 ubar with isothermal layers at
# the top-most model layer's temperature.
# ----------------------------------------------------------------------
POST_BINS = 3255
POST_P_MIN_BAR = 1e-6          # lowest pressure of the isothermal extension
POST_LAYERS_PER_DECADE = 4     # extension layers per decade of pressure
POST_L_MODEL = 40


def postproc_edges(n_bins: int = POST_BINS):
    """Bin edges (cm^-1) log-spaced over [WN_MIN, WN_MAX]: R = nu / dnu ~ 500."""
    return np.geomspace(WN_MIN, WN_MAX, n_bins + 1)


def stellar_flux_edges(edges_cm):
    """Stand-in stellar spectrum per bin for explicit edges (cm^-1)."""
    e = np.asarray(edges_cm, np.float64) * 100.0
    mid = 0.5 * (e[1:] + e[:-1])
    x = _H * _C * mid / (_KB * T_STAR)
    b_mid = 2.0 * _H * _C ** 2 * mid ** 3 / np.expm1(x)
    return np.pi * b_mid * np.diff(e) * (R_STAR / A_ORBIT) ** 2


def extend_isothermal(p_if, Tc, Ti, p_min_bar: float = POST_P_MIN_BAR,
                      per_decade: int = POST_LAYERS_PER_DECADE):
    """Extend one column above its top (layer 0) to ``p_min_bar`` with
    isothermal layers at the top-most layer's temperature.  The new layers
    are log-spaced in pressure, ``per_decade`` per decade (rounded up); a
    column whose top is already at or above p_min is returned unchanged.
    Returns (p_if, Tc, Ti, n_ext)."""
    p_top = p_if[0]
    p_min = p_min_bar * 1.0e5
    if p_top <= p_min:
        return p_if, Tc, Ti, 0
    n_ext = int(np.ceil(per_decade * np.log10(p_top / p_min)))
    p_ext = np.geomspace(p_min, p_top, n_ext + 1)[:-1]       # new interfaces above the old top
    p_if = np.concatenate([p_ext, p_if])
    Tc = np.concatenate([np.full(n_ext, Tc[0]), Tc])
    Ti = np.concatenate([np.full(n_ext, Tc[n_ext]), Ti])
    return p_if, Tc, Ti, n_ext


def postproc_profiles(n_cols: int, seed: int, L_model: int = POST_L_MODEL):
    """Per-column profiles of the post-processing workload: a model top
    log-uniform in [1e-7, 1e-3] bar (the day-to-night spread of the model top
    in Sec. 4), the model's L_model layers below it, then the isothermal
    extension to 1 ubar; mu* uniform in [-1, 1] with the night side (<= 0)
    set to 0 (no beam)."""
    rng = np.random.default_rng(seed)
    p_top = np.exp(rng.uniform(np.log(1e-7), np.log(1e-3), n_cols))
    mu = np.maximum(rng.uniform(-1.0, 1.0, n_cols), 0.0)
    prof, L = [], np.empty(n_cols, np.int32)
    for c in range(n_cols):
        p_if, Tc, Ti = _profile(rng, L_model, float(p_top[c]))
        p_if, Tc, Ti, n_ext = extend_isothermal(p_if, Tc, Ti)
        prof.append((p_if, Tc, Ti))
        L[c] = L_model + n_ext
    return L, prof, mu, rng


def postproc(n_cols: int = 64, seed: int = 5) -> Columns:
    """Post-processing batch on the host (opacity sampling, NG = 1):
    k ~ logU[1e-8, 1] m^2/kg per (layer, bin), dtau = k dp / g, w0 ~ U[0,
    0.95], g0 ~ U[0, 0.8].  Bins: ``postproc_edges()``."""
    L, prof, mu, rng = postproc_profiles(n_cols, seed)
    NB = POST_BINS
    cubes = {k: [] for k in ("dtau", "w0", "g0")}
    for c in range(n_cols):
        p_if = prof[c][0]
        shape = (int(L[c]), NB)
        k = np.exp(rng.uniform(np.log(1e-8), np.log(1.0), shape))
        cubes["dtau"].append((k * np.diff(p_if)[:, None] / GRAV).astype(np.float32).ravel())
        cubes["w0"].append(rng.uniform(0.0, 0.95, shape).astype(np.float32).ravel())
        cubes["g0"].append(rng.uniform(0.0, 0.8, shape).astype(np.float32).ravel())
    edges = postproc_edges()
    consts = dict(_consts(), wn_edges=edges)
    return Columns(n_layers=L, n_bins=np.full(n_cols, NB, np.int32), n_g=1,
                   g_weights=np.array([1.0]), dtau=np.concatenate(cubes["dtau"]),
                   w0=np.concatenate(cubes["w0"]), g0=np.concatenate(cubes["g0"]),
                   T_center=np.concatenate([p[1] for p in prof]),
                   T_iface=np.concatenate([p[2] for p in prof]),
                   p_iface=np.concatenate([p[0] for p in prof]), mu_star=mu,
                   F_star=np.tile(stellar_flux_edges(edges), n_cols), consts=consts,
                   name=f"postproc {n_cols}x~{int(L.mean())}x{NB}x1")


def postproc_device(n_cols: int = 2562, seed: int = 5, device="cuda") -> DeviceColumns:
    """The post-processing workload with its cubes drawn on the device (same
    distributions as ``postproc``, torch's generator): 2562 columns by
    default, ~8.3M (column, bin) systems."""
    import torch
    L, prof, mu, _ = postproc_profiles(n_cols, seed)
    NB = POST_BINS
    n_cube = int(L.astype(np.int64).sum()) * NB
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
    p_all = np.concatenate([p[0] for p in prof])
    dp = np.concatenate([np.diff(p[0]) for p in prof]) / GRAV               # per layer
    dtau = _device_uniform(n_cube, 1e-8, 1.0, gen, device, log=True)
    dtau.view(-1, NB).mul_(torch.from_numpy(dp.astype(np.float32)).to(device)[:, None])
    t = dict(dtau=dtau, w0=_device_uniform(n_cube, 0.0, 0.95, gen, device),
             g0=_device_uniform(n_cube, 0.0, 0.8, gen, device))
    t["T_center"] = dev(np.concatenate([p[1] for p in prof]))
    t["T_iface"] = dev(np.concatenate([p[2] for p in prof]))
    t["p_iface"] = dev(p_all)
    t["mu_star"] = dev(mu)
    edges = postproc_edges()
    t["F_star"] = dev(np.tile(stellar_flux_edges(edges), n_cols))
    return DeviceColumns(L, np.full(n_cols, NB, np.int32), 1, np.array([1.0]), t,
                         dict(_consts(), wn_edges=edges), f"postproc {n_cols} (device)")


# ----------------------------------------------------------------------
# Synthetic premixed k-table and cloud data for the input front end
# (Sec. 2.1.3): 60 temperatures on [50, 3000] K, 28 pressures log-spaced on
# [1e-6, 1e3] bar, NB bins x NG Gauss points, log10 kappa ascending over g
# within each (T, p, bin) as a sorted k-distribution is.  The enstatite
# LX-MIE cross sections are replaced by smooth stand-ins for 1 um particles.
# ----------------------------------------------------------------------
KT_NT, KT_NP = 60, 28
F_CLOUD = 1e-17          # cloud-to-gas number ratio used in the paper
X_H2, X_HE = 0.85, 0.15  # number fractions for Rayleigh scattering
MBAR_AMU = 2.34          # Table 3


def ktable(n_bins: int = 30, n_g: int = 20, seed: int = 11, edges=None):
    """Seeded synthetic k-table.  Returns a dict with T_grid, log10p_grid,
    log10_kappa [nT, nP, NB, NG] (float32), sigma_scat_cloud,
    sigma_abs_cloud, g0_cloud [NB], f_cloud, x_h2, x_he, mbar_amu, edges.

    log10 kappa = base_b + spread_b q_g + alpha_b log10(p / 1 bar) / 2
                  + beta_b (T - 1000 K) / 1000 K + N(0, 0.05), clipped to
    [-12, 3], then sorted over g;  q_g in [-1, 1] increasing, base_b ~
    U[-6, 0], spread_b ~ U[0.5, 3], alpha_b ~ U[0, 1], beta_b ~ U[-0.5, 0.5]."""
    rng = np.random.default_rng(seed)
    if edges is None:
        edges = np.linspace(WN_MIN, WN_MAX, n_bins + 1)
    edges = np.asarray(edges, np.float64)
    NB = edges.size - 1
    T_grid = np.linspace(50.0, 3000.0, KT_NT)
    lp_grid = np.linspace(np.log10(1e-6 * 1e5), np.log10(1e3 * 1e5), KT_NP)
    base = rng.uniform(-6.0, 0.0, NB)
    spread = rng.uniform(0.5, 3.0, NB)
    alpha = rng.uniform(0.0, 1.0, NB)
    beta = rng.uniform(-0.5, 0.5, NB)
    q = np.linspace(-1.0, 1.0, n_g) if n_g > 1 else np.zeros(1)
    lk = (base[None, None, :, None] + spread[None, None, :, None] * q[None, None, None, :]
          + alpha[None, None, :, None] * (lp_grid[None, :, None, None] - 5.0) / 2.0
          + beta[None, None, :, None] * (T_grid[:, None, None, None] - 1000.0) / 1000.0)
    lk = lk + rng.normal(0.0, 0.05, lk.shape)
    lk = np.sort(np.clip(lk, -12.0, 3.0), axis=-1).astype(np.float32)
    # cloud stand-in: 1 um particles, size parameter x = 2 pi r / lambda
    lam_um = 1.0e4 / (0.5 * (edges[1:] + edges[:-1]))
    x = 2.0 * np.pi * 1.0 / lam_um
    geo = np.pi * (1.0e-6) ** 2
    q_scat = 2.0 * x ** 4 / (1.0 + x ** 4)
    q_abs = 0.05 + 0.6 * np.exp(-0.5 * ((lam_um - 10.0) / 1.5) ** 2)
    g0c = 0.85 * x ** 2 / (1.0 + x ** 2)
    return dict(T_grid=T_grid, log10p_grid=lp_grid, log10_kappa=lk,
                sigma_scat_cloud=geo * q_scat, sigma_abs_cloud=geo * q_abs, g0_cloud=g0c,
                f_cloud=F_CLOUD, x_h2=X_H2, x_he=X_HE, mbar_amu=MBAR_AMU, edges=edges)


def state_columns(n_cols: int, L: int, NB: int, n_g: int, seed: int, name: str = "") -> Columns:
    """Column state without optics (for the k-table front end): profiles,
    mu and F* as ``generate_fast``; dtau/w0/g0 are empty."""
    rng = np.random.default_rng(seed)
    gx, gw = gauss_legendre_01(n_g)
    prof = [_profile(rng, L) for _ in range(n_cols)]
    mu = rng.uniform(0.1, 1.0, n_cols)
    e = np.zeros(0, np.float32)
    return Columns(n_layers=np.full(n_cols, L, np.int32), n_bins=np.full(n_cols, NB, np.int32),
                   n_g=n_g, g_weights=gw, dtau=e, w0=e, g0=e,
                   T_center=np.concatenate([p[1] for p in prof]),
                   T_iface=np.concatenate([p[2] for p in prof]),
                   p_iface=np.concatenate([p[0] for p in prof]), mu_star=mu,
                   F_star=np.tile(stellar_flux_bins(NB), n_cols), consts=_consts(),
                   name=name or f"state {n_cols}x{L}x{NB}x{n_g}")


# public names for the pieces other modules reuse (the serving pool draws its
# own profiles and cubes with them)
column_profile = _profile
device_uniform = _device_uniform
