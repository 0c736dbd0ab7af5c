"""Shared helpers for the GPU parity tests: run the oracle and the CUDA path
on the same seeded inputs and compare element by element.

Tolerances (from the stated accuracy targets):
  FP64 plain path: |x - x_ref| <= 1e-10 max(|x_ref|, 1e-6 F*_col) for the
      interface fluxes F_up and F_down.  The net flux is their difference, so
      its budget is the sum of theirs: |dF_net| <= 1e-10 (|F_up| + |F_down|)
      (with the same floor).  Heating 1e-8 relative, floor carried through
      dF/dp.
  FP32 form: |x - x_ref| <= max(1e-4 |x_ref|, 1e-6 F*_col) for the fluxes and
      max(1e-3 |Q_ref|, (g/c_P) 1e-6 F*_col / dp_l) for the heating rate,
      with F*_col = sum over the column's bins of the stellar flux normal to
      the beam (an absolute floor of one millionth of the stellar flux).
  Per-bin TOA spectrum F_up_toa: the flux bound with the column floor shared
      out over the bins, 1e-6 F*_col / NB_c per bin (so the per-bin floors add
      up to the column's).
"""
from __future__ import annotations

import numpy as np

import oracle

GRAV, CP = 47.0, 12436.0


def method_opts(**kw):
    """Same switches for both sides: improved, isothermal, resonance, e_clamp,
    eps2, T_int, F_toa."""
    d = dict(improved=True, isothermal=False, resonance="paper", e_clamp=True, eps2=2.0 / 3.0,
             T_int=100.0, F_toa=0.0)
    d.update(kw)
    return d


def oracle_solve(cols, opts):
    cfg = oracle.OracleConfig(improved=opts["improved"], isothermal=opts["isothermal"],
                              resonance=opts["resonance"], e_clamp=opts["e_clamp"],
                              eps2=opts["eps2"], T_int=opts["T_int"], F_toa=opts["F_toa"],
                              wn_min=cols.consts["wn_min"], wn_max=cols.consts["wn_max"],
                              wn_edges=cols.consts.get("wn_edges"))
    return oracle.get().solve_columns(cfg, cols)


def gpu_solver(cols, opts, precision, **extra):
    from paper_2203_02293_b300 import rt
    from paper_2203_02293_b300.solver import Solver
    return Solver(cols.g_weights,
                  two_stream=rt.RT_IMPROVED if opts["improved"] else rt.RT_REGULAR,
                  layers=rt.RT_ISOTHERMAL if opts["isothermal"] else rt.RT_NONISOTHERMAL,
                  precision=rt.RT_FP64_PLAIN if precision == "fp64" else rt.RT_FP32_FORM,
                  resonance=rt.RT_RESONANCE_PAPER if opts["resonance"] == "paper" else rt.RT_RESONANCE_LIMIT,
                  e_clamp=int(opts["e_clamp"]), eps2=opts["eps2"], T_int=opts["T_int"],
                  F_toa_diffuse=opts["F_toa"], wn_min=cols.consts["wn_min"],
                  wn_max=cols.consts["wn_max"], wn_edges=cols.consts.get("wn_edges"), **extra)


def gpu_solve(cols, opts, precision, **extra):
    from paper_2203_02293_b300.solver import DeviceBatch
    s = gpu_solver(cols, opts, precision, **extra)
    try:
        b = DeviceBatch(cols)
        out = s.solve_numpy(b)
        out["stats"] = s.stats()
    finally:
        s.close()
    return out


def column_floors(cols):
    o = cols.offsets()
    fstar = np.array([cols.F_star[o["bins"][c]:o["bins"][c + 1]].sum() for c in range(cols.n_cols)])
    L = cols.n_layers.astype(np.int64)
    f_if = np.repeat(1e-6 * fstar, L + 1)
    dp = np.diff(cols.p_iface)
    # drop the differences that straddle two columns
    keep = np.ones(dp.size, bool)
    keep[o["iface"][1:-1] - 1] = False
    dp = dp[keep]
    f_q = GRAV / CP * np.repeat(1e-6 * fstar, L) / dp
    return f_if, f_q


def bin_floors(cols):
    o = cols.offsets()
    NB = cols.n_bins.astype(np.int64)
    fstar = np.array([cols.F_star[o["bins"][c]:o["bins"][c + 1]].sum() for c in range(cols.n_cols)])
    return np.repeat(1e-6 * fstar / NB, NB)


def errors(cols, got, ref, precision):
    """Largest |error| / tolerance per quantity (<= 1 passes)."""
    f_if, f_q = column_floors(cols)
    res = {}
    for k in ("F_up", "F_down", "F_net"):
        g, r = got[k], ref[k]
        if precision == "fp64":
            scale = np.abs(ref["F_up"]) + np.abs(ref["F_down"]) if k == "F_net" else np.abs(r)
            tol = 1e-10 * np.maximum(scale, f_if)
        else:
            tol = np.maximum(1e-4 * np.abs(r), f_if)
        res[k] = float(np.max(np.abs(g - r) / tol)) if r.size else 0.0
    g, r = got["Q"], ref["Q"]
    tol = (1e-8 if precision == "fp64" else 1e-3) * np.abs(r)
    tol = np.maximum(tol, (1e-8 if precision == "fp64" else 1.0) * f_q)
    res["Q"] = float(np.max(np.abs(g - r) / tol)) if r.size else 0.0
    if "F_up_toa" in got and "F_up_toa" in ref:
        g, r = got["F_up_toa"], ref["F_up_toa"]
        fb = bin_floors(cols)
        tol = 1e-10 * np.maximum(np.abs(r), fb) if precision == "fp64" else np.maximum(1e-4 * np.abs(r), fb)
        res["F_up_toa"] = float(np.max(np.abs(g - r) / tol)) if r.size else 0.0
    return res


HIST_EDGES = (1e-4, 1e-3, 1e-2, 1e-1, 0.5, 1.0)


def error_histogram(cols, got, ref):
    """Per quantity, the distribution of FP32 error / tolerance over every
    interface (layer for Q): the fraction in each bin of HIST_EDGES (below
    1e-4, [1e-4, 1e-3), ..., [0.5, 1], above 1) and the 50th, 90th, 99th and
    99.9th percentiles."""
    f_if, f_q = column_floors(cols)
    res = {}
    for k in ("F_up", "F_down", "F_net", "Q"):
        if k == "Q":
            tol = np.maximum(1e-3 * np.abs(ref[k]), f_q)
        else:
            tol = np.maximum(1e-4 * np.abs(ref[k]), f_if)
        r = np.abs(got[k] - ref[k]) / tol
        counts = np.histogram(r, bins=(0.0, *HIST_EDGES, np.inf))[0]
        res[k] = {"fractions": [float(c) / r.size for c in counts],
                  "p50": float(np.percentile(r, 50)), "p90": float(np.percentile(r, 90)),
                  "p99": float(np.percentile(r, 99)), "p99.9": float(np.percentile(r, 99.9))}
    return res


def strict_errors(cols, got, ref):
    """FP32 errors under the stricter reading |e| <= 1e-4 max(|x|, 1e-6 F*)
    (reported, not gated)."""
    f_if, f_q = column_floors(cols)
    res = {}
    for k in ("F_up", "F_down", "F_net"):
        res[k] = float(np.max(np.abs(got[k] - ref[k]) / (1e-4 * np.maximum(np.abs(ref[k]), f_if))))
    res["Q"] = float(np.max(np.abs(got["Q"] - ref["Q"]) / (1e-3 * np.maximum(np.abs(ref["Q"]), f_q))))
    return res


def assert_parity(cols, got, ref, precision, label=""):
    e = errors(cols, got, ref, precision)
    bad = {k: v for k, v in e.items() if not (v <= 1.0)}
    assert not bad, f"{label} {precision} parity failed (error/tolerance): {e}"
    return e


def oracle_ktable_solve(cols, kt, opts, edges=None):
    """The oracle front end (FP64 optics, rounded to the float32 the solver
    takes) followed by the oracle solve."""
    from dataclasses import replace
    import oracle.frontend as FE
    K = FE.KTable(**{k: kt[k] for k in ("T_grid", "log10p_grid", "log10_kappa", "sigma_scat_cloud",
                                        "sigma_abs_cloud", "g0_cloud", "f_cloud", "x_h2", "x_he",
                                        "mbar_amu")})
    if edges is None:
        edges = cols.consts.get("wn_edges")
    if edges is None:
        edges = np.linspace(cols.consts["wn_min"], cols.consts["wn_max"], int(cols.n_bins[0]) + 1)
    o = FE.optics(K, cols, edges, GRAV)
    full = replace(cols, dtau=o["dtau"].astype(np.float32), w0=o["w0"].astype(np.float32),
                   g0=o["g0"].astype(np.float32))
    return oracle_solve(full, opts), o
