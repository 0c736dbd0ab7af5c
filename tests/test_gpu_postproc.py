"""Explicit bin edges and the per-bin TOA spectrum on the GPU: the
post-processing shape (Sec. 2.1.3: R = 500 opacity sampling, 3255 bins, one
g-point, columns extended to 1 ubar with isothermal layers) against the
oracle, and the spectrum's bin sums across work-unit boundaries."""
from dataclasses import replace

import numpy as np
import pytest

import rt_synth
from parity import assert_parity, gpu_solve, method_opts, oracle_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_02293_b300 import rt  # noqa: E402
from paper_2203_02293_b300.solver import DeviceBatch, Solver  # noqa: E402


def with_edges(cols, edges):
    n = cols.n_cols
    cols.consts = dict(cols.consts, wn_edges=np.asarray(edges, np.float64))
    cols.F_star = np.tile(rt_synth.stellar_flux_edges(edges), n)
    return cols


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_postproc_columns_match_the_oracle(prec):
    cols = rt_synth.postproc(6, seed=5)
    ref = oracle_solve(cols, method_opts())
    got = gpu_solve(cols, method_opts(), prec)
    e = assert_parity(cols, got, ref, prec, "postproc 6 cols")
    print(prec, "postproc 6 cols error/tol", e)
    assert "F_up_toa" in e


@pytest.mark.parametrize("n_g", [1, 7, 20, 32, 45])
@pytest.mark.parametrize("iso", [False, True])
def test_explicit_edges_and_spectrum_across_unit_boundaries(n_g, iso):
    NB = 37
    cols = rt_synth.generate([5, 17, 9], [NB] * 3, n_g, seed=40 + n_g, optics="ktable")
    with_edges(cols, np.geomspace(rt_synth.WN_MIN, rt_synth.WN_MAX, NB + 1))
    opts = method_opts(isothermal=iso)
    ref = oracle_solve(cols, opts)
    for prec in ("fp32", "fp64"):
        assert_parity(cols, gpu_solve(cols, opts, prec), ref, prec, f"n_g={n_g} iso={iso}")


@pytest.mark.parametrize("n_g", [1, 20, 32])
def test_spectrum_is_bitwise_reproducible(n_g):
    cols = rt_synth.generate([12, 30], [50, 41], n_g, seed=50, optics="ktable")
    s = Solver(cols.g_weights)
    b = DeviceBatch(cols)
    runs = []
    for _ in range(3):
        s.solve(b)
        runs.append(s.toa_spectrum(b).cpu().numpy())
    s.close()
    assert all(np.array_equal(runs[0], r) for r in runs[1:])


def test_uniform_bins_spectrum_matches_the_oracle():
    cols = rt_synth.generate([8, 3, 21], [30, 30, 30], 20, seed=51, optics="ktable")
    ref = oracle_solve(cols, method_opts())
    for prec in ("fp32", "fp64"):
        e = assert_parity(cols, gpu_solve(cols, method_opts(), prec), ref, prec)
        assert "F_up_toa" in e


def test_postproc_full_size_sampled_columns():
    """All 2562 columns solved in the bench's launch configuration; sampled
    columns checked against the oracle."""
    dc = rt_synth.postproc_device(2562, seed=5)
    b = DeviceBatch.from_device(dc)
    s = Solver(dc.g_weights, wn_edges=dc.consts["wn_edges"])
    s.solve(b)
    o = s.outputs(b)
    o["F_up_toa"] = s.toa_spectrum(b)
    torch.cuda.synchronize()
    full = {k: v.cpu().numpy() for k, v in o.items()}
    st = s.stats()
    s.close()
    assert st["invalid_inputs"] == 0 and st["nonfinite_outputs"] == 0
    idx = np.array([0, 1, 640, 1281, 1999, 2561])
    host = dc.host_subset(idx)
    host.consts = dc.consts
    ref = oracle_solve(host, method_opts())
    off = dc.offsets()
    pick = lambda a, key: np.concatenate([a[off[key][i]:off[key][i + 1]] for i in idx])
    got = dict(F_up=pick(full["F_up"], "iface"), F_down=pick(full["F_down"], "iface"),
               F_net=pick(full["F_net"], "iface"), Q=pick(full["Q"], "lay"),
               F_up_toa=pick(full["F_up_toa"], "bins"))
    e = assert_parity(host, got, ref, "fp32", "postproc 2562 sampled")
    print("fp32 postproc 2562 sampled error/tol", e)
    del b, dc
    torch.cuda.empty_cache()


def test_edges_need_matching_bin_counts():
    cols = rt_synth.generate([4, 4], [5, 6], 2, seed=52)
    s = Solver(cols.g_weights, wn_edges=np.linspace(50.0, 100.0, 6))
    with pytest.raises(rt.RTError) as e:
        s.solve(DeviceBatch(cols))
    assert e.value.code == rt.RT_EINVAL
    s.close()


def test_no_alloc_entry_refuses_explicit_edges():
    cols = rt_synth.generate_fast(2, 4, 5, 2, seed=53, optics="uniform")
    b = DeviceBatch(cols)
    desc = rt.make_columns(2, None, None, b.dtau, b.w0, b.g0, b.T_center, b.T_iface, b.p_iface,
                           b.mu_star, b.F_star, L=4, NB=5)
    outs = [torch.empty(n, dtype=torch.float64, device="cuda") for n in (10, 10, 10, 8)]
    cfg = rt.Config(g_weights=cols.g_weights, wn_edges=np.linspace(50.0, 100.0, 6))
    with pytest.raises(rt.RTError) as e:
        rt.rt_solve_uniform_noalloc(cfg, desc, *outs)
    assert e.value.code == rt.RT_EINVAL


def test_spectrum_before_any_solve_is_refused():
    s = Solver(np.ones(1))
    with pytest.raises(rt.RTError) as e:
        rt.rt_toa_spectrum(s.h, torch.empty(4, dtype=torch.float64, device="cuda"))
    assert e.value.code == rt.RT_ENOTSOLVED
    s.close()


MODES = (rt.RT_STAGE_SHARED, rt.RT_STAGE_DIRECT, rt.RT_STAGE_INLINE)


@pytest.mark.parametrize("n_g", [1, 3, 20])
@pytest.mark.parametrize("iso", [False, True])
@pytest.mark.parametrize("spl", [1, 2])
def test_planck_staged_direct_and_inline_agree_bitwise(n_g, iso, spl):
    """B from the pre-kernel's table (staged or read directly) and B
    evaluated in the solve kernel give the same bits: wide uniform bins."""
    cols = rt_synth.generate([9, 33, 4], [61, 17, 40], n_g, seed=60 + n_g, optics="ktable")
    b = DeviceBatch(cols)
    outs = []
    for mode in MODES:
        s = Solver(cols.g_weights, planck_staging=mode, systems_per_lane=spl,
                   layers=rt.RT_ISOTHERMAL if iso else rt.RT_NONISOTHERMAL)
        outs.append(s.solve_numpy(b))
        s.close()
    for o in outs[1:]:
        for k in outs[0]:
            assert np.array_equal(outs[0][k], o[k]), k


@pytest.mark.parametrize("spl", [1, 2])
def test_inline_unit_narrow_decision_matches_the_table(spl):
    """The solve kernel skips the per-level narrow-bin tests of inline B for a
    unit whose bins take two points at the column's coldest level.  Columns
    where that holds for every unit (hot), for none of the blue units (cold:
    their bins are wide in x there), for some levels only (a profile through
    both), and a column with a level at T = 0 (no coldest-level bound, so the
    per-level tests run): inline B equals the table bit for bit."""
    cols = rt_synth.postproc(4, seed=13)
    o = cols.offsets()
    T_c, T_i = cols.T_center.copy(), cols.T_iface.copy()
    for c, kind in enumerate(("hot", "cold", "through", "zero")):
        lay = slice(o["lay"][c], o["lay"][c + 1])
        ifc = slice(o["iface"][c], o["iface"][c + 1])
        L = o["lay"][c + 1] - o["lay"][c]
        if kind == "hot":
            T_c[lay], T_i[ifc] = 3000.0, 3000.0
        elif kind == "cold":
            T_c[lay], T_i[ifc] = 60.0, 60.0
        elif kind == "through":
            T_i[ifc] = np.geomspace(60.0, 3000.0, L + 1)
            T_c[lay] = np.sqrt(T_i[ifc][:-1] * T_i[ifc][1:])
        else:
            T_i[o["iface"][c]] = 0.0
    cols = replace(cols, T_center=T_c, T_iface=T_i)
    b = DeviceBatch(cols)
    outs = []
    for mode in (rt.RT_STAGE_DIRECT, rt.RT_STAGE_INLINE):
        s = Solver(cols.g_weights, planck_staging=mode, systems_per_lane=spl, wn_edges=cols.consts["wn_edges"])
        s.solve(b)
        out = s.outputs(b)
        out["F_up_toa"] = s.toa_spectrum(b)
        outs.append({k: v.cpu().numpy() for k, v in out.items()})
        s.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
        assert np.all(np.isfinite(outs[1][k])), k


@pytest.mark.parametrize("spl", [1, 2])
@pytest.mark.parametrize("iso", [False, True])
def test_inline_planck_on_the_postproc_shape(spl, iso):
    """Narrow R = 500 bins (Gauss-Legendre quadrature): the inline evaluation
    equals the table bit for bit and meets the oracle."""
    cols = rt_synth.postproc(4, seed=9)
    b = DeviceBatch(cols)
    outs = []
    layers = rt.RT_ISOTHERMAL if iso else rt.RT_NONISOTHERMAL
    for mode in (rt.RT_STAGE_DIRECT, rt.RT_STAGE_INLINE):
        s = Solver(cols.g_weights, planck_staging=mode, systems_per_lane=spl, wn_edges=cols.consts["wn_edges"],
                   layers=layers)
        s.solve(b)
        o = s.outputs(b)
        o["F_up_toa"] = s.toa_spectrum(b)
        outs.append({k: v.cpu().numpy() for k, v in o.items()})
        s.close()
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
    ref = oracle_solve(cols, method_opts(isothermal=iso))
    got = gpu_solve(cols, method_opts(isothermal=iso), "fp32", planck_staging=rt.RT_STAGE_INLINE, systems_per_lane=spl)
    assert_parity(cols, got, ref, "fp32", "postproc inline")
    assert got["stats"]["nonfinite_outputs"] == 0
