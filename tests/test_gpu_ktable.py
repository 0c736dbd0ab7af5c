"""The input front end on the GPU (Sec. 2.1.3: k-table interpolation, gas
and cloud mixing; App. C Rayleigh): the standalone optics kernel against the
oracle's FP64 front end, the fused solve against the oracle end to end, and
the fused solve bitwise against optics-then-solve."""
from dataclasses import replace

import numpy as np
import pytest

import rt_synth
from parity import assert_parity, method_opts, oracle_ktable_solve, oracle_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_02293_b300 import rt  # noqa: E402
from paper_2203_02293_b300.solver import DeviceBatch, Solver  # noqa: E402

# FP32 front end: log10 kappa (|x| <= 12) goes through three lerps and a
# scaled exp2 (a few e-6 relative in kappa), then one add, one multiply and
# one division: 3e-5 relative covers dtau and w0; g0 is a cast of an FP64
# value, 1e-6.
RTOL_OPTICS = 3e-5


@pytest.fixture(scope="module")
def kt():
    return rt_synth.ktable(n_bins=30, n_g=20, seed=11)


def opts_solver(cols, precision="fp32", iso=False, **kw):
    from parity import gpu_solver
    return gpu_solver(cols, method_opts(isothermal=iso), precision, **kw)


def test_optics_kernel_matches_the_oracle_front_end(kt):
    cols = rt_synth.state_columns(3, 13, 30, 20, seed=21)
    _, ref = oracle_ktable_solve(cols, kt, method_opts())
    s = opts_solver(cols)
    s.set_ktable(kt)
    got = {k: v.cpu().numpy() for k, v in s.ktable_optics(DeviceBatch(cols)).items()}
    s.close()
    for k, tol in (("dtau", RTOL_OPTICS), ("w0", RTOL_OPTICS), ("g0", 1e-6)):
        err = np.max(np.abs(got[k] - ref[k]) / np.maximum(np.abs(ref[k]), 1e-30))
        assert err <= tol, (k, err)


@pytest.mark.parametrize("iso", [False, True])
@pytest.mark.parametrize("prec,spl", [("fp32", 1), ("fp32", 2), ("fp64", 0)])
def test_fused_solve_equals_optics_then_solve(kt, iso, prec, spl):
    cols = rt_synth.state_columns(4, 17, 30, 20, seed=22)
    s = opts_solver(cols, prec, iso=iso, systems_per_lane=spl)
    s.set_ktable(kt)
    b = DeviceBatch(cols)
    s.solve_ktable(b)
    fused = {k: v.cpu().numpy() for k, v in s.outputs(b).items()}
    o = s.ktable_optics(b)
    torch.cuda.synchronize()
    full = replace(cols, **{k: v.cpu().numpy() for k, v in o.items()})
    plain = s.solve_numpy(DeviceBatch(full))
    s.close()
    for k in fused:
        assert np.array_equal(fused[k], plain[k]), k


@pytest.mark.parametrize("spl", [1, 2])
def test_fused_solve_planck_stagings_agree_bitwise(kt, spl):
    """The fused front end with B staged, read from the table or evaluated
    in the solve kernel: the same bits."""
    cols = rt_synth.state_columns(5, 23, 30, 20, seed=27)
    b = DeviceBatch(cols)
    outs = []
    for mode in (rt.RT_STAGE_SHARED, rt.RT_STAGE_DIRECT, rt.RT_STAGE_INLINE):
        s = opts_solver(cols, systems_per_lane=spl, planck_staging=mode)
        s.set_ktable(kt)
        s.solve_ktable(b)
        outs.append({k: v.cpu().numpy() for k, v in s.outputs(b).items()})
        s.close()
    for o in outs[1:]:
        for k in outs[0]:
            assert np.array_equal(outs[0][k], o[k]), k


def test_fused_solve_matches_the_oracle(kt):
    cols = rt_synth.state_columns(5, 21, 30, 20, seed=23)
    ref, _ = oracle_ktable_solve(cols, kt, method_opts())
    s = opts_solver(cols)
    s.set_ktable(kt)
    b = DeviceBatch(cols)
    s.solve_ktable(b)
    got = {k: v.cpu().numpy() for k, v in s.outputs(b).items()}
    got["F_up_toa"] = s.toa_spectrum(b).cpu().numpy()
    s.close()
    e = assert_parity(cols, got, ref, "fp32", "k-table fused")
    print("fp32 k-table fused error/tol", e)


def test_fp64_path_on_the_front_end_optics(kt):
    """FP64: the solve part to 1e-10 against the oracle on the GPU's own FP32
    optics (the optics themselves are checked against the oracle above)."""
    cols = rt_synth.state_columns(3, 9, 30, 20, seed=24)
    s = opts_solver(cols, "fp64")
    s.set_ktable(kt)
    b = DeviceBatch(cols)
    s.solve_ktable(b)
    got = {k: v.cpu().numpy() for k, v in s.outputs(b).items()}
    o = {k: v.cpu().numpy() for k, v in s.ktable_optics(b).items()}
    s.close()
    full = replace(cols, **o)
    e = assert_parity(full, got, oracle_solve(full, method_opts()), "fp64", "k-table fp64")
    print("fp64 k-table error/tol", e)


def test_postproc_shape_with_a_ktable():
    """Explicit R = 500 edges, one g-point, isothermal extension."""
    edges = rt_synth.postproc_edges()
    ktp = rt_synth.ktable(n_g=1, seed=12, edges=edges)
    L, prof, mu, _ = rt_synth.postproc_profiles(3, seed=25)
    base = rt_synth.postproc(3, seed=25)
    e = np.zeros(0, np.float32)
    cols = replace(base, dtau=e, w0=e, g0=e)
    ref, _ = oracle_ktable_solve(cols, ktp, method_opts(), edges=edges)
    s = opts_solver(cols)
    s.set_ktable(ktp)
    b = DeviceBatch(cols)
    s.solve_ktable(b)
    got = {k: v.cpu().numpy() for k, v in s.outputs(b).items()}
    got["F_up_toa"] = s.toa_spectrum(b).cpu().numpy()
    s.close()
    assert_parity(cols, got, ref, "fp32", "postproc k-table")


def test_gcm_shape_full_size_sampled(kt):
    """2562 x 40 x 30 x 20 with the fused front end; sampled columns."""
    cols = rt_synth.state_columns(2562, 40, 30, 20, seed=26)
    s = opts_solver(cols)
    s.set_ktable(kt)
    b = DeviceBatch(cols)
    s.solve_ktable(b)
    out = {k: v.cpu().numpy() for k, v in s.outputs(b).items()}
    st = s.stats()
    s.close()
    assert st["invalid_inputs"] == 0 and st["nonfinite_outputs"] == 0
    idx = np.array([0, 1, 977, 2000, 2561])
    sub = cols.subset(idx)
    ref, _ = oracle_ktable_solve(sub, kt, method_opts())
    o = cols.offsets()
    cat = lambda a, key: np.concatenate([a[o[key][i]:o[key][i + 1]] for i in idx])
    got = {"F_up": cat(out["F_up"], "iface"), "F_down": cat(out["F_down"], "iface"),
           "F_net": cat(out["F_net"], "iface"), "Q": cat(out["Q"], "lay")}
    e = assert_parity(sub, got, ref, "fp32", "k-table 2562 sampled")
    print("fp32 k-table 2562 sampled error/tol", e)


def test_front_end_errors(kt):
    cols = rt_synth.state_columns(2, 5, 30, 20, seed=27)
    b = DeviceBatch(cols)
    s = opts_solver(cols)
    with pytest.raises(rt.RTError) as e:
        s.solve_ktable(b)                       # no table yet
    assert e.value.code == rt.RT_ENOTSOLVED
    bad = dict(kt, T_grid=kt["T_grid"][::-1].copy())
    with pytest.raises(rt.RTError) as e:
        s.set_ktable(bad)
    assert e.value.code == rt.RT_EINVAL
    s.set_ktable(rt_synth.ktable(n_bins=12, n_g=20))
    with pytest.raises(rt.RTError) as e:
        s.solve_ktable(b)                       # 30-bin columns, 12-bin table
    assert e.value.code == rt.RT_EINVAL
    s.close()
    g3 = rt_synth.ktable(n_bins=30, n_g=3)
    s = opts_solver(cols)
    with pytest.raises(rt.RTError) as e:
        s.set_ktable(g3)                        # table n_g differs from the handle's
    assert e.value.code == rt.RT_EINVAL
    s.close()


def test_state_outside_the_table_grid_is_clamped_like_the_oracle(kt):
    """Columns hotter and colder than the 50-3000 K grid and reaching above
    1e-6 bar / below 1e3 bar: both sides clamp to the grid edges."""
    cols = rt_synth.state_columns(3, 12, 30, 20, seed=28)
    L = 12
    cols.T_center = cols.T_center.copy()
    cols.T_center[:L] = np.linspace(10.0, 40.0, L)          # below the grid
    cols.T_center[L:2 * L] = np.linspace(3100.0, 4000.0, L)  # above the grid
    cols.p_iface = cols.p_iface.copy()
    cols.p_iface[2 * (L + 1):] = np.geomspace(1e-4, 1e9, L + 1)   # past both pressure ends
    ref, _ = oracle_ktable_solve(cols, kt, method_opts())
    s = opts_solver(cols)
    s.set_ktable(kt)
    b = DeviceBatch(cols)
    s.solve_ktable(b)
    got = {k: v.cpu().numpy() for k, v in s.outputs(b).items()}
    s.close()
    assert_parity(cols, got, ref, "fp32", "k-table clamped")


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_gathered_state_equals_packed_state(kt, prec):
    """Columns picked out of a state pool by offsets (reordered, repeated)
    solve to the same bits as the same columns packed."""
    pool = rt_synth.state_columns(6, 14, 30, 20, seed=29)
    pb = DeviceBatch(pool)
    o = pool.offsets()
    idx = np.array([4, 1, 4, 0])
    gather = dict(center_offset=o["lay"][idx], iface_offset=o["iface"][idx], bin_offset=o["bins"][idx],
                  col_index=idx)
    desc = rt.make_columns(len(idx), pool.n_layers[idx], pool.n_bins[idx], None, None, None,
                           pb.T_center, pb.T_iface, pb.p_iface, pb.mu_star, pb.F_star, gather=gather)
    s = opts_solver(pool, prec)
    s.set_ktable(kt)
    rt.rt_solve_ktable(s.h, desc)
    sub = pool.subset(idx)
    n_if, n_lay = int((sub.n_layers + 1).sum()), int(sub.n_layers.sum())
    got = {k: torch.empty(n_if, dtype=torch.float64, device="cuda") for k in ("F_up", "F_down", "F_net")}
    got["Q"] = torch.empty(n_lay, dtype=torch.float64, device="cuda")
    rt.rt_fluxes(s.h, got["F_up"], got["F_down"], got["F_net"])
    rt.rt_heating(s.h, got["Q"])
    torch.cuda.synchronize()
    sb = DeviceBatch(sub)
    s.solve_ktable(sb)
    ref = {k: v.cpu().numpy() for k, v in s.outputs(sb).items()}
    s.close()
    for k in ref:
        assert np.array_equal(got[k].cpu().numpy(), ref[k]), k
