"""Parity of the CUDA iterative method (Sec. 2.2.2: N sweeps of the pairwise
two-stream relations) with the oracle's sweeps, element by element, on the
same seeded inputs, at N = 1, 10 and 200, and its limits: without
scattering one sweep is the exact (Thomas) solution, and many sweeps
converge to it."""
import numpy as np
import pytest

import rt_synth
from parity import assert_parity, errors, gpu_solve, method_opts, oracle_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def oracle_sweeps(cols, opts, n):
    import oracle
    from dataclasses import replace
    cfg = oracle.OracleConfig(improved=opts["improved"], isothermal=opts["isothermal"],
                              resonance=opts["resonance"], e_clamp=opts["e_clamp"], eps2=opts["eps2"],
                              T_int=opts["T_int"], F_toa=opts["F_toa"], wn_min=cols.consts["wn_min"],
                              wn_max=cols.consts["wn_max"], wn_edges=cols.consts.get("wn_edges"))
    return oracle.get().solve_columns(replace(cfg, n_sweeps=n), cols)


@pytest.fixture(scope="module")
def cfg0():
    return rt_synth.config0()


@pytest.mark.parametrize("iso", [False, True])
@pytest.mark.parametrize("n", [1, 10, 200])
def test_config0_sweeps(cfg0, iso, n):
    opts = method_opts(isothermal=iso)
    ref = oracle_sweeps(cfg0, opts, n)
    got = gpu_solve(cfg0, opts, "fp32", n_sweeps=n)
    e = assert_parity(cfg0, got, ref, "fp32", f"config0 sweeps={n} iso={iso}")
    print("config0 sweeps", n, "iso", iso, "error/tol", e)
    st, rs = got["stats"], ref["stats"]
    assert st["systems"] == 64 * 30
    assert st["etau_hits"] == rs["etau_hits"] and st["resonance_hits"] == rs["resonance_hits"]
    assert st["nonfinite_outputs"] == 0


@pytest.fixture(scope="module")
def cfg1():
    return rt_synth.config1()


@pytest.mark.parametrize("n", [10, 200])
def test_config1_sweeps_sampled(cfg1, n):
    """The GCM-shaped batch in the bench's launch shape, checked against the
    oracle's sweeps on sampled columns (the first, the last and four between)."""
    got = gpu_solve(cfg1, method_opts(), "fp32", n_sweeps=n)
    idx = np.array([0, 1, 700, 1281, 2000, 2561])
    sub = cfg1.subset(idx)
    ref = oracle_sweeps(sub, method_opts(), n)
    o = cfg1.offsets()
    pick_if = np.concatenate([np.arange(o["iface"][c], o["iface"][c + 1]) for c in idx])
    pick_l = np.concatenate([np.arange(o["lay"][c], o["lay"][c + 1]) for c in idx])
    pick_b = np.concatenate([np.arange(o["bins"][c], o["bins"][c + 1]) for c in idx])
    mine = {k: got[k][pick_if] for k in ("F_up", "F_down", "F_net")}
    mine["Q"] = got["Q"][pick_l]
    mine["F_up_toa"] = got["F_up_toa"][pick_b]
    e = assert_parity(sub, mine, ref, "fp32", f"config1 sweeps={n}")
    print("config1 sweeps", n, "sampled error/tol", e)
    assert got["stats"]["systems"] == 2562 * 600 and got["stats"]["nonfinite_outputs"] == 0


@pytest.mark.parametrize("iso", [False, True])
def test_one_sweep_without_scattering_is_thomas(iso):
    cols = rt_synth.generate([40, 7, 1, 33], [30, 5, 3, 2], 20, seed=61, optics="ktable")
    cols.w0[:] = 0.0
    opts = method_opts(isothermal=iso)
    ref = oracle_solve(cols, opts)                      # Thomas
    got = gpu_solve(cols, opts, "fp32", n_sweeps=1)
    e = assert_parity(cols, got, ref, "fp32", "one sweep, no scattering")
    print("one sweep vs Thomas, w0 = 0, iso", iso, e)


def test_many_sweeps_converge_to_thomas():
    cols = rt_synth.generate([12, 30, 5], [4, 7, 3], 3, seed=62, optics="uniform")
    ref = oracle_solve(cols, method_opts())             # Thomas
    got = gpu_solve(cols, method_opts(), "fp32", n_sweeps=3000)
    assert_parity(cols, got, ref, "fp32", "3000 sweeps vs Thomas")
    few = gpu_solve(cols, method_opts(), "fp32", n_sweeps=2)
    assert errors(cols, few, ref, "fp32")["F_up"] > 1.0


@pytest.mark.parametrize("staging", [1, 2])
def test_ragged_batch_modes_and_edges(staging):
    """Ragged L in [1, 40] (the kernel's register limit), NB in [1, 41], night
    side, F_TOA, both Planck routes; a column gives the same bits alone."""
    L, NB = rt_synth.uneven_shapes(29, seed=63, L_range=(1, 40), NB_range=(1, 41))
    L[0], L[1] = 40, 1
    cols = rt_synth.generate(L, NB, 5, seed=64, optics="uniform", mu_range=(-0.5, 1.0))
    for opts in (method_opts(), method_opts(isothermal=True, F_toa=20.0), method_opts(improved=False)):
        ref = oracle_sweeps(cols, opts, 7)
        got = gpu_solve(cols, opts, "fp32", n_sweeps=7, planck_staging=staging)
        assert_parity(cols, got, ref, "fp32", f"ragged sweeps {opts}")
    alone = gpu_solve(cols.subset(np.array([3])), method_opts(), "fp32", n_sweeps=7)
    batch = gpu_solve(cols, method_opts(), "fp32", n_sweeps=7)
    o = cols.offsets()
    assert np.array_equal(alone["F_net"], batch["F_net"][o["iface"][3]:o["iface"][4]])


def test_layer_limit_is_refused():
    from paper_2203_02293_b300 import rt
    cols = rt_synth.generate([41], [3], 2, seed=65, optics="uniform")
    with pytest.raises(rt.RTError) as ei:
        gpu_solve(cols, method_opts(), "fp32", n_sweeps=3)
    assert ei.value.code == rt.RT_EINVAL
    with pytest.raises(rt.RTError) as ei:
        gpu_solve(rt_synth.generate([4], [3], 2, seed=65), method_opts(), "fp64", n_sweeps=3)
    assert ei.value.code == rt.RT_EINVAL
