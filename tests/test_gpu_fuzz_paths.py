"""Seeded random cases for the other solve paths, against the oracle: the
iterative sweep method (Sec. 2.2.2), the k-table front end fused into the
FP32 solve (Sec. 2.1.3) and the R = 500 post-processing shape (explicit bin
edges, one g-point, per-bin TOA spectrum).  Each case draws its own shape,
seed and method switches; parity and branch counts as in the fixed tests."""
import numpy as np
import pytest

import rt_synth
from parity import assert_parity, gpu_solve, gpu_solver, method_opts, oracle_ktable_solve, oracle_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def random_opts(rng):
    return method_opts(isothermal=bool(rng.integers(0, 2)), improved=bool(rng.integers(0, 4) > 0),
                       resonance=str(rng.choice(["paper", "limit"])), eps2=float(rng.choice([2.0 / 3.0, 0.5])),
                       T_int=float(rng.choice([100.0, 0.0])), F_toa=float(rng.choice([0.0, 25.0])))


def oracle_sweeps(cols, opts, n):
    import oracle
    from dataclasses import replace
    cfg = oracle.OracleConfig(improved=opts["improved"], isothermal=opts["isothermal"],
                              resonance=opts["resonance"], e_clamp=opts["e_clamp"], eps2=opts["eps2"],
                              T_int=opts["T_int"], F_toa=opts["F_toa"], wn_min=cols.consts["wn_min"],
                              wn_max=cols.consts["wn_max"], wn_edges=cols.consts.get("wn_edges"))
    return oracle.get().solve_columns(replace(cfg, n_sweeps=n), cols)


def check_counts(got, ref):
    for k in ("etau_hits", "eclamp_hits", "resonance_hits"):
        assert got["stats"][k] == ref["stats"][k], (k, got["stats"], ref["stats"])
    assert got["stats"]["nonfinite_outputs"] == ref["stats"]["nonfinite"] == 0


@pytest.mark.parametrize("i", range(10))
def test_random_sweeps_match_oracle(i):
    rng = np.random.default_rng(8000 + i)
    n_cols = int(rng.integers(1, 9))
    L = rng.integers(1, 41, n_cols)            # the sweep kernel's layer limit is 40
    NB = rng.integers(1, 33, n_cols)
    NG = int(rng.choice([1, 3, 8, 20]))
    n = int(rng.choice([1, 4, 25, 150]))
    opts = random_opts(rng)
    cols = rt_synth.generate(L, NB, NG, seed=8100 + i, optics=str(rng.choice(["uniform", "ktable"])),
                             mu_range=(-0.3, 1.0))
    ref = oracle_sweeps(cols, opts, n)
    got = gpu_solve(cols, opts, "fp32", n_sweeps=n, planck_staging=int(rng.integers(0, 4)))
    assert_parity(cols, got, ref, "fp32", f"sweeps case {i} n={n} {opts}")
    check_counts(got, ref)


@pytest.mark.parametrize("i", range(6))
def test_random_ktable_cases_match_oracle(i):
    from paper_2203_02293_b300.solver import DeviceBatch
    rng = np.random.default_rng(8200 + i)
    NB = int(rng.choice([1, 7, 30, 45]))
    NG = int(rng.choice([1, 4, 20]))
    kt = rt_synth.ktable(n_bins=NB, n_g=NG, seed=8300 + i)
    cols = rt_synth.state_columns(int(rng.integers(1, 7)), int(rng.integers(1, 61)), NB, NG, seed=8400 + i)
    opts = random_opts(rng)
    ref, _ = oracle_ktable_solve(cols, kt, opts)
    s = gpu_solver(cols, opts, "fp32")
    s.set_ktable(kt)
    b = DeviceBatch(cols)
    s.solve_ktable(b)
    got = {k: v.cpu().numpy() for k, v in s.outputs(b).items()}
    got["F_up_toa"] = s.toa_spectrum(b).cpu().numpy()
    got["stats"] = s.stats()
    s.close()
    assert_parity(cols, got, ref, "fp32", f"k-table case {i} {opts}")
    check_counts(got, ref)


@pytest.mark.parametrize("i", range(4))
def test_random_postprocessing_cases_match_oracle(i):
    rng = np.random.default_rng(8500 + i)
    cols = rt_synth.postproc(int(rng.integers(1, 4)), seed=8600 + i)
    opts = random_opts(rng)
    ref = oracle_solve(cols, opts)
    for staging in (0, 1, 2, 3):
        got = gpu_solve(cols, opts, "fp32", planck_staging=staging)
        assert_parity(cols, got, ref, "fp32", f"post-processing case {i} staging {staging} {opts}")
        check_counts(got, ref)


@pytest.mark.parametrize("NG", [32, 33, 50, 64])
def test_many_g_points_match_oracle(NG):
    """Up to the 64 g-points the ABI allows: bins then span one, two or (with
    one system per lane) three work units."""
    rng = np.random.default_rng(8700 + NG)
    L = rng.integers(1, 50, 5)
    NB = rng.integers(1, 12, 5)
    cols = rt_synth.generate(L, NB, NG, seed=8800 + NG, optics="ktable", mu_range=(-0.3, 1.0))
    opts = random_opts(rng)
    ref = oracle_solve(cols, opts)
    for spl in (1, 2):
        for staging in (0, 1, 2, 3):
            got = gpu_solve(cols, opts, "fp32", systems_per_lane=spl, planck_staging=staging)
            assert_parity(cols, got, ref, "fp32", f"NG={NG} spl={spl} staging={staging} {opts}")
            check_counts(got, ref)
    got = gpu_solve(cols, opts, "fp64")
    assert_parity(cols, got, ref, "fp64", f"NG={NG} fp64 {opts}")
    check_counts(got, ref)


def test_extreme_shapes_match_oracle():
    """The ABI's limits: columns of 1024 layers (the staged Planck values of a
    unit no longer fit beside the default launch) and 4096 bins, beside small
    columns in the same batch."""
    cols = rt_synth.generate([1024, 700, 3, 2], [2, 5, 4096, 1], 3, seed=8900, optics="uniform",
                             mu_range=(-0.3, 1.0))
    opts = method_opts()
    ref = oracle_solve(cols, opts)
    for spl in (1, 2):
        for staging in (0, 1, 2, 3):
            got = gpu_solve(cols, opts, "fp32", systems_per_lane=spl, planck_staging=staging)
            assert_parity(cols, got, ref, "fp32", f"extreme shapes spl={spl} staging={staging}")
            check_counts(got, ref)
    got = gpu_solve(cols, opts, "fp64")
    assert_parity(cols, got, ref, "fp64", "extreme shapes fp64")
    check_counts(got, ref)
