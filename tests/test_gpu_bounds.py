"""The bounds-check build of the library (RT_BOUNDS_CHECK: every main
device-memory access compared with its array's extent; an access outside is
counted in rt_stats' bounds_violations and skipped, nothing traps).  Each
path of the solver runs under it on valid inputs and must read zero
violations and still match the oracle."""
import numpy as np
import pytest

import rt_synth
from parity import assert_parity, gpu_solve, method_opts, oracle_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_02293_b300 import build, rt  # noqa: E402


@pytest.fixture(scope="module")
def checked():
    """Route the binding to librt_bounds.so for the tests of this module."""
    import os
    if not os.path.exists(build.LIB_BOUNDS) or build.stale(build.LIB_BOUNDS):
        build.build_bounds()
    old = rt._lib
    rt._lib = rt._load(build.LIB_BOUNDS)
    yield rt._lib
    rt._lib = old


def _zero(got):
    assert got["stats"]["bounds_violations"] == 0, got["stats"]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_config0_under_bounds_checks(checked, precision):
    cols = rt_synth.config0()
    got = gpu_solve(cols, method_opts(), precision)
    _zero(got)
    assert_parity(cols, got, oracle_solve(cols, method_opts()), precision, "config0 checked")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_config3_sample_under_bounds_checks(checked, precision):
    L, NB = rt_synth.uneven_shapes(4096, seed=3)
    idx = np.array([0, 17, 1024, 2048, 4095, int(np.argmax(L * NB)), int(np.argmin(L * NB))])
    cols = rt_synth.generate(L[idx], NB[idx], 20 if precision == "fp32" else 4, seed=3, optics="uniform")
    for extra in ({}, dict(systems_per_lane=1), dict(planck_staging=rt.RT_STAGE_DIRECT),
                  dict(staging_depth=rt.RT_STAGING_DEPTH_MAX)):
        if precision == "fp64" and extra:
            continue
        got = gpu_solve(cols, method_opts(), precision, **extra)
        _zero(got)
        assert_parity(cols, got, oracle_solve(cols, method_opts()), precision, f"config3 sample {extra}")


def test_inline_planck_and_sweeps_under_bounds_checks(checked):
    pp = rt_synth.postproc(2, seed=5)
    got = gpu_solve(pp, method_opts(), "fp32")
    _zero(got)
    assert_parity(pp, got, oracle_solve(pp, method_opts()), "fp32", "post-processing checked")
    cols = rt_synth.generate([40, 7, 33], [30, 5, 12], 20, seed=81, optics="ktable")
    got = gpu_solve(cols, method_opts(), "fp32", n_sweeps=5)
    _zero(got)


def test_ktable_front_end_under_bounds_checks(checked):
    from parity import gpu_solver, oracle_ktable_solve
    from paper_2203_02293_b300.solver import DeviceBatch
    kt = rt_synth.ktable(n_bins=30, n_g=20, seed=11)
    state = rt_synth.state_columns(3, 17, 30, 20, seed=1)
    ref, _ = oracle_ktable_solve(state, kt, method_opts())
    for precision in ("fp32", "fp64"):
        s = gpu_solver(state, method_opts(), precision)
        s.set_ktable(kt)
        b = DeviceBatch(state)
        s.solve_ktable(b)
        got = {k: v.cpu().numpy() for k, v in s.outputs(b).items()}
        st = s.stats()
        s.close()
        assert st["bounds_violations"] == 0
        if precision == "fp32":
            assert_parity(state, got, ref, "fp32", "k-table checked")


def test_the_checks_count_and_skip_reads_past_a_declared_extent(checked, monkeypatch):
    """The checking build's test hook declares the cube arrays one element
    shorter than the packed batch (the real arrays are full size, so the
    skipped read would have been valid): the last system's read of it is
    counted and skipped, nothing else changes."""
    cols = rt_synth.generate([6, 5], [3, 4], 2, seed=82, optics="uniform")
    monkeypatch.setenv("RT_BOUNDS_TEST_CUBE_EXTENT", str(cols.dtau.size - 1))
    got = gpu_solve(cols, method_opts(), "fp32")
    assert got["stats"]["bounds_violations"] > 0
    monkeypatch.delenv("RT_BOUNDS_TEST_CUBE_EXTENT")
    assert gpu_solve(cols, method_opts(), "fp32")["stats"]["bounds_violations"] == 0


@pytest.mark.parametrize("i", range(12))
def test_random_batches_under_bounds_checks(checked, i):
    """Seeded random batches (ragged shapes up to the ABI's 64 g-points, the
    three optics families, night side, every launch variant of the FP32 form
    and the sweep method) read zero violations and keep their parity."""
    rng = np.random.default_rng(9100 + i)
    n_cols = int(rng.integers(1, 9))
    L = rng.integers(1, 41, n_cols)
    NB = rng.integers(1, 33, n_cols)
    NG = int(rng.choice([1, 3, 20, 33, 64]))
    optics = str(rng.choice(["uniform", "ktable", "stress"]))
    cols = rt_synth.generate(L, NB, NG, seed=9200 + i, optics=optics, mu_range=(-0.3, 1.0))
    opts = method_opts(isothermal=bool(rng.integers(0, 2)), resonance=str(rng.choice(["paper", "limit"])))
    ref = oracle_solve(cols, opts)
    runs = [("fp32", dict(systems_per_lane=spl, planck_staging=st)) for spl in (1, 2) for st in (0, 1, 2, 3)]
    runs += [("fp32", dict(n_sweeps=int(rng.choice([1, 5])))), ("fp64", {})]
    for precision, kw in runs:
        if precision == "fp64" and optics == "stress":
            continue
        got = gpu_solve(cols, opts, precision, **kw)
        _zero(got)
        if "n_sweeps" not in kw:
            assert_parity(cols, got, ref, precision, f"checked random {i} {kw}")
