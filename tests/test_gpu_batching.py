"""Uneven batches, CUDA-graph replay and the launch-shape autotuner."""
import numpy as np
import pytest

import rt_synth
from parity import assert_parity, method_opts, oracle_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_02293_b300 import rt  # noqa: E402
from paper_2203_02293_b300.solver import DeviceBatch, Solver  # noqa: E402
from paper_2203_02293_b300.tuning import GraphSolve, autotune  # noqa: E402


@pytest.fixture(scope="module")
def cfg3():
    dc = rt_synth.config3_device()
    return dc, DeviceBatch.from_device(dc)


def sample_columns(dc, k=24, seed=0):
    rng = np.random.default_rng(seed)
    cost = dc.n_layers.astype(np.int64) * dc.n_bins
    extremes = [int(np.argmax(cost)), int(np.argmin(cost)), int(np.argmax(dc.n_layers)),
                int(np.argmax(dc.n_bins))]
    pick = rng.choice(dc.n_cols, k - len(extremes), replace=False)
    return np.unique(np.concatenate([extremes, pick]))


def slice_outputs(dc, out, idx):
    o = dc.offsets()
    cat = lambda a, key: np.concatenate([a[o[key][i]:o[key][i + 1]] for i in idx])
    return {"F_up": cat(out["F_up"], "iface"), "F_down": cat(out["F_down"], "iface"),
            "F_net": cat(out["F_net"], "iface"), "Q": cat(out["Q"], "lay"),
            "F_up_toa": cat(out["F_up_toa"], "bins")}


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_config3_uneven_full_batch_sampled_parity(cfg3, precision):
    """4096 columns, L in [20, 200], NB in [30, 300], 20 g, one launch; the
    oracle checks sampled columns (largest, smallest, random)."""
    dc, b = cfg3
    s = Solver(dc.g_weights, precision=rt.RT_FP64_PLAIN if precision == "fp64" else rt.RT_FP32_FORM)
    out = s.solve_numpy(b)
    st = s.stats()
    s.close()
    assert st["systems"] == dc.n_systems and st["nonfinite_outputs"] == 0
    idx = sample_columns(dc)
    host = dc.host_subset(idx)
    ref = oracle_solve(host, method_opts())
    e = assert_parity(host, slice_outputs(dc, out, idx), ref, precision, "config3")
    print(precision, "config3 sampled error/tol", e, "systems", dc.n_systems)


def test_graph_replay_equals_eager(cfg3):
    dc, b = cfg3
    s = Solver(dc.g_weights)
    eager = s.solve_numpy(b)
    g = GraphSolve(s, b)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    o = s.outputs(b)
    o["F_up_toa"] = s.toa_spectrum(b)
    torch.cuda.synchronize()
    for k in eager:
        assert np.array_equal(o[k].cpu().numpy(), eager[k]), k
    s.close()


def test_autotuner_candidates_agree():
    L, NB = rt_synth.uneven_shapes(300, seed=77, L_range=(20, 120), NB_range=(30, 200))
    cols = rt_synth.generate(L, NB, 20, seed=78, optics="uniform")
    b = DeviceBatch(cols)
    cands = [dict(block_threads=bt, ctas_per_sm=c, systems_per_lane=n)
             for n in (1, 2) for bt, c in ((64, 0), (128, 2), (256, 0), (256, 1))]
    cands.append(dict(block_threads=128, ctas_per_sm=0, systems_per_lane=2, planck_staging=rt.RT_STAGE_DIRECT))
    cands.append(dict(block_threads=256, ctas_per_sm=0, systems_per_lane=2, planck_staging=rt.RT_STAGE_INLINE))
    cands.append(dict(block_threads=128, ctas_per_sm=0, systems_per_lane=2, staging_depth=3))
    res = autotune(b, cols.g_weights, candidates=cands, reps=2)
    assert res["stable"], res["table"]
    assert res["block_threads"] in (64, 128, 256)
    ref = oracle_solve(cols, method_opts())
    from paper_2203_02293_b300.tuning import KNOBS
    s = Solver(cols.g_weights, **{k: res[k] for k in KNOBS if k in res})
    assert_parity(cols, s.solve_numpy(b), ref, "fp32", "autotuned")
    s.close()


@pytest.mark.parametrize("staging", [rt.RT_STAGE_SHARED, rt.RT_STAGE_DIRECT, rt.RT_STAGE_INLINE])
def test_staging_depths_give_the_same_bits(staging):
    """The back-substitution's prefetch depth (RT_STAGING_DEPTH_MIN to _MAX levels
    through the shared-memory ring) moves loads, not arithmetic: every depth
    gives the same bits, for ragged columns (L from 1 to 200, so the ring's
    slots wrap at every offset), one and two systems per lane; out-of-range
    depths are refused."""
    L, NB = rt_synth.uneven_shapes(40, seed=79, L_range=(1, 200), NB_range=(1, 30))
    L[:4] = [1, 2, 3, 4]
    cols = rt_synth.generate(L, NB, 3, seed=80, optics="uniform")
    b = DeviceBatch(cols)
    for spl in (1, 2):
        outs = []
        for d in range(rt.RT_STAGING_DEPTH_MIN, rt.RT_STAGING_DEPTH_MAX + 1):
            s = Solver(cols.g_weights, systems_per_lane=spl, planck_staging=staging, staging_depth=d)
            outs.append(s.solve_numpy(b))
            s.close()
        for o in outs[1:]:
            for k in outs[0]:
                assert np.array_equal(o[k], outs[0][k]), (spl, k)
    assert_parity(cols, outs[0], oracle_solve(cols, method_opts()), "fp32", f"staging depths {staging}")
    for bad in (-1, 1, rt.RT_STAGING_DEPTH_MAX + 1):
        with pytest.raises(rt.RTError) as e:
            Solver(cols.g_weights, staging_depth=bad)
        assert e.value.code == rt.RT_EINVAL
