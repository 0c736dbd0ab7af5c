"""C-ABI behaviour on the GPU: validation, error codes, budgets, streams."""
import numpy as np
import pytest

import rt_synth
from parity import assert_parity, gpu_solver, method_opts, oracle_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_02293_b300 import rt  # noqa: E402
from paper_2203_02293_b300.solver import DeviceBatch, Solver  # noqa: E402


@pytest.fixture(scope="module")
def small():
    cols = rt_synth.generate([5, 9, 3], [4, 2, 6], 3, seed=61, optics="uniform")
    return cols, DeviceBatch(cols)


def test_fluxes_before_solve(small):
    s = Solver(small[0].g_weights)
    with pytest.raises(rt.RTError) as e:
        s.outputs(small[1])
    assert e.value.code == rt.RT_ENOTSOLVED
    s.close()


def test_malformed_descriptors(small):
    cols, b = small
    s = Solver(cols.g_weights, max_layers=8)
    with pytest.raises(rt.RTError) as e:      # 9 layers > max_layers
        s.solve(b)
    assert e.value.code == rt.RT_EINVAL and "n_layers" in str(e.value)
    s.close()
    s = Solver(cols.g_weights)
    bad = rt.make_columns(3, b.n_layers, b.n_bins, b.dtau, b.w0, None, b.T_center, b.T_iface,
                          b.p_iface, b.mu_star, b.F_star)
    with pytest.raises(rt.RTError) as e:
        rt.rt_solve_columns(s.h, bad)
    assert e.value.code == rt.RT_EINVAL and "g0" in str(e.value)
    neg = rt.make_columns(-1, None, None, b.dtau, b.w0, b.g0, b.T_center, b.T_iface, b.p_iface,
                          b.mu_star, b.F_star, L=5, NB=4)
    with pytest.raises(rt.RTError):
        rt.rt_solve_columns(s.h, neg)
    zero_nb = rt.make_columns(3, b.n_layers, np.array([4, 0, 6], np.int32), b.dtau, b.w0, b.g0,
                              b.T_center, b.T_iface, b.p_iface, b.mu_star, b.F_star)
    with pytest.raises(rt.RTError):
        rt.rt_solve_columns(s.h, zero_nb)
    s.close()


def test_empty_batch_is_a_no_op(small):
    cols, b = small
    s = Solver(cols.g_weights)
    empty = rt.make_columns(0, None, None, None, None, None, None, None, None, None, None, L=1, NB=1)
    rt.rt_solve_columns(s.h, empty)
    rt.rt_fluxes(s.h, None, None, None)
    assert s.stats()["systems"] == 0
    s.close()


def test_budget_refusal(small):
    cols, b = small
    s = Solver(cols.g_weights, hbm_budget_bytes=1024)
    need = s.query_bytes(b)
    assert need > 1024
    with pytest.raises(rt.RTError) as e:
        s.solve(b)
    assert e.value.code == rt.RT_EBUDGET
    s.close()
    s = Solver(cols.g_weights, hbm_budget_bytes=need)
    s.solve(b)
    s.close()


def test_uniform_shape_descriptor_and_side_stream(small):
    cols = rt_synth.generate([12] * 5, [7] * 5, 4, seed=62, optics="ktable")
    b = DeviceBatch(cols)
    ref = oracle_solve(cols, method_opts())
    s = gpu_solver(cols, method_opts(), "fp32")
    desc = rt.make_columns(5, None, None, b.dtau, b.w0, b.g0, b.T_center, b.T_iface, b.p_iface,
                           b.mu_star, b.F_star, L=12, NB=7)
    st = torch.cuda.Stream()
    rt.rt_solve_columns(s.h, desc, st)
    o = s.outputs(b, stream=st)
    st.synchronize()
    got = {k: v.cpu().numpy() for k, v in o.items()}
    assert_parity(cols, got, ref, "fp32", "uniform+stream")
    # outputs read on another stream after the solve are ordered after it
    o2 = s.outputs(b, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(o2["F_up"].cpu().numpy(), got["F_up"])
    s.close()


def test_outputs_to_host_memory(small):
    cols, b = small
    s = Solver(cols.g_weights)
    s.solve(b)
    up = np.zeros(b.n_if)
    q = np.zeros(b.n_lay)
    rt.rt_fluxes(s.h, up, None, None)
    rt.rt_heating(s.h, q)
    torch.cuda.synchronize()
    o = s.outputs(b)
    torch.cuda.synchronize()
    assert np.array_equal(up, o["F_up"].cpu().numpy())
    assert np.array_equal(q, o["Q"].cpu().numpy())
    s.close()


def test_repeated_solves_reuse_workspace_and_change_shape():
    a = rt_synth.generate([30, 4], [10, 3], 5, seed=63, optics="uniform")
    c = rt_synth.generate([7, 50, 2, 9], [2, 12, 20, 1], 5, seed=64, optics="uniform")
    s = gpu_solver(a, method_opts(), "fp32")
    for cols in (a, c, a, c):
        b = DeviceBatch(cols)
        got = s.solve_numpy(b)
        assert_parity(cols, got, oracle_solve(cols, method_opts()), "fp32", "reuse")
    s.close()


def test_gathered_columns_equal_packed_columns():
    """Columns picked out of a pool by offsets (reordered, repeated) give the
    same bits as the same columns packed back to back."""
    pool = rt_synth.generate([12, 30, 7, 22, 40], [5, 9, 3, 17, 30], 20, seed=65, optics="ktable")
    pb = DeviceBatch(pool)
    o = pool.offsets()
    idx = np.array([3, 0, 3, 4, 1])
    gather = dict(cube_offset=o["cube"][idx], center_offset=o["lay"][idx],
                  iface_offset=o["iface"][idx], bin_offset=o["bins"][idx], col_index=idx)
    desc = rt.make_columns(len(idx), pool.n_layers[idx], pool.n_bins[idx], pb.dtau, pb.w0, pb.g0,
                           pb.T_center, pb.T_iface, pb.p_iface, pb.mu_star, pb.F_star,
                           gather=gather)
    for precision in (rt.RT_FP32_FORM, rt.RT_FP64_PLAIN):
        s = Solver(pool.g_weights, precision=precision)
        rt.rt_solve_columns(s.h, desc)
        sub = pool.subset(idx)
        n_if, n_lay = int((sub.n_layers + 1).sum()), int(sub.n_layers.sum())
        got = {k: torch.empty(n_if, dtype=torch.float64, device="cuda") for k in ("F_up", "F_down", "F_net")}
        got["Q"] = torch.empty(n_lay, dtype=torch.float64, device="cuda")
        rt.rt_fluxes(s.h, got["F_up"], got["F_down"], got["F_net"])
        rt.rt_heating(s.h, got["Q"])
        got["F_up_toa"] = torch.empty(int(sub.n_bins.sum()), dtype=torch.float64, device="cuda")
        rt.rt_toa_spectrum(s.h, got["F_up_toa"])
        torch.cuda.synchronize()
        ref = s.solve_numpy(DeviceBatch(sub))
        for k in ref:
            assert np.array_equal(got[k].cpu().numpy(), ref[k]), k
        s.close()


def test_negative_gather_offset_is_rejected():
    pool = rt_synth.generate([4, 4], [2, 2], 2, seed=66, optics="uniform")
    pb = DeviceBatch(pool)
    desc = rt.make_columns(2, pool.n_layers, pool.n_bins, pb.dtau, pb.w0, pb.g0, pb.T_center,
                           pb.T_iface, pb.p_iface, pb.mu_star, pb.F_star,
                           gather=dict(col_index=np.array([0, -1])))
    s = Solver(pool.g_weights)
    with pytest.raises(rt.RTError) as e:
        rt.rt_solve_columns(s.h, desc)
    assert e.value.code == rt.RT_EINVAL
    s.close()


@pytest.mark.parametrize("key", ["cube_offset", "center_offset", "iface_offset", "bin_offset", "col_index"])
def test_gather_offset_past_the_end_is_refused_before_launch(key):
    """An offset that puts a column's block one element past its array's end
    returns RT_EINVAL and enqueues nothing: the handle keeps the previous
    solve's results, bit for bit."""
    pool = rt_synth.generate([6, 9, 4], [5, 3, 7], 4, seed=67, optics="uniform")
    pb = DeviceBatch(pool)
    o = pool.offsets()
    idx = np.array([2, 0, 1])
    good = dict(cube_offset=o["cube"][idx], center_offset=o["lay"][idx], iface_offset=o["iface"][idx],
                bin_offset=o["bins"][idx], col_index=idx)
    mk = lambda g: rt.make_columns(len(idx), pool.n_layers[idx], pool.n_bins[idx], pb.dtau, pb.w0, pb.g0,
                                   pb.T_center, pb.T_iface, pb.p_iface, pb.mu_star, pb.F_star, gather=g)
    sub = pool.subset(idx)
    n_if = int((sub.n_layers + 1).sum())
    for precision in (rt.RT_FP32_FORM, rt.RT_FP64_PLAIN):
        s = Solver(pool.g_weights, precision=precision)
        rt.rt_solve_columns(s.h, mk(good))
        before = torch.empty(n_if, dtype=torch.float64, device="cuda")
        rt.rt_fluxes(s.h, None, None, before)
        bad = {k: v.copy() for k, v in good.items()}
        # the last column of the pool (batch entry 0) ends exactly at each array's end
        bad[key][0] += 1
        with pytest.raises(rt.RTError) as e:
            rt.rt_solve_columns(s.h, mk(bad))
        assert e.value.code == rt.RT_EINVAL
        with pytest.raises(rt.RTError) as e:
            rt.rt_query_bytes(s.h, mk(bad))
        assert e.value.code == rt.RT_EINVAL
        after = torch.empty(n_if, dtype=torch.float64, device="cuda")
        rt.rt_fluxes(s.h, None, None, after)
        torch.cuda.synchronize()
        assert torch.equal(before, after)
        s.close()


def test_kernel_times_are_recorded_on_request():
    cols = rt_synth.generate([20, 35], [30, 12], 20, seed=70, optics="ktable")
    b = DeviceBatch(cols)
    s = Solver(cols.g_weights)
    s.solve(b)
    with pytest.raises(rt.RTError) as e:
        rt.rt_kernel_times(s.h)                 # timing not asked for
    assert e.value.code == rt.RT_ENOTSOLVED
    s.close()
    for prec in (rt.RT_FP32_FORM, rt.RT_FP64_PLAIN):
        s = Solver(cols.g_weights, precision=prec, kernel_timing=1)
        s.solve(b)
        prep, solve = rt.rt_kernel_times(s.h)
        assert solve > 0.0 and prep >= 0.0
        assert (prep > 0.0) == (prec == rt.RT_FP32_FORM)
        s.close()


def test_injected_allocation_failure_leaves_the_handle_usable():
    """An allocation failure injected on the host (the next workspace
    allocation fails as on an out-of-memory device): the solve returns
    RT_ENOMEM with its message, nothing is left pending, and the same handle's
    next solve allocates and gives the same results as a fresh handle."""
    cols = rt_synth.generate([12, 30, 7], [9, 4, 11], 20, seed=91, optics="uniform")
    b = DeviceBatch(cols)
    fresh = Solver(cols.g_weights)
    ref = fresh.solve_numpy(b)
    fresh.close()
    s = Solver(cols.g_weights)
    rt.rt_inject_alloc_failures(1)
    with pytest.raises(rt.RTError) as e:
        s.solve(b)
    assert e.value.code == rt.RT_ENOMEM and "injected" in str(e.value)
    got = s.solve_numpy(b)
    for k in ref:
        assert np.array_equal(got[k], ref[k]), k
    # a workspace that must grow again after a larger batch
    big = DeviceBatch(rt_synth.generate([40] * 8, [30] * 8, 20, seed=92, optics="uniform"))
    rt.rt_inject_alloc_failures(2)
    for _ in range(2):
        with pytest.raises(rt.RTError) as e:
            s.solve(big)
        assert e.value.code == rt.RT_ENOMEM
    s.solve(big)
    torch.cuda.synchronize()
    rt.rt_inject_alloc_failures(0)
    with pytest.raises(rt.RTError):
        rt.rt_inject_alloc_failures(-1)
    s.close()
