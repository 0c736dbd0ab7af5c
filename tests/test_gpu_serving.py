"""Continuous batching: results alone vs in the mix, admission by HBM budget,
cancellation and timeout on the host, latency percentiles."""
import numpy as np
import pytest

import rt_synth
from parity import assert_parity, method_opts, oracle_solve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_02293_b300 import rt  # noqa: E402
from paper_2203_02293_b300.serve import Pool, Server, make_requests  # noqa: E402
from paper_2203_02293_b300.solver import Solver  # noqa: E402


@pytest.fixture(scope="module")
def pool():
    return Pool(rt_synth, n_pool=64, L_range=(10, 30), NB_range=(5, 40), n_g=20)


def solve_alone(pool, r):
    s = Solver(pool.g_weights)
    desc, nl = pool.descriptor([r])
    rt.rt_solve_columns(s.h, desc)
    out = s.outputs_host(int((nl + 1).sum()), int(nl.sum()))
    s.close()
    return out


def test_each_result_is_the_same_alone_and_in_the_mix(pool):
    reqs = make_requests(pool, 48, rate_hz=4000.0, seed=5, C_range=(1, 64))
    srv = Server(pool, n_slots=3, keep_outputs=True)
    summ = srv.run(reqs)
    srv.close()
    assert summ["done"] == 48 and summ["batches"] < 48     # requests shared launches
    for r in reqs[::5]:
        alone = solve_alone(pool, r)
        for k in alone:
            assert np.array_equal(alone[k], r.outputs[k]), (r.rid, k)


def test_served_results_match_the_oracle(pool):
    reqs = make_requests(pool, 6, rate_hz=2000.0, seed=6, C_range=(1, 8))
    srv = Server(pool, n_slots=2, keep_outputs=True)
    srv.run(reqs)
    srv.close()
    import types
    for r in reqs:
        nl, nb, g = pool.gather([r])
        cols = rt_synth.Columns(
            n_layers=nl, n_bins=nb, n_g=pool.n_g, g_weights=pool.g_weights,
            dtau=np.concatenate([pool.dtau[o:o + r.L * r.NB * pool.n_g].cpu().numpy() for o in g["cube_offset"]]),
            w0=np.concatenate([pool.w0[o:o + r.L * r.NB * pool.n_g].cpu().numpy() for o in g["cube_offset"]]),
            g0=np.concatenate([pool.g0[o:o + r.L * r.NB * pool.n_g].cpu().numpy() for o in g["cube_offset"]]),
            T_center=np.concatenate([pool.T_center[o:o + r.L].cpu().numpy() for o in g["center_offset"]]),
            T_iface=np.concatenate([pool.T_iface[o:o + r.L + 1].cpu().numpy() for o in g["iface_offset"]]),
            p_iface=np.concatenate([pool.p_iface[o:o + r.L + 1].cpu().numpy() for o in g["iface_offset"]]),
            mu_star=pool.mu_star[torch.as_tensor(g["col_index"], device="cuda")].cpu().numpy(),
            F_star=np.concatenate([pool.F_star[o:o + r.NB].cpu().numpy() for o in g["bin_offset"]]),
            consts=rt_synth._consts())
        assert_parity(cols, r.outputs, oracle_solve(cols, method_opts()), "fp32", f"request {r.rid}")


def test_admission_refuses_what_never_fits_and_serves_the_rest(pool):
    reqs = make_requests(pool, 12, rate_hz=3000.0, seed=7, C_range=(1, 64))
    sizes = sorted(reqs, key=lambda r: r.systems)
    budget = Server(pool, n_slots=1)
    # budget between the two largest requests' needs
    need = [budget._bytes(budget.slots[0], r) for r in sizes]
    budget.close()
    srv = Server(pool, n_slots=2, hbm_budget_bytes=(need[-1] + need[-2]) // 2)
    summ = srv.run(reqs)
    srv.close()
    assert sizes[-1].status == "refused"
    assert summ["refused"] >= 1 and summ["done"] == 12 - summ["refused"]


def test_cancel_and_timeout_on_the_host(pool):
    reqs = make_requests(pool, 20, rate_hz=20000.0, seed=8, C_range=(32, 64))
    srv = Server(pool, n_slots=1, keep_outputs=False)
    summ = srv.run(reqs, cancel={3, 11})
    srv.close()
    assert reqs[3].status in ("cancelled", "done") and reqs[11].status in ("cancelled", "done")
    assert summ["cancelled"] + summ["done"] == 20
    srv = Server(pool, n_slots=1, wait_timeout_s=1e-9)
    reqs = make_requests(pool, 20, rate_hz=1e6, seed=9, C_range=(32, 64))
    summ = srv.run(reqs)
    srv.close()
    assert summ["timeout"] >= 1 and summ["timeout"] + summ["done"] == 20
    assert summ["p50_ms"] is None or summ["p99_ms"] >= summ["p50_ms"]


def test_split_requests_give_the_same_bits_as_whole(pool):
    """Requests cut into pieces of a few columns, the pieces batched with
    other requests and run on several slots: each request's result equals
    its result solved alone."""
    reqs = make_requests(pool, 24, rate_hz=4000.0, seed=10, C_range=(8, 64))
    srv = Server(pool, n_slots=3, keep_outputs=True, split_systems=3 * 40 * 20, policy="sjf")
    summ = srv.run(reqs)
    srv.close()
    assert summ["done"] == 24
    assert any(r.pieces for r in reqs)
    for r in reqs[::3]:
        alone = solve_alone(pool, r)
        for k in alone:
            assert np.array_equal(alone[k], r.outputs[k]), (r.rid, k)


def test_cancelling_a_split_request_drops_its_waiting_pieces(pool):
    reqs = make_requests(pool, 10, rate_hz=1e6, seed=11, C_range=(32, 64))
    srv = Server(pool, n_slots=1, split_systems=2 * 40 * 20)
    summ = srv.run(reqs, cancel={4})
    srv.close()
    assert reqs[4].status in ("cancelled", "done")
    assert summ["cancelled"] + summ["done"] == 10
    if reqs[4].status == "cancelled":
        assert all(p.status in ("dropped", "cancelled", "done") for p in reqs[4].pieces)


def test_a_refused_launch_fails_its_requests_and_serving_goes_on(pool):
    """An allocation failure injected on the host makes one batch's launch
    return RT_ENOMEM: that batch's requests fail, the slot and its handle
    serve the rest, and every other request completes."""
    reqs = make_requests(pool, 12, rate_hz=3000.0, seed=12, C_range=(1, 16))
    srv = Server(pool, n_slots=2)
    rt.rt_inject_alloc_failures(1)
    try:
        summ = srv.run(reqs)
    finally:
        rt.rt_inject_alloc_failures(0)
        srv.close()
    assert summ["failed"] >= 1 and summ["done"] + summ["failed"] == 12, summ
    assert srv.failures and "injected" in srv.failures[0]
    assert all(r.status in ("done", "failed") for r in reqs)
