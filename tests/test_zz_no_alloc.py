"""The no-allocation entry point against the regular one.

rt_solve_uniform_noalloc serves callers that cannot allocate device memory
(programs whose device memory belongs to their own pool or framework, loops
that cannot afford an allocation's synchronisation).  It keeps all of
its intermediates in a fixed file-scope device array.  Here it is called
twice in a row through the C ABI and each result is compared with
rt_solve_columns on the same inputs, within the FP32 tolerance the parity
tests use.  This file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import rt_synth
from parity import errors

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2203_02293_b300 import rt  # noqa: E402
from paper_2203_02293_b300.solver import DeviceBatch, Solver  # noqa: E402


def _uniform_desc(b: DeviceBatch, L: int, NB: int):
    return rt.make_columns(b.n_cols, None, None, b.dtau, b.w0, b.g0, b.T_center, b.T_iface,
                           b.p_iface, b.mu_star, b.F_star, L=L, NB=NB)


def _noalloc(cols, b, L, NB, stream=None, **method):
    out = {k: torch.full((b.n_if,), float("nan"), dtype=torch.float64, device="cuda")
           for k in ("F_up", "F_down", "F_net")}
    out["Q"] = torch.full((b.n_lay,), float("nan"), dtype=torch.float64, device="cuda")
    cfg = rt.Config(g_weights=cols.g_weights, **method)
    rt.rt_solve_uniform_noalloc(cfg, _uniform_desc(b, L, NB), out["F_up"], out["F_down"],
                                out["F_net"], out["Q"], stream)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_noalloc_matches_regular_entry_point_twice():
    shapes = [(300, 40, 30, 20, "ktable", 71), (57, 17, 9, 20, "uniform", 72)]
    for n_cols, L, NB, NG, optics, seed in shapes:
        cols = rt_synth.generate([L] * n_cols, [NB] * n_cols, NG, seed=seed, optics=optics)
        b = DeviceBatch(cols)
        s = Solver(cols.g_weights)
        ref = s.solve_numpy(b)
        s.close()
        first = _noalloc(cols, b, L, NB)
        second = _noalloc(cols, b, L, NB)
        for got in (first, second):
            e = errors(cols, got, ref, "fp32")
            assert all(v <= 1.0 for v in e.values()), e
        assert all(np.isfinite(first[k]).all() for k in first)


def test_noalloc_isothermal_and_regular_closures():
    """The other method switches (isothermal layers; the regular two-stream
    closure, E = 1) through the no-allocation entry point, against the
    regular one."""
    cols = rt_synth.generate([23] * 41, [11] * 41, 20, seed=73, optics="uniform")
    b = DeviceBatch(cols)
    for method in (dict(layers=rt.RT_ISOTHERMAL), dict(two_stream=rt.RT_REGULAR),
                   dict(layers=rt.RT_ISOTHERMAL, two_stream=rt.RT_REGULAR)):
        s = Solver(cols.g_weights, **method)
        ref = s.solve_numpy(b)
        s.close()
        got = _noalloc(cols, b, 23, 11, **method)
        e = errors(cols, got, ref, "fp32")
        assert all(v <= 1.0 for v in e.values()), (method, e)


def test_noalloc_refuses_batches_beyond_its_scratch():
    """A batch whose inputs and outputs are really allocated at full size
    (4096 x 40 x 32 x 20: 1.3 GB of cubes) but whose scratch would pass
    the fixed array is refused with RT_EBUDGET; descriptors that overstate
    their arrays, or ask for what this entry point does not do, with
    RT_EINVAL.  Nothing is launched in either case."""
    n, L, NB, NG = 4096, 40, 32, 20
    f32 = lambda m: torch.zeros(m, dtype=torch.float32, device="cuda")
    f64 = lambda m: torch.ones(m, dtype=torch.float64, device="cuda")
    cubes = [f32(n * L * NB * NG) for _ in range(3)]
    desc = rt.make_columns(n, None, None, *cubes, f64(n * L), f64(n * (L + 1)), f64(n * (L + 1)),
                           f64(n), f64(n * NB), L=L, NB=NB)
    outs = [f64(n * (L + 1)) for _ in range(3)] + [f64(n * L)]
    cfg = rt.Config(g_weights=np.full(NG, 1.0 / NG))
    with pytest.raises(rt.RTError) as e:
        rt.rt_solve_uniform_noalloc(cfg, desc, *outs)
    assert e.value.code == rt.RT_EBUDGET
    # element counts below the packed batch
    small = rt.make_columns(n, None, None, *cubes, f64(n * L), f64(n * (L + 1)), f64(n * (L + 1)),
                            f64(n), f64(n * NB), L=L + 1, NB=NB)
    with pytest.raises(rt.RTError) as e:
        rt.rt_solve_uniform_noalloc(cfg, small, *outs)
    assert e.value.code == rt.RT_EINVAL
    for bad in (rt.Config(g_weights=np.ones(1), precision=rt.RT_FP64_PLAIN),
                rt.Config(g_weights=np.array([1.5, -0.5])),
                rt.Config(g_weights=np.ones(1), n_sweeps=3)):
        with pytest.raises(rt.RTError) as e:
            rt.rt_solve_uniform_noalloc(bad, desc, *outs)
        assert e.value.code == rt.RT_EINVAL
    assert torch.all(outs[0] == 1.0)


def test_noalloc_allocates_nothing_and_replays_from_a_cuda_graph():
    """What the entry point is for: after the first call on the device (which
    looks up the fixed array's address and sets the kernels' shared-memory
    limits), repeated calls leave the free device memory as it was (a device
    allocation reserves at least a 2 MiB page), and the call can be captured
    into a CUDA graph whose replay writes the direct call's outputs bit for
    bit."""
    L, NB = 17, 9
    cols = rt_synth.generate([L] * 33, [NB] * 33, 20, seed=74, optics="uniform")
    b = DeviceBatch(cols)
    desc = _uniform_desc(b, L, NB)
    cfg = rt.Config(g_weights=cols.g_weights)
    outs = [torch.zeros(b.n_if, dtype=torch.float64, device="cuda") for _ in range(3)]
    outs.append(torch.zeros(b.n_lay, dtype=torch.float64, device="cuda"))
    rt.rt_solve_uniform_noalloc(cfg, desc, *outs)
    torch.cuda.synchronize()
    direct = [o.clone() for o in outs]
    assert all(torch.isfinite(o).all() for o in direct)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rt.rt_solve_uniform_noalloc(cfg, desc, *outs)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (1 << 20)
    assert all(torch.equal(o, d) for o, d in zip(outs, direct))

    for o in outs:
        o.fill_(float("nan"))
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rt.rt_solve_uniform_noalloc(cfg, desc, *outs, stream=s)
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(o, d) for o, d in zip(outs, direct))
