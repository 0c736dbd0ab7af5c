"""Column sharding on CPU with two gloo ranks: the partition covers every
column once, the per-rank results assemble into the unsharded result, and the
step time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import rt_synth
from paper_2203_02293_b300.shard import max_over_ranks, partition


def test_partition_is_exact_and_balanced():
    L, NB = rt_synth.uneven_shapes(4096, seed=3)
    for world in (1, 2, 3, 8):
        parts = partition(L, NB, world)
        assert parts[0][0] == 0 and parts[-1][1] == 4096
        assert all(a[1] == b[0] for a, b in zip(parts[:-1], parts[1:]))
        cost = L.astype(np.int64) * NB
        shares = [cost[a:b].sum() for a, b in parts]
        assert max(shares) - min(shares) <= cost.max() + 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cols = rt_synth.generate([7, 30, 12, 5, 22, 9], [4, 8, 2, 11, 3, 6], 3, seed=21, optics="ktable")
    a, b = partition(cols.n_layers, cols.n_bins, world)[rank]
    mine = cols.subset(np.arange(a, b))
    out = oracle.get().solve_columns(oracle.OracleConfig(), mine)
    gathered = [None] * world
    dist.all_gather_object(gathered, (a, b, out["F_net"], out["Q"]))
    t = max_over_ranks(0.1 * (rank + 1), dist)
    if rank == 0:
        full = oracle.get().solve_columns(oracle.OracleConfig(), cols)
        net = np.concatenate([g[2] for g in sorted(gathered, key=lambda g: g[0])])
        Q = np.concatenate([g[3] for g in sorted(gathered, key=lambda g: g[0])])
        q.put((np.array_equal(net, full["F_net"]), np.array_equal(Q, full["Q"]), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_assemble_the_unsharded_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    same_net, same_q, t = res
    assert same_net and same_q
    assert t == pytest.approx(0.2)
