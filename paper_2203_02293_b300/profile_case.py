"""One workload, solved a few times, for profilers.

    python -m paper_2203_02293_b300.profile_case fp32 2562       # GCM shape, cubes in
    python -m paper_2203_02293_b300.profile_case fp64 2562       # same, FP64 plain path
    python -m paper_2203_02293_b300.profile_case postproc 2562   # R = 500 post-processing shape
    python -m paper_2203_02293_b300.profile_case ktable 2562     # GCM shape, k-table front end

Each case runs two solves of the same batch (the second is the one to
capture with ``ncu -s 1 -c 1`` on the solve kernel, or ``-s 1`` on the
pre-kernel) and exits 0.  The GCM cubes of 2562 columns are 738 MB and the
post-processing cubes 4.5 GB, both above the 126 MB L2.
"""
import sys

import torch

import rt_synth
from paper_2203_02293_b300 import rt
from paper_2203_02293_b300.solver import DeviceBatch, Solver


def main(argv):
    case = argv[1] if len(argv) > 1 else "fp32"
    ncols = int(argv[2]) if len(argv) > 2 else 2562
    if case in ("fp32", "fp64"):
        cols = rt_synth.config1(n_cols=ncols)
        b = DeviceBatch(cols)
        s = Solver(cols.g_weights, precision=rt.RT_FP32_FORM if case == "fp32" else rt.RT_FP64_PLAIN)
        run = lambda: s.solve(b)
        n_sys = cols.n_systems
    elif case == "postproc":
        dc = rt_synth.postproc_device(ncols, seed=5)
        b = DeviceBatch.from_device(dc)
        s = Solver(dc.g_weights, wn_edges=dc.consts["wn_edges"])
        run = lambda: s.solve(b)
        n_sys = dc.n_systems
    elif case == "ktable":
        cols = rt_synth.state_columns(ncols, 40, 30, 20, seed=26)
        b = DeviceBatch(cols)
        s = Solver(cols.g_weights)
        s.set_ktable(rt_synth.ktable(n_bins=30, n_g=20, seed=11))
        run = lambda: s.solve_ktable(b)
        n_sys = cols.n_systems
    else:
        raise SystemExit(f"unknown case {case}")
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    s.close()
    print("ok", case, ncols, n_sys)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
