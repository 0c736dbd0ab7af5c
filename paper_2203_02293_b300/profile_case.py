"""One solve of the GCM-shaped workload (or its first N columns), for profilers.

    python -m paper_2203_02293_b300.profile_case fp32 2562

runs two solves of the same batch (the second is the one to capture with
``ncu -s 1 -c 1``) and exits 0.  The cubes of the full 2562-column batch are
738 MB, above the 126 MB L2, and the whole run holds under 1 GB on the device.
"""
import sys

import torch

import rt_synth
from paper_2203_02293_b300 import rt
from paper_2203_02293_b300.solver import DeviceBatch, Solver


def main(argv):
    prec = argv[1] if len(argv) > 1 else "fp32"
    ncols = int(argv[2]) if len(argv) > 2 else 2562
    cols = rt_synth.config1(n_cols=ncols)
    b = DeviceBatch(cols)
    s = Solver(cols.g_weights, precision=rt.RT_FP32_FORM if prec == "fp32" else rt.RT_FP64_PLAIN)
    for _ in range(2):
        s.solve(b)
    torch.cuda.synchronize()
    s.close()
    print("ok", prec, ncols, cols.n_systems)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
