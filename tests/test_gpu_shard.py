"""Column sharding with the CUDA library: a batch cut by ``shard.partition``
into contiguous column slices, each solved on its own (as each rank would
on its own GPU), reassembles into the unsharded result bit for bit --
columns are independent and every column's spectral sums run in a fixed
order.  Here the slices run one after another on one GPU."""
import numpy as np
import pytest

import rt_synth
from paper_2203_02293_b300.shard import partition
from parity import gpu_solve, method_opts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("world", [2, 3])
def test_slices_reassemble_the_unsharded_result(precision, world):
    L, NB = rt_synth.uneven_shapes(48, seed=3)          # config 3's shape distribution
    cols = rt_synth.generate(L, NB, 20 if precision == "fp32" else 4, seed=3, optics="uniform")
    full = gpu_solve(cols, method_opts(), precision)
    parts = partition(cols.n_layers, cols.n_bins, world)
    assert parts[0][0] == 0 and parts[-1][1] == cols.n_cols
    pieces = [gpu_solve(cols.subset(np.arange(a, b)), method_opts(), precision) for a, b in parts]
    for k in ("F_up", "F_down", "F_net", "Q", "F_up_toa"):
        joined = np.concatenate([p[k] for p in pieces])
        assert np.array_equal(joined, full[k]), k
    assert sum(p["stats"]["etau_hits"] for p in pieces) == full["stats"]["etau_hits"]
