"""The workload definitions (rt_synth/configs.json) and the generators that
read them: shapes, distributions' ranges and seeds as stated."""
import numpy as np

import rt_synth


def test_configs_file_defines_the_five_workloads():
    c = rt_synth.CONFIGS
    assert set(c) == {"config0", "config1", "config2", "config3", "config4"}
    assert (c["config0"]["n_cols"], c["config0"]["layers"], c["config0"]["bins"], c["config0"]["g_points"]) == (64, 40, 30, 1)
    for k in ("config1", "config2"):
        assert (c[k]["n_cols"], c[k]["layers"], c[k]["bins"], c[k]["g_points"]) == (2562, 40, 30, 20)
    assert c["config3"]["layers"] == [20, 200] and c["config3"]["bins"] == [30, 300] and c["config3"]["n_cols"] == 4096
    assert c["config4"]["rate_hz"] == 200.0 and c["config4"]["columns"] == [1, 2562] and c["config4"]["layers"] == [40, 100]
    assert [c[f"config{i}"]["seed"] for i in range(5)] == [0, 1, 2, 3, 4]


def test_generators_follow_the_file():
    a = rt_synth.config0()
    assert a.n_cols == 64 and set(a.n_layers) == {40} and set(a.n_bins) == {30} and a.n_g == 1
    assert np.all(a.dtau >= 1e-6 * (1 - 1e-6)) and np.all(a.dtau <= 10 * (1 + 1e-6))
    assert np.all((a.w0 >= 0) & (a.w0 <= 0.95)) and np.all((a.g0 >= 0) & (a.g0 <= 0.8))
    b = rt_synth.config2(n_cols=8)
    assert np.all((b.w0 >= 0.99) & (b.w0 <= 1 - 1e-6)) and np.all((b.g0 >= 0.5) & (b.g0 <= 0.95))
    L, NB = rt_synth.uneven_shapes(4096, rt_synth.CONFIGS["config3"]["seed"])
    assert L.min() >= 20 and L.max() <= 200 and NB.min() >= 30 and NB.max() <= 300
    assert L.min() == 20 and L.max() == 200          # 4096 draws reach both ends
