"""The benchmark's contract pieces that run without a GPU: the reference arm
(the oracle timed on the host on a bounded sample) prints one JSON line with
the contract's keys, and the ncu-summary reader accepts only a summary taken
on the current kernel source."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.fixture(scope="module")
def reference_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT, check=True)
    lines = [l for l in out.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_line_has_the_contract_keys(reference_line):
    l = reference_line
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"):
        assert k in l, k
    assert l["impl"] == "reference" and l["n_gpus"] == 1 and l["steps"] == 1 and l["warmup"] == 3
    assert l["higher_is_better"] is True and l["value"] > 0 and l["ms_per_step"] > 0
    assert "workload" in l["config"]
    assert l["e2e"]["value"] == l["value"] and l["e2e"]["h2d_bytes_per_step"] == 0
    cb = l["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == l["value"] and cb["sample"]


def test_reference_arm_uses_the_main_metric(reference_line):
    assert reference_line["metric"] == bench.METRIC and reference_line["unit"] == bench.UNIT


def test_profile_summary_is_used_only_for_the_current_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    body = "# header\nflop_per_system: 10.0\nfp32_pipe_ops_per_system: 7.0\ndram_bytes_per_launch: 5\n"
    (prof / "x.txt").write_text(body + f"source_sha1: {bench.kernel_source_sha1()}\n")
    (prof / "y.txt").write_text(body + "source_sha1: 0000\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the hash of the kernel sources is read from the real tree
    monkeypatch.setattr(bench, "kernel_source_sha1", lambda: (prof / "x.txt").read_text().split()[-1])
    got = bench.read_profile("x.txt")
    assert got is not None and float(got["fp32_pipe_ops_per_system"]) == 7.0
    assert bench.read_profile("y.txt") is None
    assert bench.read_profile("missing.txt") is None


def test_kernel_source_hash_is_stable():
    assert bench.kernel_source_sha1() == bench.kernel_source_sha1()
    assert len(bench.kernel_source_sha1()) == 40


def test_algorithmic_count_is_the_per_equation_table():
    f, m = bench.algorithmic_ops_per_system(40)
    per_layer_f = sum(v[0] for v in bench.ALG_LAYER.values())
    per_layer_m = sum(v[1] for v in bench.ALG_LAYER.values())
    assert (per_layer_f, per_layer_m) == (121, 11)
    assert (f, m) == (40 * 121 + bench.ALG_BOA[0], 40 * 11 + bench.ALG_BOA[1]) == (4848, 441)


def test_metrics_log_writes_one_record_per_section(tmp_path):
    line = {"value": 2.0e9, "unit": "solves/s", "ms_per_step": 0.7,
            "roofline": {"frac": 0.3, "hbm": {"frac": 0.18}, "mufu": {"frac": 0.22}},
            "fp64_plain": {"value": 1.4e7}, "e2e": {"value": 1.1e8},
            "branch_counts": {"resonance_hits": 354}, "sweeps": {"runs": []},
            "serving": {"p50_ms": 2.8, "p99_ms": 31.0},
            "fp32_error_vs_fp64": {"F_net": {"max_rel": 0.3, "max_err_over_tol": 0.32}}}
    path = tmp_path / "m.jsonl"
    bench.write_metrics_log(str(path), line)
    bench.write_metrics_log(str(path), line)
    recs = [json.loads(l) for l in path.read_text().splitlines()]
    sections = [r["section"] for r in recs]
    assert sections.count("gcm_fp32_form") == 2 and "serving" in sections and "host" in sections
    first = recs[0]
    assert first["roofline_frac"] == 0.3 and first["value"] == 2.0e9 and "time" in first
    assert next(r for r in recs if r["section"] == "serving")["p99_ms"] == 31.0
    assert next(r for r in recs if r["section"] == "fp32_error_vs_fp64")["F_net"]["max_err_over_tol"] == 0.32


def test_bench_accuracy_block_matches_the_parity_tolerances(monkeypatch):
    """The bench line's fp32_error_vs_fp64 uses the parity tests' FP32
    tolerance (same floors, same formula) on the outputs it is given."""
    import numpy as np
    import torch
    import rt_synth
    from parity import errors
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    cols = rt_synth.generate([5, 3, 7], [4, 2, 3], 2, seed=1)
    n_if, n_l = int((cols.n_layers + 1).sum()), int(cols.n_layers.sum())
    rng = np.random.default_rng(0)
    ref = {k: rng.uniform(-2, 2, n_if) for k in ("F_up", "F_down", "F_net")}
    ref["Q"] = rng.uniform(-2, 2, n_l)
    got = {k: v * (1 + 3e-5) + 1e-3 for k, v in ref.items()}
    e = bench.fp32_errors(cols, {k: torch.tensor(v) for k, v in got.items()},
                          {k: torch.tensor(v) for k, v in ref.items()})
    p = errors(cols, got, ref, "fp32")
    for k in ("F_up", "F_down", "F_net", "Q"):
        assert abs(e[k]["max_err_over_tol"] - p[k]) <= 1e-12 * p[k]
        assert e[k]["max_err_over_strict_tol"] >= e[k]["max_err_over_tol"]
