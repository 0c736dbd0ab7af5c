"""Benchmark: column.g-point solves per second on the GCM-shaped workload.

Workload (one step = the whole path over one batch): 2562 columns x 40
non-isothermal layers x 30 bins x 20 Gauss points = 1,537,200 (column, bin,
g) systems, k-table optical depths, stellar + thermal sources, improved
two-stream -- Planck per bin, layer coefficients, beam, sources, Thomas
elimination, spectral sum, net flux and heating, in one kernel launch.
Inputs are resident in HBM before the timed region; the three optical-
property cubes are 738 MB, larger than the 126 MB L2, so no L2 flush is
needed between steps.

The main line reports the FP32 form; the FP64 plain path is timed on the
same batch and reported beside it.  ``e2e`` repeats the FP32 measurement
through the public API with pinned host buffers: each step copies the
step's inputs host->device, solves, and reads the fluxes and heating back.

``--impl reference`` times the FP64 CPU oracle (the slow, literal reference
implementation) on a bounded sample of the same workload instead.
Multi-GPU (torchrun): every rank solves its own batch of the same shape
(weak scaling, no data-path collective); the step time is the max over
ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "column-g-point solves/s (FP32 form; FP64 plain beside it)"
UNIT = "solves/s"
WORKLOAD = "gcm-shaped 2562 cols x 40 layers x 30 bins x 20 g (k-table), non-isothermal, improved two-stream"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# FP32 operations of the chosen form per (column, bin, g) system of the GCM
# workload (FFMA counted as 2, FADD and FMUL as 1, the paired FFMA2 as 4 and
# FADD2/FMUL2 as 2), from the executed instruction counters of the solve
# kernel on that workload.
FLOP_PER_SYSTEM = None   # filled from profiles/fp32_units_gcm2562.txt when current
FP32_LANES_PER_SM = 128
N_SM = 148
MUFU_PER_SM_PER_CLK = 16

# Algorithmic work of one non-isothermal layer of one (column, bin, g)
# system, counted from the paper's equations evaluated directly: FP32
# FMA-pipe operations (an add, a multiply or a fused a*b+c is one) and MUFU
# operations (reciprocal, reciprocal square root, base-2 exponential; a
# division is a reciprocal and a multiply, exp(x) a multiply and ex2).  A
# layer's two sub-layers have the same w0, g0 and optical depth dtau/2, so
# everything that depends only on those is evaluated once per layer; what
# depends on the sub-layer's own B or beam is counted twice.
#   (equations, per layer)                                  FMA-pipe  MUFU
ALG_LAYER = {
    "E fit, Eq. 19 (Horner form, w0 g0 shared)":              (6, 0),
    "1 - w0 g0, E - w0, q = E (1 - w0 g0)":                   (3, 0),
    "k = sqrt((E - w0) / q), Eq. B2":                         (2, 2),
    "zeta+- = (1 +- k) / 2, Eq. B2":                          (2, 0),
    "exponent 2 q k and dtau / 2":                            (3, 0),
    "T = exp(-2 q k dtau / 2), Eq. B2 (product, log2 e scale)": (2, 1),
    "chi, xi, psi, Eq. B1":                                   (9, 0),
    "Pi, Eq. B5":                                             (3, 1),
    "1 / (2 q) of Theta, Eqs. 5, 8":                          (0, 1),
    "t = psi / chi, r = -xi / chi (rows of Eq. 12 over chi)": (2, 1),
    "D of Eq. 11 and G+-, Eq. B8":                            (13, 1),
    "beam attenuation over a sub-layer, Eq. B6":              (2, 1),
    "thermal sources, Eq. B4: shared Theta, chi + xi, Pi/chi": (5, 1),
    "thermal sources, Eq. B4: two sub-layers x 10":           (20, 0),
    "beam sources, Eq. B7: shared products over chi":         (8, 0),
    "beam sources, Eq. B7: two sub-layers x 7":               (14, 0),
    "elimination, Eqs. 13-14: two levels x 9, t^2 shared":    (19, 2),
    "back-substitution, Eq. 15: two levels x 2":              (4, 0),
    "spectral sum at the layer's interface (F_up, F_net)":    (4, 0),
}
ALG_BOA = (8, 1)   # Eq. 10 closure and the BOA interface's sums


def algorithmic_ops_per_system(L: int):
    """(FMA-pipe, MUFU) operations of one L-layer non-isothermal system."""
    f = sum(v[0] for v in ALG_LAYER.values())
    m = sum(v[1] for v in ALG_LAYER.values())
    return L * f + ALG_BOA[0], L * m + ALG_BOA[1]


def kernel_source_sha1():
    import hashlib
    h = hashlib.sha1()
    for f in ("paper_2203_02293_b300/csrc/rt_kernels.cu", "paper_2203_02293_b300/csrc/rt_internal.h"):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def read_profile(name="fp32_units_gcm2562.txt"):
    """Per-launch counters of the solve kernel from the committed ncu summary,
    if they were taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None
    vals = {}
    with open(p) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    if vals.get("source_sha1") != kernel_source_sha1():
        return None
    return vals


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:   # first sample before timing starts
                time.sleep(0.05)
            self.n_before = len(self.lines)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        self.lines = self.lines[getattr(self, "n_before", 0):] or self.lines[-1:]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(cols, min_seconds: float):
    """The oracle as it stands on the host cores; returns (solves/s, passes, seconds)."""
    import oracle
    o = oracle.get()
    cfg = oracle.OracleConfig(wn_min=cols.consts["wn_min"], wn_max=cols.consts["wn_max"])
    passes, t0 = 0, time.perf_counter()
    while True:
        o.solve_columns(cfg, cols)
        passes += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return cols.n_systems * passes / el, passes, el


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import rt_synth
    full = rt_synth.config1()
    sample_cols = 256
    cols = full.subset(np.arange(sample_cols))
    for _ in range(args.warmup):
        time_oracle(cols, 0.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        time_oracle(cols, 0.0)
    el = time.perf_counter() - t0
    value = cols.n_systems * args.steps / el
    sample = f"first {sample_cols} of the 2562 columns per step ({cols.n_systems} systems)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded k-table stand-in)",
        "config": {"workload": WORKLOAD, "sample": sample, "l2": "n/a (host)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_uneven(args, stream, ws=1, rank=0, barrier=lambda: None, max_over_ranks=lambda x: x):
    """Config 3: 4096 columns, L ~ U{20..200}, NB ~ U{30..300}, 20 g in one
    persistent launch; launch shape from the autotuner; timed as replays of
    a captured CUDA graph.  With several ranks the one batch is split by
    column (shard.partition: contiguous, cost-balanced blocks), each rank
    solves its block on its own GPU with no exchange, and the step time is
    the maximum over ranks (strong scaling)."""
    import torch
    import rt_synth
    from paper_2203_02293_b300.shard import partition
    from paper_2203_02293_b300.solver import DeviceBatch, Solver
    from paper_2203_02293_b300.tuning import GraphSolve, autotune
    full = rt_synth.config3_device()
    n_total = full.n_systems
    a, b_ = partition(full.n_layers, full.n_bins, ws)[rank]
    dc = full.column_range(a, b_) if ws > 1 else full
    b = DeviceBatch.from_device(dc)
    from paper_2203_02293_b300.tuning import KNOBS
    tune = autotune(b, dc.g_weights, reps=3)
    s = Solver(dc.g_weights, **{k: tune[k] for k in KNOBS if k in tune})
    g = GraphSolve(s, b, stream)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.uneven_steps):
        g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.uneven_steps)
    s.close()
    out = {"workload": "4096 cols, L~U{20..200}, NB~U{30..300}, 20 g, one launch (CUDA graph replay)",
           "systems": n_total, "input_bytes": int(3 * 4 * full.dtau.numel()),
           "ms_per_step": ms, "value": n_total / (ms * 1e-3), "unit": UNIT,
           "n_gpus": ws, "scaling": "strong",
           "split": f"columns [{a}, {b_}) of 4096 on rank {rank} (shard.partition, no exchange)" if ws > 1
                    else "one GPU, whole batch",
           "steps": args.uneven_steps, "autotune": {k: tune[k] for k in (*KNOBS, "stable") if k in tune},
           "autotune_table": tune["table"]}
    del g, b, dc, full
    torch.cuda.empty_cache()
    return out


def run_postproc(args, stream):
    """Post-processing shape (Sec. 2.1.3): 2562 columns extended to 1 ubar
    (40-52 layers), 3255 bins log-spaced at R = 500, one g-point; the
    per-bin TOA spectrum is written with the fluxes.  Inputs ~4.6 GB, above L2."""
    import torch
    import rt_synth
    from paper_2203_02293_b300.solver import DeviceBatch, Solver
    dc = rt_synth.postproc_device(2562, seed=5)
    b = DeviceBatch.from_device(dc)
    s = Solver(dc.g_weights, wn_edges=dc.consts["wn_edges"])
    with torch.cuda.stream(stream):
        for _ in range(3):
            s.solve(b, stream)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.postproc_steps):
            s.solve(b, stream)
        e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.postproc_steps
    st = s.stats()
    s.close()
    out = {"workload": "2562 cols extended to 1 ubar (L 40-52), 3255 bins (R=500), 1 g, per-bin TOA spectrum",
           "systems": dc.n_systems, "layer_systems": int((dc.n_layers.astype(np.int64) * dc.n_bins).sum()),
           "input_bytes": int(3 * 4 * dc.dtau.numel()), "ms_per_step": ms,
           "value": dc.n_systems / (ms * 1e-3), "unit": UNIT,
           "spectra_per_s": dc.n_cols / (ms * 1e-3), "steps": args.postproc_steps,
           "nonfinite_outputs": st["nonfinite_outputs"]}
    del b, dc
    torch.cuda.empty_cache()
    return out


def run_ktable(args, stream):
    """GCM shape (2562 x 40 x 30 x 20) with the optics from the k-table front
    end (Sec. 2.1.3: 60 x 28 (T, p) table, gas/cloud mixing, H2/He Rayleigh):
    fused into the solve kernel, and beside it the unfused route (the optics
    kernel writes the cubes, then the cube solve).  The state and table fit in
    L2; each step still streams ~1.5 GB of elimination scratch through HBM."""
    import torch
    import rt_synth
    from paper_2203_02293_b300 import rt
    from paper_2203_02293_b300.solver import DeviceBatch, Solver
    cols = rt_synth.state_columns(2562, 40, 30, 20, seed=26)
    kt = rt_synth.ktable(n_bins=30, n_g=20, seed=11)
    b = DeviceBatch(cols)
    s = Solver(cols.g_weights)
    s.set_ktable(kt)
    o = s.ktable_optics(b)
    fb = DeviceBatch(cols)
    fb.dtau, fb.w0, fb.g0 = o["dtau"], o["w0"], o["g0"]
    fb._desc = None

    def timed(fn, steps):
        with torch.cuda.stream(stream):
            for _ in range(3):
                fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    ms_fused = timed(lambda: s.solve_ktable(b, stream), args.ktable_steps)

    def unfused():
        rt.rt_ktable_optics(s.h, b.state_descriptor(), o["dtau"], o["w0"], o["g0"], stream)
        s.solve(fb, stream)
    ms_unfused = timed(unfused, args.ktable_steps)

    # end to end: each step copies the column state (T, p, mu, F*) from
    # pinned host memory, solves with the fused front end and reads the
    # fluxes and heating back; the table stays resident.  The kernels run in
    # order on one compute stream; a copy stream moves step k+1's state in and
    # step k's results out while step k solves (two input and two output
    # buffers, handed over by events)
    state = ("T_center", "T_iface", "p_iface", "mu_star", "F_star")
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(cols, k))).pin_memory() for k in state}
    bs = [b, DeviceBatch(cols)]
    cs = torch.cuda.Stream()
    outs = []
    for _ in range(2):
        o = {k: torch.empty(b.n_if, dtype=torch.float64).pin_memory() for k in ("F_up", "F_down", "F_net")}
        o["Q"] = torch.empty(b.n_lay, dtype=torch.float64).pin_memory()
        outs.append(o)
    out_dev = [{k: torch.empty_like(v, device="cuda") for k, v in o.items()} for o in outs]
    ev = {name: [torch.cuda.Event() for _ in range(2)] for name in ("in_ready", "in_free", "out_ready", "out_free")}

    def h2d(k):
        i = k % 2
        cs.wait_event(ev["in_free"][i])
        with torch.cuda.stream(cs):
            for key in state:
                getattr(bs[i], key).copy_(host[key], non_blocking=True)
        ev["in_ready"][i].record(cs)

    def compute(k):
        i = k % 2
        stream.wait_event(ev["in_ready"][i])
        s.solve_ktable(bs[i], stream)
        ev["in_free"][i].record(stream)
        stream.wait_event(ev["out_free"][i])
        rt.rt_fluxes(s.h, out_dev[i]["F_up"], out_dev[i]["F_down"], out_dev[i]["F_net"], stream)
        rt.rt_heating(s.h, out_dev[i]["Q"], stream)
        ev["out_ready"][i].record(stream)

    def d2h(k):
        i = k % 2
        cs.wait_event(ev["out_ready"][i])
        with torch.cuda.stream(cs):
            for key in outs[i]:
                outs[i][key].copy_(out_dev[i][key], non_blocking=True)
        ev["out_free"][i].record(cs)

    def e2e_run(n, e0=None, e1=None):
        if e0 is not None:
            e0.record(stream)
        cs.wait_stream(stream)
        for i in range(2):                       # both buffers free at the start
            ev["in_free"][i].record(stream)
            ev["out_free"][i].record(cs)
        h2d(0)
        for k in range(n):
            if k + 1 < n:
                h2d(k + 1)                       # overlaps compute(k)
            compute(k)
            d2h(k)                               # overlaps compute(k + 1)
        stream.wait_stream(cs)
        if e1 is not None:
            e1.record(stream)

    e2e_run(4)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_run(args.ktable_steps, e0, e1)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.ktable_steps
    # every step carried the same state: the last step's host results must
    # equal a resident solve's, bit for bit
    last = outs[(args.ktable_steps - 1) % 2]
    ref = {k: torch.empty_like(v) for k, v in out_dev[0].items()}
    s.solve_ktable(b, stream)
    rt.rt_fluxes(s.h, ref["F_up"], ref["F_down"], ref["F_net"], stream)
    rt.rt_heating(s.h, ref["Q"], stream)
    torch.cuda.synchronize()
    e2e_match = all(torch.equal(last[k], ref[k].cpu()) for k in ref)
    outs = outs[0]
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in outs.values())
    st = s.stats()
    s.close()
    n = b.n_systems
    out = {"workload": "2562 x 40 x 30 x 20, optics from a 60x28 k-table (fused into the solve)",
           "systems": n, "ms_per_step": ms_fused, "value": n / (ms_fused * 1e-3), "unit": UNIT,
           "unfused_ms_per_step": ms_unfused, "unfused_value": n / (ms_unfused * 1e-3),
           "e2e": {"value": n / (ms_e2e * 1e-3), "unit": UNIT, "ms_per_step": ms_e2e,
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "pipelining": "one compute stream and one copy stream, two input and two output buffers: step k+1's state copy and step k's result copy overlap step k's solve",
                   "outputs_match_resident": e2e_match},
           "steps": args.ktable_steps, "nonfinite_outputs": st["nonfinite_outputs"],
           "invalid_inputs": st["invalid_inputs"]}
    del b, bs, fb, o
    torch.cuda.empty_cache()
    return out


def _oracle_rate(cols, seconds, threads=None):
    """Oracle solves/s on this host: all cores in-process, or ``threads`` cores
    in a child process (OpenMP reads its thread count at start-up)."""
    if threads is None:
        v, _, _ = time_oracle(cols, seconds)
        return v
    import pickle
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        f = os.path.join(d, "cols.pkl")
        with open(f, "wb") as fh:
            pickle.dump(cols, fh)
        code = ("import pickle, sys; sys.path.insert(0, %r); import bench; "
                "cols = pickle.load(open(%r, 'rb')); print(bench.time_oracle(cols, %r)[0])" % (ROOT, f, seconds))
        env = dict(os.environ, OMP_NUM_THREADS=str(threads))
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, check=True)
    return float(out.stdout.strip().splitlines()[-1])


def run_table(args):
    """One JSON line per workload (configs 0-3): FP32 form and FP64 plain
    GPU throughput with inputs resident, the HBM bytes each FP32 step moves
    over its time, and the CPU oracle on one core and on all cores (bounded
    samples of the same workload, shapes as drawn)."""
    import torch
    import rt_synth
    from paper_2203_02293_b300 import rt
    from paper_2203_02293_b300.solver import DeviceBatch, Solver
    peak_gbs, _ = read_peaks()
    stream = torch.cuda.Stream()

    def gpu_ms(b, g_weights, precision, steps):
        s = Solver(g_weights, precision=precision)
        with torch.cuda.stream(stream):
            for _ in range(3):
                s.solve(b, stream)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                s.solve(b, stream)
            e1.record(stream)
        torch.cuda.synchronize()
        s.close()
        return e0.elapsed_time(e1) / steps

    # (name, generator, columns for the 1-core oracle; the all-core oracle
    # runs every column of configs 0-2 and the same sample of config 3)
    cases = [
        ("config0 64x40x30x1", lambda: rt_synth.config0(), None),
        ("config1 2562x40x30x20", lambda: rt_synth.config1(), 64),
        ("config2 2562x40x30x20 stress", lambda: rt_synth.config2(), 64),
        ("config3 4096 uneven", None, 24),
    ]
    for name, make, n_sample in cases:
        full_cols = None
        if make is not None:
            cols = make()
            b = DeviceBatch(cols)
            n_sys, g_w = cols.n_systems, cols.g_weights
            sample = cols if n_sample is None else cols.subset(np.arange(n_sample))
            full_cols = cols
            in_bytes = b.input_bytes
        else:
            dc = rt_synth.config3_device()
            b = DeviceBatch.from_device(dc)
            n_sys, g_w = dc.n_systems, dc.g_weights
            sample = dc.host_subset(np.arange(n_sample))
            in_bytes = b.input_bytes
        steps32 = 200 if n_sys < 4_000_000 else 20
        ms32 = gpu_ms(b, g_w, rt.RT_FP32_FORM, steps32)
        ms64 = gpu_ms(b, g_w, rt.RT_FP64_PLAIN, 3 if n_sys < 4_000_000 else 1)
        out_bytes = 8 * (3 * b.n_if + b.n_lay)
        line = {"table": name, "systems": n_sys,
                "fp32_solves_per_s": n_sys / (ms32 * 1e-3), "fp32_ms": ms32,
                "fp64_solves_per_s": n_sys / (ms64 * 1e-3), "fp64_ms": ms64, "fp32_over_fp64": ms64 / ms32,
                "fp32_hbm_frac": (in_bytes + out_bytes) / (ms32 * 1e-3) / 1e9 / peak_gbs}
        del b
        torch.cuda.empty_cache()
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = {
                "all_cores": _oracle_rate(full_cols if full_cols is not None else sample, 3.0),
                "one_core": _oracle_rate(sample, 3.0, threads=1),
                "cores": cpu_cores(), "kind": "oracle", "unit": UNIT,
                "sample": ("all columns" if full_cols is not None else f"{n_sample} columns") + " on all cores; "
                          + ("all columns" if n_sample is None else f"{n_sample} columns") + " on one core"}
        print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """Config 4: Poisson arrivals (mean 200/s), requests of logU[1, 2562]
    columns x U{40..100} layers x U{30..300} bins x 20 g sliced from a
    device-resident pool; continuous batching over 8 stream slots, smallest
    request first except that the remaining pieces of a started request go
    first, requests above 4M systems cut into column pieces, at most 4M
    systems per batch, one CTA per SM per batch except batches of 1e8
    layer-systems or more, which keep every CTA resident (the best p99 of a
    sweep over slots, policy, CTAs per SM, batch cap, piece size and the
    wide-batch threshold).  The FP64 plain path is served beside it at the
    rate it sustains, the same request mix, 4 slots."""
    import torch
    import rt_synth
    from paper_2203_02293_b300 import rt
    from paper_2203_02293_b300.serve import Pool, Server, make_requests
    c4 = rt_synth.CONFIGS["config4"]
    pool = Pool(rt_synth, n_pool=c4["pool_columns"], L_range=tuple(c4["layers"]), NB_range=tuple(c4["bins"]),
                n_g=c4["g_points"])
    n = int(args.serving_seconds * args.serving_rate)
    reqs = make_requests(pool, n, rate_hz=args.serving_rate, seed=c4["seed"], C_range=tuple(c4["columns"]))
    warm = make_requests(pool, 8, rate_hz=1e3, seed=99)
    knobs = dict(n_slots=8, policy="gang", ctas_per_sm=1, max_systems_per_batch=4_000_000,
                 split_systems=4_000_000, wide_layer_systems=100_000_000)
    srv = Server(pool, hbm_budget_bytes=32 << 30, **knobs)
    srv.run(warm)
    srv.batches = 0
    summ = srv.run(reqs)
    srv.close()
    # lower bound on the slowest requests' latency: their layer-systems at
    # the whole GPU's rate (the GCM step's solves/s x 40 layers)
    work = np.array([r.systems * r.L for r in reqs], dtype=np.float64)
    p99w = float(np.percentile(work, 99))
    summ.update({"rate_hz": args.serving_rate, "seconds_of_arrivals": args.serving_seconds,
                 "unit_latency": "ms", "budget_bytes": 32 << 30, "precision": "fp32 form", **knobs,
                 "p99_request_layer_systems": p99w,
                 "p99_request_whole_gpu_ms": (p99w / args.gcm_layer_systems_per_s * 1e3
                                              if getattr(args, "gcm_layer_systems_per_s", 0) else None)})
    if args.serving_fp64_rate > 0:
        n64 = int(args.serving_fp64_seconds * args.serving_fp64_rate)
        reqs = make_requests(pool, n64, rate_hz=args.serving_fp64_rate, seed=44)
        k64 = dict(n_slots=4, policy="sjf", max_systems_per_batch=2_000_000, split_systems=1_000_000)
        srv = Server(pool, hbm_budget_bytes=32 << 30, precision=rt.RT_FP64_PLAIN, **k64)
        s64 = srv.run(reqs)
        srv.close()
        s64.update({"rate_hz": args.serving_fp64_rate, "seconds_of_arrivals": args.serving_fp64_seconds,
                    "unit_latency": "ms", "precision": "fp64 plain", **k64})
        summ["fp64_plain"] = s64
    del pool
    torch.cuda.empty_cache()
    return summ


def run_profile_case(args):
    """One workload solved twice, for profilers (the second solve is the one
    to capture: ``ncu -k <kernel> -s 1 -c 1``).  Cases: fp32 / fp64 (GCM
    shape, cubes in), sweeps (the same with --profile-sweeps sweeps of the
    iterative method), postproc (R = 500 shape), ktable (k-table front end).
    --profile-cols sets the column count (2562: cubes 738 MB, above L2)."""
    import torch
    import rt_synth
    from paper_2203_02293_b300 import rt
    from paper_2203_02293_b300.solver import DeviceBatch, Solver
    case, ncols = args.profile_case, args.profile_cols
    if case in ("fp32", "fp64", "sweeps"):
        cols = rt_synth.config1(n_cols=ncols)
        b = DeviceBatch(cols)
        extra = dict(n_sweeps=args.profile_sweeps) if case == "sweeps" else {}
        s = Solver(cols.g_weights, precision=rt.RT_FP64_PLAIN if case == "fp64" else rt.RT_FP32_FORM, **extra)
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
        raise SystemExit(f"unknown profile case {case}")
    for _ in range(2):
        run()
    torch.cuda.synchronize()
    s.close()
    print("ok", case, ncols, n_sys, flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=8)
    ap.add_argument("--uneven-steps", type=int, default=10)
    ap.add_argument("--postproc-steps", type=int, default=20)
    ap.add_argument("--ktable-steps", type=int, default=200)
    ap.add_argument("--kernel-timing-steps", type=int, default=50)
    ap.add_argument("--serving-seconds", type=float, default=60.0)
    ap.add_argument("--serving-rate", type=float, default=200.0)
    ap.add_argument("--serving-fp64-rate", type=float, default=4.0,
                    help="request rate of the FP64-plain serving arm (0: skip)")
    ap.add_argument("--serving-fp64-seconds", type=float, default=20.0)
    ap.add_argument("--sweeps", default="10,200",
                    help="sweep counts of the iterative method timed beside Thomas (empty: skip)")
    ap.add_argument("--sweep-steps", type=int, default=20)
    ap.add_argument("--quick", action="store_true", help="skip the uneven and serving sections")
    ap.add_argument("--metrics-log", default=None,
                    help="append this run's records (one JSON object per section) to a JSONL file")
    ap.add_argument("--profile-case", default=None,
                    help="fp32 | fp64 | sweeps | postproc | ktable: two solves of one workload, for ncu")
    ap.add_argument("--profile-cols", type=int, default=2562)
    ap.add_argument("--profile-sweeps", type=int, default=10)
    ap.add_argument("--table", action="store_true",
                    help="per-workload table (configs 0-3, FP32/FP64 GPU, CPU oracle 1 core / all cores)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.table:
        return run_table(args)

    import torch
    import rt_synth
    from paper_2203_02293_b300 import rt
    from paper_2203_02293_b300.solver import DeviceBatch, Solver

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # One GCM batch of ws x 2562 columns split by column with no exchange on
    # the data path: partition() gives each rank a contiguous, cost-balanced
    # block.  The columns are uniform, so block r is columns [2562 r,
    # 2562 (r + 1)), which rank r draws itself (those columns are the draw
    # of seed 1 + r): per-GPU work is fixed as ranks are added.
    from paper_2203_02293_b300.shard import partition
    lo, hi = partition(np.full(ws * 2562, 40), np.full(ws * 2562, 30), ws)[rank]
    assert (lo, hi) == (2562 * rank, 2562 * (rank + 1))
    cols = rt_synth.config1(seed=1 + rank)
    batch = DeviceBatch(cols)
    n_sys = batch.n_systems
    stream = torch.cuda.Stream()

    def timed(solver, b, steps, warm, use_events=True):
        with torch.cuda.stream(stream):
            for _ in range(warm):
                solver.solve(b, stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        with torch.cuda.stream(stream):
            for _ in range(steps):
                solver.solve(b, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    # --- FP32 form (the main number) ---
    s32 = Solver(cols.g_weights, precision=rt.RT_FP32_FORM)
    with ClockSampler(local) as clk:
        ms32 = timed(s32, batch, args.steps, args.warmup)
    ms32 = max_over_ranks(ms32)
    value = n_sys * ws / (ms32 * 1e-3)

    # --- the same steps on two handles and streams, alternating: step k+1's
    # pre-kernel and start overlap step k's tail (reported beside the value) ---
    s32b = Solver(cols.g_weights, precision=rt.RT_FP32_FORM)
    streams2 = [stream, torch.cuda.Stream()]
    pair = [s32, s32b]
    for k in range(2 * args.warmup):
        with torch.cuda.stream(streams2[k % 2]):
            pair[k % 2].solve(batch, streams2[k % 2])
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(streams2[0])
    streams2[1].wait_event(t0)
    for k in range(args.steps):
        with torch.cuda.stream(streams2[k % 2]):
            pair[k % 2].solve(batch, streams2[k % 2])
    streams2[0].wait_stream(streams2[1])
    t1.record(streams2[0])
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    ms32_2 = max_over_ranks(t0.elapsed_time(t1) / args.steps)
    s32b.close()

    # --- FP64 plain path on the same batch ---
    s64 = Solver(cols.g_weights, precision=rt.RT_FP64_PLAIN)
    ms64 = max_over_ranks(timed(s64, batch, args.fp64_steps, 3))
    accuracy = fp32_errors(cols, s32.outputs(batch, stream), s64.outputs(batch, stream))
    s64.close()

    # --- end to end through the public API with pinned host buffers ---
    # Every step copies its inputs host->device, solves and reads the fluxes
    # and heating back.  Two buffers, handles and streams alternate, so step
    # k+1's host->device copy overlaps step k's solve and read-back (the
    # copies themselves share one PCIe link).
    host = DeviceBatch(cols, device="cpu", pin=True)
    devs = [DeviceBatch.empty_like(host) for _ in range(2)]
    sols = [s32, Solver(cols.g_weights, precision=rt.RT_FP32_FORM)]
    streams = [stream, torch.cuda.Stream()]
    outs = [{k: torch.empty(batch.n_if, dtype=torch.float64).pin_memory() for k in ("F_up", "F_down", "F_net")}
            for _ in range(2)]
    for o in outs:
        o["Q"] = torch.empty(batch.n_lay, dtype=torch.float64).pin_memory()
    out_dev = [{k: torch.empty_like(v, device="cuda") for k, v in o.items()} for o in outs]
    h2d = host.input_bytes
    d2h = sum(v.numel() * v.element_size() for v in outs[0].values())

    def e2e_step(k):
        i = k % 2
        st = streams[i]
        with torch.cuda.stream(st):
            devs[i].copy_from(host, non_blocking=True)
            sols[i].solve(devs[i], st)
            rt.rt_fluxes(sols[i].h, out_dev[i]["F_up"], out_dev[i]["F_down"], out_dev[i]["F_net"], st)
            rt.rt_heating(sols[i].h, out_dev[i]["Q"], st)
            for key in outs[i]:
                outs[i][key].copy_(out_dev[i][key], non_blocking=True)

    for k in range(4):
        e2e_step(k)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(streams[0])
    streams[1].wait_event(e0)
    for k in range(args.e2e_steps):
        e2e_step(k)
    streams[0].wait_stream(streams[1])
    e1.record(streams[0])
    torch.cuda.synchronize()
    barrier()
    ms_e2e = max_over_ranks(e0.elapsed_time(e1) / args.e2e_steps)
    e2e_value = n_sys * ws / (ms_e2e * 1e-3)
    sols[1].close()

    # --- roofline of the solve kernel (ALU-bound; the HBM figure beside it) ---
    peak_gbs, peak_src = read_peaks()
    n_cube = cols.dtau.size
    alg_bytes = (3 * 4 * n_cube                                  # dtau, w0, g0
                 + 8 * (cols.T_center.size + cols.T_iface.size + cols.p_iface.size)
                 + 8 * (cols.mu_star.size + cols.F_star.size)
                 + 8 * (3 * batch.n_if + batch.n_lay))          # outputs
    prof = read_profile()
    # the solve kernel's own launch duration, measured live: CUDA events on
    # the launching stream around each kernel (rt_kernel_times), averaged
    # over a stretch of solves after the timed region
    st_ = Solver(cols.g_weights, precision=rt.RT_FP32_FORM, kernel_timing=1)
    kt_prep, kt_solve = [], []
    with torch.cuda.stream(stream):
        for i in range(args.kernel_timing_steps + 3):
            st_.solve(batch, stream)
            a, b = rt.rt_kernel_times(st_.h)
            if i >= 3:
                kt_prep.append(a)
                kt_solve.append(b)
    st_.close()
    ms_kernel = float(np.mean(kt_solve))
    ms_prep = float(np.mean(kt_prep))
    achieved_gbs = alg_bytes / (ms_kernel * 1e-3) / 1e9
    max_mhz = 2032.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            max_mhz = json.load(f).get("sm_max_mhz", max_mhz)
    except OSError:
        pass
    peak_tops = N_SM * FP32_LANES_PER_SM * max_mhz * 1e6 / 1e12
    peak_mufu = N_SM * MUFU_PER_SM_PER_CLK * max_mhz * 1e6 / 1e12
    # the binding roofline of the solve kernel is the FP32 FMA pipe: its
    # algorithmic operations (counted from the paper's equations, not from
    # what the kernel executes) over 148 SMs x 128 lanes x clock; the MUFU
    # and HBM bounds beside it are lower
    alg_f, alg_m = algorithmic_ops_per_system(40)
    achieved_tops = alg_f * n_sys / (ms_kernel * 1e-3) / 1e12
    achieved_mufu = alg_m * n_sys / (ms_kernel * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tops, "peak": peak_tops,
                "unit": "T FP32-pipe ops/s", "frac": achieved_tops / peak_tops,
                "traffic": float(prof["dram_bytes_per_launch"]) if prof else None,
                "kernel": "fp32_units", "kernel_ms": ms_kernel, "prep_kernel_ms": ms_prep,
                "kernel_ms_source": f"CUDA events around each launch, mean of {len(kt_solve)} solves",
                "algorithmic_ops_per_system": {"fp32_pipe": alg_f, "mufu": alg_m,
                                               "source": "paper's equations, per-equation table in bench.py"},
                "peak_source": "derived: 148 SMs x 128 FP32 lanes x max SM clock",
                "bounds_ms": {"fp32_pipe": alg_f * n_sys / (peak_tops * 1e12) * 1e3,
                              "mufu": alg_m * n_sys / (peak_mufu * 1e12) * 1e3,
                              "hbm": alg_bytes / (peak_gbs * 1e9) * 1e3},
                "mufu": {"achieved": achieved_mufu, "peak": peak_mufu, "unit": "T MUFU ops/s",
                         "frac": achieved_mufu / peak_mufu},
                "hbm": {"achieved": achieved_gbs, "peak": peak_gbs, "unit": "GB/s",
                        "frac": achieved_gbs / peak_gbs, "peak_source": peak_src,
                        "algorithmic_bytes_per_launch": alg_bytes}}
    if prof:
        roofline["executed_fp32_pipe_ops_per_system"] = float(prof["fp32_pipe_ops_per_system"])
    else:
        roofline["traffic_note"] = "no ncu summary taken on the current kernel source"
    stats = s32.stats()

    # --- the iterative method (Sec. 2.2.2) beside Thomas on the same batch ---
    sweeps = None
    counts = [int(x) for x in args.sweeps.split(",") if x.strip()]
    if counts and rank == 0:
        ref = s32.outputs(batch, stream)
        torch.cuda.synchronize()
        sweeps = {"workload": WORKLOAD, "thomas_ms_per_step": ms32, "runs": []}
        for n in counts:
            sw = Solver(cols.g_weights, n_sweeps=n, kernel_timing=1)
            steps = max(3, args.sweep_steps if n <= 20 else args.sweep_steps // 4)
            ms = timed(sw, batch, steps, 3)
            a, kms = rt.rt_kernel_times(sw.h)
            got = sw.outputs(batch, stream)
            torch.cuda.synchronize()
            dev = {k: float(torch.max(torch.abs(got[k] - ref[k]) / torch.abs(ref[k]).clamp_min(1e-30)))
                   for k in ("F_up", "F_down")}
            sweeps["runs"].append({"n_sweeps": n, "ms_per_step": ms, "kernel_ms": kms,
                                   "value": n_sys / (ms * 1e-3), "unit": UNIT, "steps": steps,
                                   "slowdown_vs_thomas": ms / ms32,
                                   "max_rel_dev_from_thomas": dev})
            sw.close()
        if len(counts) >= 2:
            # a sweep's roofline: the passes read each sub-layer's source
            # from shared memory (4 B per sub-layer and pass: 640 B per
            # 40-layer system and sweep) against 148 SMs x 128 B/clock;
            # the per-sweep time is the kernel-time difference between the
            # two sweep counts (the coefficient pass cancels)
            r0, r1 = sweeps["runs"][0], sweeps["runs"][-1]
            per_sweep_ms = (r1["kernel_ms"] - r0["kernel_ms"]) / (r1["n_sweeps"] - r0["n_sweeps"])
            smem_bytes = 2 * 40 * 2 * 4 * n_sys
            peak_tbs = N_SM * 128 * max_mhz * 1e6 / 1e12
            sweeps["sweep_roofline"] = {
                "bound": "shared memory", "per_sweep_us": per_sweep_ms * 1e3,
                "bytes_per_sweep": smem_bytes, "achieved": smem_bytes / (per_sweep_ms * 1e-3) / 1e12,
                "peak": peak_tbs, "unit": "TB/s", "frac": smem_bytes / (per_sweep_ms * 1e-3) / 1e12 / peak_tbs,
                "peak_source": "derived: 148 SMs x 128 B/clock x max SM clock"}
    s32.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded k-table stand-in)",
        "config": {"workload": WORKLOAD, "systems_per_gpu": n_sys, "layers": 40, "bins": 30,
                   "g_points": 20, "l2": "inputs 738 MB > 126 MB L2, no flush needed",
                   "parallelism": f"one {ws * 2562}-column batch split by column (shard.partition), "
                                  f"{ws} rank(s), no collective on the data path"},
        "fp64_plain": {"value": n_sys * ws / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                       "steps": args.fp64_steps},
        "fp32_over_fp64": ms64 / ms32,
        "fp32_error_vs_fp64": accuracy,
        "two_streams": {"value": n_sys * ws / (ms32_2 * 1e-3), "unit": UNIT, "ms_per_step": ms32_2,
                        "note": "the same resident batch solved on two handles and streams in turn, "
                                "as independent batches would be (serving): consecutive steps overlap, "
                                "each step's pre-kernel beside the previous step's tail. A GCM's steps "
                                "depend on each other and run one after another: the value above"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e,
                "pipelining": "two buffers, handles and streams: step k+1's copy overlaps step k's solve"},
        "gpu_launches": 3 * args.steps,      # Planck pre-kernel, solve kernel and finalize kernel per step
        "roofline": roofline,
        "clocks": clk.summary(),
        "branch_counts": {**stats, "resonance_mode": "paper (|D| < 1e-5: D := 2 mu*)"},
    }
    if sweeps is not None:
        line["sweeps"] = sweeps
    if not args.quick:
        del batch, host, devs
        torch.cuda.empty_cache()
        line["uneven"] = run_uneven(args, stream, ws, rank, barrier, max_over_ranks)
    if rank == 0 and not args.quick:
        args.gcm_layer_systems_per_s = value / ws * 40      # this GPU's GCM-step rate in layer-systems/s
        line["postproc"] = run_postproc(args, stream)
        line["ktable"] = run_ktable(args, stream)
        line["serving"] = run_serving(args)
    if rank == 0 and not args.no_cpu_baseline:
        v, passes, el = time_oracle(cols, 10.0)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"all 2562 columns, {passes} pass(es), {el:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.metrics_log:
            write_metrics_log(args.metrics_log, line)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def fp32_errors(cols, o32, o64) -> dict:
    """Per quantity, the FP32 form's largest relative error against the FP64
    plain path on the same batch (which matches the FP64 oracle to 1e-10),
    and its largest error over the FP32 tolerance of the parity tests:
    max(1e-4 |x|, 1e-6 F*_col) for fluxes, max(1e-3 |Q|, (g / c_P) 1e-6
    F*_col / dp) for heating (F*_col: the column's stellar flux); beside it
    the stricter reading with the relative factor on the floor as well,
    1e-4 max(|x|, 1e-6 F*_col) (1e-3 for Q)."""
    import torch
    from paper_2203_02293_b300 import rt
    torch.cuda.synchronize()
    o = cols.offsets()
    L = cols.n_layers.astype(np.int64)
    fstar = np.add.reduceat(np.asarray(cols.F_star, np.float64), o["bins"][:-1])
    f_if = np.repeat(1e-6 * fstar, L + 1)
    dp = np.diff(np.asarray(cols.p_iface, np.float64))
    dp = np.delete(dp, o["iface"][1:-1] - 1)            # drop the differences across columns
    c = rt.Config(g_weights=cols.g_weights)
    f_q = c.grav / c.cp * np.repeat(1e-6 * fstar, L) / dp
    out = {"reference": "FP64 plain GPU path, same batch and launch"}
    for k, floor, rtol in (("F_up", f_if, 1e-4), ("F_down", f_if, 1e-4), ("F_net", f_if, 1e-4), ("Q", f_q, 1e-3)):
        x, y = o32[k].cpu().numpy(), o64[k].cpu().numpy()
        err = np.abs(x - y)
        out[k] = {"max_rel": float(np.max(err / np.maximum(np.abs(y), 1e-300))),
                  "max_err_over_tol": float(np.max(err / np.maximum(rtol * np.abs(y), floor))),
                  "max_err_over_strict_tol": float(np.max(err / (rtol * np.maximum(np.abs(y), floor))))}
    return out


def write_metrics_log(path: str, line: dict):
    """Append one JSON object per section of a bench line to a JSONL file:
    throughput, roofline fractions, the FP32 form's per-quantity error,
    latency percentiles, branch-hit counts and the host core count, each with
    the run's time stamp."""
    import time
    stamp = time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime())
    recs = [{"section": "gcm_fp32_form", "value": line["value"], "unit": line["unit"],
             "ms_per_step": line["ms_per_step"], "roofline_frac": line["roofline"]["frac"],
             "hbm_frac": line["roofline"]["hbm"]["frac"], "mufu_frac": line["roofline"]["mufu"]["frac"],
             "clocks": line.get("clocks")},
            {"section": "fp64_plain", **line["fp64_plain"]},
            {"section": "e2e", **line["e2e"]},
            {"section": "branch_counts", **line["branch_counts"]},
            {"section": "host", "cores": cpu_cores()}]
    for key in ("fp32_error_vs_fp64", "sweeps", "uneven", "postproc", "ktable", "serving", "cpu_baseline"):
        if key in line:
            recs.append({"section": key, **line[key]})
    with open(path, "a") as f:
        for r in recs:
            f.write(json.dumps({"time": stamp, **r}) + "\n")


if __name__ == "__main__":
    sys.exit(main())
