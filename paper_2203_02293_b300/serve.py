"""Continuous-batching request loop over the C ABI.

Requests (columns x layers x bins of the same shape within a request) arrive
at given times.  Their inputs are slices of a device-resident pool: the
batch descriptor points into the pool through per-column gather offsets, so
no input is copied per request.  The server keeps a ring of slots (a CUDA
stream and a library handle each).  Whenever a slot is free and requests are
waiting, it admits waiting requests (in arrival order, or smallest first with
``policy="sjf"``) while the bytes of the batches in flight stay within the HBM
budget, and launches them as one solve on that slot's stream; batches on
different slots overlap on the device.  A
request's latency runs from its arrival to the host seeing its batch's
completion event.  Requests that can never fit the budget are refused; a
request may be cancelled while it waits or refused after a waiting timeout.
A batch whose launch the library refuses (its workspace could not be
allocated: RT_ENOMEM, or RT_EBUDGET) fails its requests; the slot and its
handle go on serving.

With ``split_systems`` set, a request larger than that many systems is cut
into pieces of whole columns when it arrives; the pieces wait, are admitted
and run like requests of their own (on several slots at once when free),
and the request completes when its last piece does.  A large request then
neither holds one slot for its whole duration nor delays the small requests
queued behind it, and its results are the same bits as unsplit (columns are
independent and each column's sums run in a fixed order).
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import rt
from .solver import Solver


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    n_cols: int
    L: int
    NB: int
    cols: np.ndarray               # pool column indices (for the per-column inputs)
    cube_base: int                 # element offset of the request's cube block in the pool
    n_g: int = 20
    status: str = "new"            # new, waiting, running, done, refused, cancelled, timeout
    nbytes: int = 0                # workspace of the request alone (upper bound per request)
    t_admit: float = -1.0
    t_done: float = -1.0
    outputs: dict | None = None
    parent: "Request | None" = None   # for a piece: the request it belongs to
    pieces: list | None = None         # for a split request: its pieces, in column order
    pieces_left: int = 0

    @property
    def systems(self) -> int:
        return self.n_cols * self.NB * self.n_g

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


class Pool:
    """Device-resident inputs that requests slice.

    Cubes are flat arrays of independent draws, so any contiguous block of the
    right length is a valid request cube.  Per-column profiles are stored for
    every layer count L in [L_min, L_max] (n_pool columns each), F* for every
    bin count in [NB_min, NB_max]."""

    def __init__(self, draw, n_pool: int, L_range, NB_range, n_g: int = 20, cube_elems: int = 0,
                 device="cuda"):
        # ``draw`` is an rt_synth-like module providing the generators
        self.n_g = n_g
        self.L_range, self.NB_range = L_range, NB_range
        self.n_pool = n_pool
        Ls = range(L_range[0], L_range[1] + 1)
        NBs = range(NB_range[0], NB_range[1] + 1)
        rng = np.random.default_rng(12345)
        tc, ti, pi = [], [], []
        self.tc_off, self.if_off = {}, {}
        ntc = nif = 0
        for L in Ls:
            self.tc_off[L], self.if_off[L] = ntc, nif
            for _ in range(n_pool):
                p, Tc, Ti = draw.column_profile(rng, L)
                tc.append(Tc); ti.append(Ti); pi.append(p)
            ntc += n_pool * L
            nif += n_pool * (L + 1)
        fs = []
        self.fs_off = {}
        nfs = 0
        for NB in NBs:
            self.fs_off[NB] = nfs
            fs.append(draw.stellar_flux_bins(NB))
            nfs += NB
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(np.concatenate(a), dtype=np.float64)).to(device)
        self.T_center, self.T_iface, self.p_iface = dev(tc), dev(ti), dev(pi)
        self.F_star = dev(fs)
        self.mu_star = torch.from_numpy(rng.uniform(0.1, 1.0, n_pool)).to(device)
        if cube_elems <= 0:
            cube_elems = n_pool * L_range[1] * NB_range[1] * n_g
        gen = torch.Generator(device=device)
        gen.manual_seed(777)
        self.dtau = draw.device_uniform(cube_elems, 1e-6, 10.0, gen, device, log=True)
        self.w0 = draw.device_uniform(cube_elems, 0.0, 0.95, gen, device)
        self.g0 = draw.device_uniform(cube_elems, 0.0, 0.8, gen, device)
        self.cube_elems = cube_elems
        _, self.g_weights = draw.gauss_legendre_01(n_g)

    KEYS = ("cube_offset", "center_offset", "iface_offset", "bin_offset", "col_index")

    def _request_gather(self, r):
        """Shapes and gather offsets of one request's columns (array
        arithmetic, computed once per request)."""
        g = getattr(r, "_gather", None)
        if g is None:
            n = r.n_cols
            cols = np.asarray(r.cols, np.int64)
            per = r.L * r.NB * self.n_g
            g = (np.full(n, r.L, np.int32), np.full(n, r.NB, np.int32),
                 dict(cube_offset=r.cube_base + per * np.arange(n, dtype=np.int64),
                      center_offset=self.tc_off[r.L] + cols * r.L,
                      iface_offset=self.if_off[r.L] + cols * (r.L + 1),
                      bin_offset=np.full(n, self.fs_off[r.NB], np.int64),
                      col_index=cols))
            r._gather = g
        return g

    def gather(self, reqs):
        """Shapes and gather offsets of a batch made of ``reqs`` (in order)."""
        parts = [self._request_gather(r) for r in reqs]
        if len(parts) == 1:
            return parts[0]
        nl = np.concatenate([p[0] for p in parts])
        nb = np.concatenate([p[1] for p in parts])
        g = {k: np.concatenate([p[2][k] for p in parts]) for k in self.KEYS}
        return nl, nb, g

    def descriptor(self, reqs):
        nl, nb, g = self.gather(reqs)
        return rt.make_columns(len(nl), nl, nb, self.dtau, self.w0, self.g0, self.T_center,
                               self.T_iface, self.p_iface, self.mu_star, self.F_star, gather=g), nl


def make_requests(pool: Pool, n: int, rate_hz: float, seed: int, C_range=(1, 2562)):
    """Poisson arrivals; C ~ logU[C_range], L and NB uniform over the pool's ranges."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    reqs = []
    for i in range(n):
        C = int(np.clip(np.round(np.exp(rng.uniform(np.log(C_range[0]), np.log(C_range[1] + 0.5)))),
                        C_range[0], min(C_range[1], pool.n_pool)))
        L = int(rng.integers(pool.L_range[0], pool.L_range[1] + 1))
        NB = int(rng.integers(pool.NB_range[0], pool.NB_range[1] + 1))
        cols = rng.choice(pool.n_pool, C, replace=False)
        need = C * L * NB * pool.n_g
        base = int(rng.integers(0, pool.cube_elems - need + 1))
        reqs.append(Request(i, float(t[i]), C, L, NB, cols, base, n_g=pool.n_g))
    return reqs


def split_request(r: Request, max_systems: int) -> list:
    """``r`` as pieces of whole columns of at most ``max_systems`` systems
    each (at least one column per piece); ``[r]`` if it is small enough."""
    per_col = r.NB * r.n_g
    if max_systems <= 0 or r.systems <= max_systems or r.n_cols == 1:
        return [r]
    k = max(1, max_systems // per_col)
    pieces = []
    for j0 in range(0, r.n_cols, k):
        cols = r.cols[j0:j0 + k]
        pieces.append(Request(r.rid, r.arrival, len(cols), r.L, r.NB, cols,
                              r.cube_base + j0 * r.L * per_col, n_g=r.n_g, parent=r))
    r.pieces = pieces
    r.pieces_left = len(pieces)
    return pieces


@dataclass
class Slot:
    stream: torch.cuda.Stream
    solver: Solver
    event: torch.cuda.Event = field(default_factory=torch.cuda.Event)
    reqs: list = field(default_factory=list)
    nbytes: int = 0
    n_if: int = 0
    busy: bool = False
    wide: Solver | None = None     # a handle with every CTA resident, for large batches
    active: Solver | None = None   # the handle of the batch in flight


class Server:
    def __init__(self, pool: Pool, n_slots: int = 4, hbm_budget_bytes: int = 8 << 30,
                 max_systems_per_batch: int = 24_000_000, wait_timeout_s: float = 0.0,
                 keep_outputs: bool = False, policy: str = "fifo", split_systems: int = 0,
                 wide_layer_systems: int = 0, **cfg):
        # wide_layer_systems > 0: a batch of at least that many layer-systems
        # (systems x layers) runs on a second handle of the slot that keeps
        # every CTA resident, so a large request alone on the GPU gets all of
        # it; smaller batches keep the slot's own launch shape
        # policy: "fifo" admits in arrival order; "sjf" admits the smallest
        # waiting requests first (shorter latency for small requests);
        # "gang" is sjf with the pieces of started split requests first
        self.policy = policy
        self.split = split_systems
        self.pool = pool
        self.budget = hbm_budget_bytes
        self.max_sys = max_systems_per_batch
        self.wait_timeout = wait_timeout_s
        self.keep_outputs = keep_outputs
        self.wide_at = wide_layer_systems
        wide_cfg = {k: v for k, v in cfg.items() if k != "ctas_per_sm"}
        self.slots = [Slot(torch.cuda.Stream(), Solver(pool.g_weights, **cfg),
                           wide=Solver(pool.g_weights, **wide_cfg) if wide_layer_systems > 0 else None)
                      for _ in range(n_slots)]
        self.in_flight_bytes = 0
        self.batches = 0
        self.failures: list[str] = []    # messages of launches the library refused

    def close(self):
        for s in self.slots:
            s.solver.close()
            if s.wide is not None:
                s.wide.close()

    def _bytes(self, slot: Slot, r: Request) -> int:
        # workspace of the request alone (a first estimate for composing a batch)
        if not r.nbytes:
            desc, _ = self.pool.descriptor([r])
            r.nbytes = rt.rt_query_bytes(slot.solver.h, desc)
        return r.nbytes

    def _complete(self, slot: Slot, now: float) -> int:
        """Retire a finished batch; returns how many requests it completed."""
        if self.keep_outputs:
            o = slot.active.outputs_host(slot.n_if, sum(r.n_cols * r.L for r in slot.reqs))
            i0 = l0 = 0
            for r in slot.reqs:
                ni, nl = r.n_cols * (r.L + 1), r.n_cols * r.L
                r.outputs = {"F_up": o["F_up"][i0:i0 + ni], "F_down": o["F_down"][i0:i0 + ni],
                             "F_net": o["F_net"][i0:i0 + ni], "Q": o["Q"][l0:l0 + nl]}
                i0 += ni
                l0 += nl
        finished = 0
        for r in slot.reqs:
            r.t_done = now
            r.status = "done"
            p = r.parent
            if p is None:
                finished += 1
            elif p.status in ("waiting", "running"):
                p.pieces_left -= 1
                if p.pieces_left == 0:
                    p.t_done, p.status = now, "done"
                    if self.keep_outputs:
                        p.outputs = {k: np.concatenate([q.outputs[k] for q in p.pieces]) for k in r.outputs}
                    finished += 1
        self.in_flight_bytes -= slot.nbytes
        slot.reqs, slot.busy, slot.nbytes = [], False, 0
        return finished

    @staticmethod
    def _end(r: Request, status: str, now: float) -> int:
        """End a waiting request or piece; returns 1 when that ends a request
        (a split request ends with its first piece to be refused, cancelled,
        timed out or failed; its other pieces are then dropped)."""
        r.status, r.t_done = status, now
        p = r.parent
        if p is None:
            return 1
        if p.status in ("waiting", "running"):
            p.status, p.t_done = status, now
            return 1
        return 0

    def run(self, requests, cancel: set | None = None, poll_sleep: float = 5e-5):
        """Serve ``requests`` (sorted by arrival); returns a summary dict."""
        cancel = cancel or set()
        arrivals = deque(sorted(requests, key=lambda r: r.arrival))
        waiting: deque = deque()
        t0 = time.perf_counter()
        done = 0
        total = len(arrivals)
        while done < total:
            now = time.perf_counter() - t0
            while arrivals and arrivals[0].arrival <= now:
                r = arrivals.popleft()
                r.status = "waiting"
                for piece in split_request(r, self.split):
                    piece.status = "waiting"
                    waiting.append(piece)
            # completions
            for s in self.slots:
                if s.busy and s.event.query():
                    done += self._complete(s, time.perf_counter() - t0)
            # cancellations, timeouts, and pieces of requests that have ended
            keep = deque()
            for r in waiting:
                if r.parent is not None and r.parent.status not in ("waiting", "running"):
                    r.status = "dropped"
                elif r.rid in cancel:
                    done += self._end(r, "cancelled", now)
                elif self.wait_timeout and now - r.arrival > self.wait_timeout:
                    done += self._end(r, "timeout", now)
                else:
                    keep.append(r)
            waiting = keep
            if self.policy in ("sjf", "gang") and len(waiting) > 1:
                # "gang": the remaining pieces of a request that has started
                # go first, so a split request's pieces run together
                started = lambda r: 0 if (self.policy == "gang" and r.parent is not None
                                          and r.parent.status == "running") else 1
                waiting = deque(sorted(waiting, key=lambda r: (started(r), r.systems * r.L)))
            # admission into free slots
            for s in self.slots:
                if s.busy or not waiting:
                    continue
                batch, nsys, need = [], 0, 0
                while waiting:
                    r = waiting[0]
                    if batch and nsys + r.systems > self.max_sys:
                        break
                    if r.parent is not None and r.parent.status not in ("waiting", "running"):
                        waiting.popleft()              # its request has ended
                        r.status = "dropped"
                        continue
                    rb = self._bytes(s, r)
                    if rb > self.budget:
                        waiting.popleft()              # can never fit
                        done += self._end(r, "refused", now)
                        continue
                    if self.in_flight_bytes + need + rb > self.budget:
                        break
                    batch.append(waiting.popleft())
                    nsys += r.systems
                    need += rb
                if not batch:
                    continue
                # the handle for this batch, then its exact need; hand requests
                # back until it fits
                pick = lambda b: s.wide if (s.wide is not None and
                                            sum(r.systems * r.L for r in b) >= self.wide_at) else s.solver
                desc, nl = self.pool.descriptor(batch)
                need = rt.rt_query_bytes(pick(batch).h, desc)
                while len(batch) > 1 and self.in_flight_bytes + need > self.budget:
                    waiting.appendleft(batch.pop())
                    desc, nl = self.pool.descriptor(batch)
                    need = rt.rt_query_bytes(pick(batch).h, desc)
                if self.in_flight_bytes + need > self.budget:
                    waiting.appendleft(batch.pop())
                    continue
                torch.cuda.nvtx.range_push(f"serve batch {self.batches}: {len(batch)} requests")
                s.active = pick(batch)
                try:
                    rt.rt_solve_columns(s.active.h, desc, s.stream)
                except rt.RTError as e:
                    # the launch was refused (e.g. its workspace could not be
                    # allocated): its requests fail, the slot stays free and
                    # the handle serves the next batch
                    torch.cuda.nvtx.range_pop()
                    if e.code not in (rt.RT_ENOMEM, rt.RT_EBUDGET):
                        raise
                    for r in batch:
                        done += self._end(r, "failed", now)
                    self.failures.append(str(e))
                    continue
                s.event.record(s.stream)
                torch.cuda.nvtx.range_pop()
                t_admit = time.perf_counter() - t0
                for r in batch:
                    r.status, r.t_admit = "running", t_admit
                    if r.parent is not None and r.parent.status == "waiting":
                        r.parent.status, r.parent.t_admit = "running", t_admit
                s.reqs, s.busy, s.nbytes = batch, True, need
                s.n_if = int((nl + 1).sum())
                self.in_flight_bytes += need
                self.batches += 1
            if not any(s.busy for s in self.slots) and not waiting and arrivals:
                gap = arrivals[0].arrival - (time.perf_counter() - t0)
                if gap > 0:
                    time.sleep(min(gap, 1e-3))
            else:
                time.sleep(poll_sleep)
        return summarize(requests, time.perf_counter() - t0, self.batches)


def summarize(requests, wall: float, batches: int) -> dict:
    ok = [r for r in requests if r.status == "done"]
    lat = np.array([r.latency for r in ok]) * 1e3
    sys_done = sum(r.systems for r in ok)
    span = (max(r.t_done for r in ok) - min(r.arrival for r in ok)) if ok else 0.0
    return {
        "requests": len(requests), "done": len(ok),
        "refused": sum(r.status == "refused" for r in requests),
        "cancelled": sum(r.status == "cancelled" for r in requests),
        "timeout": sum(r.status == "timeout" for r in requests),
        "failed": sum(r.status == "failed" for r in requests),
        "batches": batches,
        "p50_ms": float(np.percentile(lat, 50)) if ok else None,
        "p99_ms": float(np.percentile(lat, 99)) if ok else None,
        "mean_ms": float(lat.mean()) if ok else None,
        "solves_per_s": sys_done / span if span > 0 else None,
        "wall_s": wall,
    }
