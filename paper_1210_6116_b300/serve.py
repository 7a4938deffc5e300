"""Continuous-batching server for helicity-modulus PCC runs.

Each request is one PCC run (the paper's self-adapting search for the KT
point, Sec. 2): an L x L lattice that starts at beta0 and after every sweep
steps beta up or down by dbeta depending on beta*Upsilon against the target.
Requests arrive over time; the server admits an arrived request as soon as a
slot is free and its workspace fits the HBM budget, runs all admitted
requests together in an Engine (one launch per kernel per sweep for all of
them), and retires each request when its sweep budget is spent, returning its
observable series.  Requests therefore join and leave between chunks of
sweeps while the others keep running ("continuous batching").

Latency is measured from a request's arrival to the moment its result is on
the host.  `run_loop` serves the same trace the plain way -- one request at a
time, in arrival order, each on its own lattice -- for comparison.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

import paper_1210_6116_b300 as xy


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the start of the trace
    L: int
    budget: int     # sweeps
    seed: int
    beta0: float = 1.0


@dataclass
class PCC:
    target: float = 2.0 / math.pi
    dbeta0: float = 0.01
    halve_every: int = 500
    block: int = 1

    def params(self) -> xy.xy_pcc_params:
        return xy.xy_pcc_params(target=self.target, dbeta0=self.dbeta0,
                                halve_every=self.halve_every, block=self.block)


@dataclass
class Result:
    rid: int
    L: int
    budget: int
    arrival: float
    admitted: float
    finished: float
    records: np.ndarray
    final_beta: float
    cancelled: bool = False

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    wall: float = 0.0
    rejected: list = field(default_factory=list)
    peak_bytes: int = 0

    def summary(self) -> dict:
        lat = np.array([r.latency for r in self.results])
        sweeps = sum(r.budget for r in self.results)
        updates = sum(r.budget * r.L * r.L for r in self.results)
        buckets = {}
        for lo, hi in ((500, 1000), (1000, 2000), (2000, 3000), (3000, 4000), (4000, 5001)):
            sel = np.array([lo <= r.budget < hi for r in self.results])
            if sel.any():
                buckets[f"[{lo},{min(hi, 5000)}]"] = {
                    "n": int(sel.sum()), "p50_s": round(float(np.percentile(lat[sel], 50)), 4),
                    "p99_s": round(float(np.percentile(lat[sel], 99)), 4)}
        return {"requests": len(self.results), "wall_s": round(self.wall, 3),
                "p50_latency_s": round(float(np.percentile(lat, 50)), 4) if len(lat) else None,
                "p99_latency_s": round(float(np.percentile(lat, 99)), 4) if len(lat) else None,
                "sweeps_per_s": round(sweeps / self.wall, 1),
                "updates_per_ns": round(updates / (self.wall * 1e9), 3),
                "by_budget": buckets, "rejected": len(self.rejected)}


class Server:
    """Admission by free slots and HBM footprint, continuous batching.

    policy "fifo" admits arrived requests in arrival order; "small-first"
    admits the arrived request with the least work (L^2 x budget) first and
    stops admitting once the active lattices' tiles reach tile_cap (about what
    keeps every SM busy), so short requests are not held behind long ones
    while the GPU stays full."""

    def __init__(self, max_slots: int = 64, hbm_budget: int | None = None, *,
                 dtype: str = "f32", exact: bool = False, tile_y: int = 64,
                 chunk: int = 100, pcc: PCC | None = None, policy: str = "small-first",
                 tile_cap: int = 16384):
        import torch

        self.engine = xy.Engine(max_slots, dtype=dtype, exact=exact, tile_y=tile_y)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info()
            hbm_budget = int(0.8 * free)
        self.hbm_budget = hbm_budget
        self.max_slots = max_slots
        self.chunk = chunk
        self.pcc = pcc or PCC()
        if policy not in ("fifo", "small-first"):
            raise ValueError("policy must be 'fifo' or 'small-first'")
        self.policy = policy
        self.tile_cap = tile_cap
        self.tile_y = tile_y

    def tiles(self, req: Request) -> int:
        return ((req.L + 31) // 32) * ((req.L + self.tile_y - 1) // self.tile_y)

    def footprint(self, req: Request) -> int:
        return self.engine.footprint(self._cfg(req))

    def _cfg(self, req: Request):
        return self.engine.config(req.L, req.beta0, req.seed, record_cap=max(req.budget, 1))

    def run(self, trace: list[Request], realtime: bool = True,
            should_cancel=None) -> ServeStats:
        """Serve a trace.  realtime=True honours the arrival times (the server
        idles until the next arrival); False admits requests as if they had
        all arrived already.  should_cancel(request, sweeps_done) is asked
        after every chunk; True retires the request at once (its partial
        series is returned with cancelled=True) and frees its slot and
        memory for waiting requests."""
        pending = deque(sorted(trace, key=lambda r: r.arrival))
        arrived = []  # arrived, not yet admitted
        active = {}  # slot -> (req, remaining, footprint, admitted_at)
        used = 0
        tiles = 0
        stats = ServeStats()
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: math.inf)
        while pending or arrived or active:
            now = clock()
            while pending and pending[0].arrival <= now:
                arrived.append(pending.popleft())
            if self.policy == "small-first":
                arrived.sort(key=lambda r: r.L * r.L * r.budget)
            while arrived and len(active) < self.max_slots:
                req = arrived[0]
                fp = self.footprint(req)
                if fp > self.hbm_budget:
                    stats.rejected.append(arrived.pop(0))  # can never fit
                    continue
                if used + fp > self.hbm_budget:
                    break  # wait for memory to free up
                if active and tiles >= self.tile_cap:
                    break  # the GPU is full
                arrived.pop(0)
                slot = self.engine.admit(self._cfg(req), self.pcc.params())
                active[slot] = (req, req.budget, fp, time.perf_counter() - t0)
                used += fp
                tiles += self.tiles(req)
                stats.peak_bytes = max(stats.peak_bytes, used)
            if not active:
                if pending and realtime:
                    time.sleep(max(0.0, min(pending[0].arrival - clock(), 0.01)))
                continue
            n = min(self.chunk, min(rem for _, rem, _, _ in active.values()))
            self.engine.step(n)
            done = []
            for slot, (req, rem, fp, adm) in list(active.items()):
                rem -= n
                active[slot] = (req, rem, fp, adm)
                if rem == 0:
                    done.append((slot, False))
                elif should_cancel is not None and should_cancel(req, req.budget - rem):
                    done.append((slot, True))
            for slot, cancelled in done:
                req, _, fp, adm = active.pop(slot)
                recs = self.engine.measure(slot)  # synchronises
                beta, _ = self.engine.state(slot)
                stats.results.append(Result(req.rid, req.L, req.budget, req.arrival, adm,
                                            time.perf_counter() - t0, recs, beta, cancelled))
                self.engine.retire(slot)
                used -= fp
                tiles -= self.tiles(req)
        stats.wall = time.perf_counter() - t0
        return stats

    def close(self):
        self.engine.close()


def run_loop(trace: list[Request], pcc: PCC | None = None, *, dtype: str = "f32",
             exact: bool = False, realtime: bool = True) -> ServeStats:
    """The plain per-request loop: one lattice at a time, in arrival order."""
    pcc = pcc or PCC()
    stats = ServeStats()
    t0 = time.perf_counter()
    for req in sorted(trace, key=lambda r: r.arrival):
        if realtime:
            wait = req.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        adm = time.perf_counter() - t0
        lat = xy.Lattice(req.L, req.beta0, req.seed, dtype=dtype, exact=exact,
                         tile_y=32 if req.L <= 256 else 64, record_cap=max(req.budget, 1))
        lat.pcc_step(req.budget, target=pcc.target, dbeta0=pcc.dbeta0,
                     halve_every=pcc.halve_every, block=pcc.block)
        recs = lat.measure()
        beta, _ = lat.state()
        stats.results.append(Result(req.rid, req.L, req.budget, req.arrival, adm,
                                    time.perf_counter() - t0, recs, beta))
        lat.close()
    stats.wall = time.perf_counter() - t0
    return stats
