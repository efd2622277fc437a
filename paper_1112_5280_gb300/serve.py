"""Serving loop: a stream of solve requests, continuous batching on the Krylov engine.

Requests (lattice, gauge field, kappa, source, tolerance) arrive over time. Gauge
fields stay resident on the device. A request is admitted as soon as the engine
has a free slot and enough of its HBM budget (lqcd_engine_submit returns EBUSY
otherwise and the request waits); all admitted requests advance together in the
same batched launches (one CUDA-graph replay of `chunk` iterations per step),
finished ones are retired between replays and the freed slot and memory go to
the next waiting request. Latency is measured from arrival to the host seeing
the finished result.

The scheduler only needs an engine with submit / step / completed / result /
cancel (the native lqcd.Engine, or a stand-in for host-side tests).
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, Sequence

import numpy as np

LATTICES = ((8, 8, 8, 8), (16, 16, 16, 32), (24, 24, 24, 48), (32, 32, 32, 64))
WEIGHTS = (0.4, 0.3, 0.2, 0.1)
KAPPA_RANGE = (0.12, 0.155)


@dataclasses.dataclass
class Request:
    rid: int                 # caller's id
    arrival: float           # seconds after the stream starts
    lattice: int             # index into the lattice list
    gauge: int               # index into that lattice's resident gauge pool
    source: int              # index into that lattice's source pool
    kappa: float
    tol: float = 1e-10
    deadline: float | None = None  # seconds after arrival; None = no deadline


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    status: int
    iters: int
    true_resid: float
    lattice: int = -1

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def poisson_stream(n: int, rate: float, seed: int = 4004, lattices=LATTICES, weights=WEIGHTS,
                   gauge_pool: int = 4, source_pool: int = 4, kappa_range=KAPPA_RANGE,
                   tol: float = 1e-10) -> list[Request]:
    """n requests with exponential inter-arrival times (mean 1/rate), seeded."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n)) if rate > 0 else np.zeros(n)
    lat = rng.choice(len(lattices), size=n, p=np.asarray(weights) / np.sum(weights))
    kap = rng.uniform(kappa_range[0], kappa_range[1], size=n)
    gi = rng.integers(0, gauge_pool, size=n)
    si = rng.integers(0, source_pool, size=n)
    return [Request(i, float(t[i]), int(lat[i]), int(gi[i]), int(si[i]), float(kap[i]), tol)
            for i in range(n)]


def shard(requests: Sequence[Request], rank: int, world: int) -> list[Request]:
    """Requests handled by one of `world` independent replicas (round robin)."""
    return [r for i, r in enumerate(requests) if i % world == rank]


def percentile(values, q):
    if len(values) == 0:
        return None
    return float(np.percentile(np.asarray(values, dtype=np.float64), q))


def summarize(results: Sequence[Result], wall: float) -> dict:
    lat = [r.latency for r in results]
    ok = [r for r in results if r.status == 0]
    return {
        "requests": len(results),
        "converged": len(ok),
        "solves_per_s": len(ok) / wall if wall > 0 else None,
        "p50_ms": None if not lat else 1e3 * percentile(lat, 50),
        "p99_ms": None if not lat else 1e3 * percentile(lat, 99),
        "mean_ms": None if not lat else 1e3 * float(np.mean(lat)),
        "max_resid": max((r.true_resid for r in ok), default=None),
        "wall_s": wall,
        "by_lattice": by_lattice(results),
    }


def by_lattice(results: Sequence[Result], lattices=LATTICES) -> dict:
    """Request count, p50 and p99 latency per lattice size ("LxLyLzLt")."""
    out = {}
    for li in sorted({r.lattice for r in results if r.lattice >= 0}):
        lat = [r.latency for r in results if r.lattice == li]
        name = "x".join(map(str, lattices[li])) if li < len(lattices) else str(li)
        out[name] = {"n": len(lat), "p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99)}
    return out


class Scheduler:
    """Continuous batching of a request stream on one engine.

    submit_fn(req) -> engine id or None (busy); the engine advances with step();
    completed() lists finished engine ids; collect(eid) -> (status, iters, resid)
    releases the slot. clock() is wall time in seconds.
    """

    def __init__(self, engine, submit_fn: Callable, collect_fn: Callable,
                 clock: Callable[[], float] = time.perf_counter):
        self.engine = engine
        self.submit_fn = submit_fn
        self.collect_fn = collect_fn
        self.clock = clock
        self.max_active = 0

    def run(self, requests: Sequence[Request], realtime: bool = True) -> tuple[list[Result], float]:
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting: list[Request] = []
        active: dict[int, tuple[Request, float]] = {}
        results: list[Result] = []
        cancelled: set = set()
        t0 = self.clock()
        i = 0
        while i < len(pending) or waiting or active:
            now = self.clock() - t0
            while i < len(pending) and (not realtime or pending[i].arrival <= now):
                waiting.append(pending[i])
                i += 1
            # deadlines of waiting requests
            still = []
            for r in waiting:
                if r.deadline is not None and now - r.arrival > r.deadline:
                    results.append(Result(r.rid, r.arrival, now, now, -6, 0, float("nan"), r.lattice))
                else:
                    still.append(r)
            waiting = still
            # admit in arrival order while the engine has room
            while waiting:
                eid = self.submit_fn(waiting[0])
                if eid is None:
                    break
                active[eid] = (waiting.pop(0), now)
            self.max_active = max(self.max_active, len(active))
            # deadlines of running requests
            for eid, (r, adm) in list(active.items()):
                if r.deadline is not None and now - r.arrival > r.deadline and eid not in cancelled:
                    self.engine.cancel(eid)
                    cancelled.add(eid)
            if active:
                self.engine.step()
                now = self.clock() - t0
                for eid in self.engine.completed():
                    r, adm = active.pop(eid)
                    status, iters, resid = self.collect_fn(eid)
                    results.append(Result(r.rid, r.arrival, adm, now, status, iters, resid, r.lattice))
            elif i < len(pending):
                # idle until the next arrival
                if realtime:
                    wait = pending[i].arrival - (self.clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.01))
        wall = self.clock() - t0
        return results, wall


class GpuServer:
    """Resident gauge and source pools on one device, and an engine that serves requests."""

    def __init__(self, ctx, lattices, gauge_pools, source_pools, opts=None, hbm_budget=0,
                 max_slots=64):
        from . import lqcd
        self.lqcd = lqcd
        self.ctx = ctx
        self.lattices = [tuple(d) for d in lattices]
        self.gauges = [[ctx.gauge(d, U, prec="f64") for U in pool]
                       for d, pool in zip(self.lattices, gauge_pools)]
        self.sources = [[ctx.field(d, "f64", lqcd.FULL, data=b) for b in pool]
                        for d, pool in zip(self.lattices, source_pools)]
        self.xout = [ctx.field(d, "f64", lqcd.FULL) for d in self.lattices]
        self.engine = lqcd.Engine(ctx, opts, hbm_budget=hbm_budget, max_slots=max_slots)
        self.lat_of = {}

    def submit(self, r: Request):
        eid = self.engine.submit(self.gauges[r.lattice][r.gauge], self.sources[r.lattice][r.source],
                                 r.kappa, r.tol)
        if eid is not None:
            self.lat_of[eid] = r.lattice
        return eid

    def collect(self, eid):
        lat = self.lat_of.pop(eid)
        try:
            info = self.engine.result(eid, self.xout[lat])
            return info["status"], info["iters"], info["true_resid"]
        except self.lqcd.LqcdError as e:
            return e.code, 0, float("nan")

    def scheduler(self):
        return Scheduler(self.engine, self.submit, self.collect)

    def close(self):
        self.engine.close()
