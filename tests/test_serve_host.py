"""Host-side logic of the serving loop and the multi-replica path (CPU only).

The scheduler is driven by a stand-in engine with a fixed number of slots and a
memory budget; the N > 1 replica path (request sharding, max-over-ranks timing)
runs as two gloo ranks.
"""
import os

import numpy as np
import pytest

from paper_1112_5280_gb300 import serve


class FakeEngine:
    """Slots and a byte budget; a request needs `cost` steps; step() advances all active."""

    def __init__(self, slots, budget, cost_of, bytes_of):
        self.slots, self.budget = slots, budget
        self.cost_of, self.bytes_of = cost_of, bytes_of
        self.active, self.done, self.used, self.next = {}, [], 0, 1
        self.steps = 0
        self.max_active = 0

    def submit(self, req):
        need = self.bytes_of(req)
        if need > self.budget:
            raise RuntimeError("never fits")
        if len(self.active) >= self.slots or self.used + need > self.budget:
            return None
        eid = self.next
        self.next += 1
        self.active[eid] = [req, self.cost_of(req), need, 0]
        self.used += need
        self.max_active = max(self.max_active, len(self.active))
        return eid

    def step(self):
        self.steps += 1
        for eid, a in list(self.active.items()):
            if a[1] <= 0 and eid in self.done:
                continue
            a[1] -= 1
            if a[1] <= 0 and eid not in self.done:
                self.done.append(eid)

    def completed(self):
        out, self.done = self.done, []
        return out

    def cancel(self, eid):
        if eid in self.active:  # finishes at the next step, like the native engine
            self.active[eid][3] = -6
            self.active[eid][1] = 0

    def collect(self, eid):
        req, _, need, status = self.active.pop(eid)
        self.used -= need
        return status, 10, 1e-11


def _fake(slots=3, budget=10):
    cost = {0: 2, 1: 5, 2: 9, 3: 20}
    size = {0: 1, 1: 2, 2: 4, 3: 8}
    return FakeEngine(slots, budget, lambda r: cost[r.lattice], lambda r: size[r.lattice])


def test_poisson_stream_is_seeded_and_weighted():
    a = serve.poisson_stream(2000, rate=50.0, seed=4004)
    b = serve.poisson_stream(2000, rate=50.0, seed=4004)
    assert [(r.arrival, r.lattice, r.kappa) for r in a] == [(r.arrival, r.lattice, r.kappa) for r in b]
    arr = np.array([r.arrival for r in a])
    assert np.all(np.diff(arr) >= 0)
    assert abs(np.mean(np.diff(arr)) - 1 / 50.0) < 0.1 / 50.0
    frac = np.bincount([r.lattice for r in a], minlength=4) / len(a)
    assert np.allclose(frac, serve.WEIGHTS, atol=0.04)
    k = np.array([r.kappa for r in a])
    assert k.min() >= 0.12 and k.max() <= 0.155


def test_scheduler_continuous_batching_and_budget():
    eng = _fake(slots=3, budget=10)
    reqs = serve.poisson_stream(40, rate=0, seed=1)  # all arrive at t = 0
    sch = serve.Scheduler(eng, eng.submit, eng.collect)
    res, wall = sch.run(reqs, realtime=False)
    assert sorted(r.rid for r in res) == list(range(40))
    assert all(r.status == 0 for r in res)
    assert eng.max_active <= 3 and eng.used == 0
    # continuous batching: slots refill as requests finish, so the step count is far
    # below running the 40 requests one after another
    serial = sum({0: 2, 1: 5, 2: 9, 3: 20}[r.lattice] for r in reqs)
    assert eng.steps < serial
    s = serve.summarize(res, wall)
    assert s["converged"] == 40 and s["p50_ms"] <= s["p99_ms"]


def test_scheduler_never_exceeds_budget():
    eng = _fake(slots=8, budget=9)
    orig = eng.submit

    def checked(r):
        eid = orig(r)
        assert eng.used <= eng.budget
        return eid
    reqs = serve.poisson_stream(30, rate=0, seed=2)
    serve.Scheduler(eng, checked, eng.collect).run(reqs, realtime=False)


def test_deadline_cancels_running_request():
    eng = _fake(slots=1, budget=100)
    t = [0.0]

    def clock():
        t[0] += 0.001
        return t[0]
    r = serve.Request(0, 0.0, 3, 0, 0, 0.13, deadline=0.005)
    res, _ = serve.Scheduler(eng, eng.submit, eng.collect, clock=clock).run([r], realtime=False)
    assert res[0].status == -6


def test_percentiles():
    assert serve.percentile([1, 2, 3, 4], 50) == 2.5
    assert serve.percentile([], 99) is None


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    reqs = serve.poisson_stream(25, rate=10.0, seed=4004)
    mine = serve.shard(reqs, rank, world)
    t = bench.max_over_ranks(float(rank + 1), world)
    bench.barrier(world)
    q.put((rank, [r.rid for r in mine], t))
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids = sorted(i for _, rids, _ in out for i in rids)
    assert ids == list(range(25))
    assert all(t == 2.0 for _, _, t in out)
    per = {r: set(rids) for r, rids, _ in out}
    assert not (per[0] & per[1])
