"""Serving loop on the GPU: continuous batching of a request stream on the engine.

Every result converges (oracle-measured residual) and equals the same request
solved alone, bit for bit, whatever else shared its launches; a small HBM
budget limits how many requests run at once.
"""
import numpy as np
import pytest

import oracle
from paper_1112_5280_gb300 import lqcd, serve, synth

pytestmark = pytest.mark.gpu

LATS = [(4, 4, 4, 4), (6, 4, 4, 6), (8, 4, 4, 4)]


@pytest.fixture(scope="module")
def server():
    ctx = lqcd.Context(0)
    gauges = [[synth.random_links(d, 0.5, seed=900 + 10 * i + k) for k in range(2)]
              for i, d in enumerate(LATS)]
    sources = [[synth.gaussian_spinor(d, seed=950 + 10 * i + k) for k in range(2)]
               for i, d in enumerate(LATS)]
    opts = lqcd.solve_opts(sloppy_prec="f16", chunk=8)
    probe = lqcd.Engine(ctx, opts)
    budget = 2 * max(probe.request_bytes(d) for d in LATS) + 1
    probe.close()
    srv = serve.GpuServer(ctx, LATS, gauges, sources, opts=opts, hbm_budget=budget, max_slots=4)
    srv.budget = budget
    yield srv, gauges, sources, opts
    srv.close()


def _run(srv, reqs, realtime):
    xs = {}

    def collect(eid):
        r = srv.lat_of[eid]
        out = srv.collect(eid)
        xs[eid] = (r, srv.xout[r].download())
        return out
    eids = {}

    def submit(r):
        eid = srv.submit(r)
        if eid is not None:
            eids[eid] = r
            assert srv.engine.stats()[1] <= srv.budget  # admission keeps the device bytes in budget
        return eid
    sch = serve.Scheduler(srv.engine, submit, collect)
    res, wall = sch.run(reqs, realtime=realtime)
    by_rid = {eids[e].rid: (eids[e], x) for e, (_, x) in xs.items()}
    return res, wall, sch.max_active, by_rid


def test_stream_all_at_once(server):
    srv, gauges, sources, opts = server
    reqs = serve.poisson_stream(14, rate=0, seed=4004, lattices=LATS, weights=(1, 1, 1),
                                gauge_pool=2, source_pool=2)
    res, wall, max_active, by_rid = _run(srv, reqs, realtime=False)
    assert len(res) == 14 and all(r.status == 0 for r in res)
    assert 1 < max_active < 4  # requests overlap, and the budget (not the 4 slots) limits them
    for rid, (r, x) in by_rid.items():
        d = LATS[r.lattice]
        U = gauges[r.lattice][r.gauge]
        b = sources[r.lattice][r.source]
        assert oracle.true_residual(d, U, r.kappa, b, x) <= 1e-10
    # the same request alone gives the same bits
    for rid in (0, 5, 9):
        r, x = by_rid[rid]
        g = srv.gauges[r.lattice][r.gauge]
        xs = srv.ctx.field(LATS[r.lattice], "f64", lqcd.FULL)
        lqcd.solve_fields(g, srv.sources[r.lattice][r.source], r.kappa, r.tol, xs, opts)
        assert np.array_equal(xs.download(), x)


def test_stream_realtime_poisson(server):
    srv, *_ = server
    reqs = serve.poisson_stream(10, rate=400.0, seed=7, lattices=LATS, weights=(1, 1, 1),
                                gauge_pool=2, source_pool=2)
    res, wall, _, _ = _run(srv, reqs, realtime=True)
    s = serve.summarize(res, wall)
    assert s["converged"] == 10 and s["p99_ms"] >= s["p50_ms"] > 0
    assert all(r.finished >= r.arrival for r in res)
