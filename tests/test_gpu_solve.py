"""GPU solves (CG on Mhat^dag Mhat with FP64 reliable updates, BiCGStab on Mhat) vs the oracle.

Paper Section 3: the inversion of the even-odd preconditioned fermion matrix is
the dominant cost. Bars: every GPU solution has ||b - M x|| <= tol ||b|| with
the full operator, measured by the FP64 oracle on the returned x; and agrees
with the oracle's own solution within C * tol (C = 100 covers the condition
numbers of these workloads, checked against the oracle's iterate).
"""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1112_5280_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = lqcd.Context(0)
    yield c
    c.close()


def _solve_check(ctx, dims, eps, kappa, prec, compress=12, solver=lqcd.CG, tol=1e-10,
                 seed_u=1001, seed_b=2002, xtol=1e-8):
    U = synth.random_links(dims, eps, seed=seed_u)
    b = synth.gaussian_spinor(dims, seed=seed_b)
    g = ctx.gauge(dims, U, prec="f64")
    opts = lqcd.solve_opts(sloppy_prec=prec, sloppy_compress=compress, solver=solver)
    x, info = lqcd.solve(g, b, kappa, tol, opts)
    assert info["status"] == 0, info
    assert info["true_resid"] <= tol, info
    res = oracle.true_residual(dims, U, kappa, b, x)
    assert res <= tol, (res, info)
    xo, st, _, _ = oracle.solve(dims, U, kappa, b, tol=tol * 1e-2, method=oracle.METHOD_CG_EO)
    assert st == 0
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < xtol
    return x, info


def test_cg_fp64_small_workload(ctx):
    """4^4, kappa 0.12, eps 0.3: plain FP64 CG on the GPU."""
    _solve_check(ctx, (4, 4, 4, 4), 0.3, 0.12, "f64", compress=18)


def test_cg_df64(ctx):
    """CG entirely in double-float (storage and arithmetic)."""
    _solve_check(ctx, (6, 4, 4, 6), 0.5, 0.15, "df64", compress=18)


@pytest.mark.parametrize("true_prec", ["f64", "df64"])
def test_mixed_true_residual_precision(ctx, true_prec):
    """The FP64-class outer correction in native FP64 or in double-float reaches the same bar."""
    dims = (6, 4, 4, 6)
    U = synth.random_links(dims, 0.5, seed=1001)
    b = synth.gaussian_spinor(dims, seed=2002)
    g = ctx.gauge(dims, U, prec="f64")
    x, info = lqcd.solve(g, b, 0.15, 1e-10, lqcd.solve_opts(sloppy_prec="f16", true_prec=true_prec))
    assert info["status"] == 0 and oracle.true_residual(dims, U, 0.15, b, x) <= 1e-10


@pytest.mark.parametrize("prec,compress", [("f32", 18), ("f32", 12), ("f16", 12), ("bf16", 12),
                                           ("f16", 18)])
def test_cg_mixed_precision(ctx, prec, compress):
    """Mixed precision with FP64 reliable updates reaches 1e-10 on a ragged lattice."""
    _solve_check(ctx, (6, 4, 4, 6), 0.5, 0.15, prec, compress)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_bicgstab(ctx, prec):
    _solve_check(ctx, (6, 4, 4, 6), 0.5, 0.15, prec, 12, solver=lqcd.BICGSTAB)
    _solve_check(ctx, (4, 4, 4, 4), 0.3, 0.12, prec, 18, solver=lqcd.BICGSTAB)


@pytest.mark.parametrize("solver", [lqcd.CG, lqcd.BICGSTAB])
def test_cached_buffers_reuse_and_release(ctx, solver):
    """One-shot solves keep their buffers on the context: a solve after a larger lattice
    grew them, and a solve after lqcd_ctx_release_cache freed them, equal the first bit for bit."""
    opts = lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=12, solver=solver)
    small, large = (4, 4, 4, 6), (6, 6, 4, 8)
    gs = ctx.gauge(small, synth.random_links(small, 0.4, seed=1011))
    gl = ctx.gauge(large, synth.random_links(large, 0.4, seed=1012))
    bs = synth.gaussian_spinor(small, seed=1013)
    bl = synth.gaussian_spinor(large, seed=1014)
    x0, i0 = lqcd.solve(gs, bs, 0.13, 1e-10, opts)
    assert i0["status"] == 0
    _, il = lqcd.solve(gl, bl, 0.13, 1e-10, opts)
    assert il["status"] == 0
    x1, _ = lqcd.solve(gs, bs, 0.13, 1e-10, opts)
    assert np.array_equal(x0, x1)
    ctx.release_cache()
    ctx.release_cache()  # nothing cached: a no-op
    x2, _ = lqcd.solve(gs, bs, 0.13, 1e-10, opts)
    assert np.array_equal(x0, x2)


def test_free_field_fft(ctx):
    """U = 1 on 8^3 x 16: the GPU solution equals the exact Fourier solution."""
    dims = (8, 8, 8, 16)
    kappa = 0.124
    b = synth.gaussian_spinor(dims, seed=61)
    g = ctx.gauge(dims, synth.unit_links(dims), prec="f64")
    x, info = lqcd.solve(g, b, kappa, 1e-11, lqcd.solve_opts(sloppy_prec="f16"))
    assert info["status"] == 0
    xf = dense.free_solve_fft(dims, kappa, b)
    assert np.linalg.norm(x - xf) / np.linalg.norm(xf) < 1e-9


def test_solve_gauge_covariance(ctx):
    dims = (4, 4, 4, 6)
    U = synth.random_links(dims, 0.5, seed=71)
    gt = synth.gauge_transform_field(dims, seed=72)
    b = synth.gaussian_spinor(dims, seed=73)
    opts = lqcd.solve_opts(sloppy_prec="f32")
    x1, i1 = lqcd.solve(ctx.gauge(dims, U), b, 0.13, 1e-11, opts)
    x2, i2 = lqcd.solve(ctx.gauge(dims, dense.gauge_transform_links(dims, U, gt)),
                        dense.gauge_transform_spinor(gt, b), 0.13, 1e-11, opts)
    ref = dense.gauge_transform_spinor(gt, x1)
    assert i1["status"] == 0 and i2["status"] == 0
    assert np.linalg.norm(x2 - ref) / np.linalg.norm(ref) < 1e-9


def _point_sources(dims, site):
    return [synth.point_source(dims, site, s, c) for s in range(4) for c in range(3)]


def test_multi_rhs_point_sources_match_single(ctx):
    """12 point sources (spin x colour) solved together equal the same solves one by one,
    bit for bit (reductions depend only on each slot's own geometry)."""
    dims = (4, 4, 4, 8)
    U = synth.random_links(dims, 0.5, seed=81)
    site = synth.point_site(dims)
    srcs_h = _point_sources(dims, site)
    g = ctx.gauge(dims, U, prec="f64")
    opts = lqcd.solve_opts(sloppy_prec="f32")
    srcs = [ctx.field(dims, "f64", lqcd.FULL, data=s) for s in srcs_h]
    xs = [ctx.field(dims, "f64", lqcd.FULL) for _ in srcs_h]
    infos = lqcd.solve_multi(g, srcs, 0.15, 1e-10, xs, opts)
    for k, (inf, s, xf) in enumerate(zip(infos, srcs_h, xs)):
        assert inf["status"] == 0 and inf["true_resid"] <= 1e-10, (k, inf)
        x = xf.download()
        assert oracle.true_residual(dims, U, 0.15, s, x) <= 1e-10
        if k in (0, 7):
            x1 = ctx.field(dims, "f64", lqcd.FULL)
            lqcd.solve_fields(g, srcs[k], 0.15, 1e-10, x1, opts)
            assert np.array_equal(x1.download(), x), k


@pytest.mark.parametrize("prec,compress", [("f32", 12), ("f16", 12), ("f32", 18), ("bf16", 12)])
def test_multi_rhs_shared_links_match_single(ctx, prec, compress):
    """Section 4's 12 point sources on 16^3x32, large enough for the shared-link multi-RHS
    Dslash (each site block's links loaded once for a group of sources): every solution equals
    the same solve alone and the same batch with per-source link loads
    (multi_rhs_links = -1), bit for bit, and meets 1e-10 by the oracle's residual."""
    dims = (16, 16, 16, 32)
    U = synth.random_links(dims, 0.5, seed=83)
    site = synth.point_site(dims)
    srcs_h = _point_sources(dims, site)
    g = ctx.gauge(dims, U, prec="f64")
    srcs = [ctx.field(dims, "f64", lqcd.FULL, data=s) for s in srcs_h]
    shared = [ctx.field(dims, "f64", lqcd.FULL) for _ in srcs_h]
    own = [ctx.field(dims, "f64", lqcd.FULL) for _ in srcs_h]
    o_sh = lqcd.solve_opts(sloppy_prec=prec, sloppy_compress=compress, multi_rhs_links=1)
    o_own = lqcd.solve_opts(sloppy_prec=prec, sloppy_compress=compress, multi_rhs_links=-1)
    infos = lqcd.solve_multi(g, srcs, 0.15, 1e-10, shared, o_sh)
    infos_own = lqcd.solve_multi(g, srcs, 0.15, 1e-10, own, o_own)
    x1 = ctx.field(dims, "f64", lqcd.FULL)
    for k, (inf, s) in enumerate(zip(infos, srcs_h)):
        assert inf["status"] == 0 and inf["true_resid"] <= 1e-10, (k, inf)
        assert infos_own[k]["iters"] == inf["iters"], k
        x = shared[k].download()
        assert np.array_equal(own[k].download(), x), k
        if k in (0, 5, 11):
            assert oracle.true_residual(dims, U, 0.15, s, x) <= 1e-10, k
            lqcd.solve_fields(g, srcs[k], 0.15, 1e-10, x1, o_sh)
            assert np.array_equal(x1.download(), x), k
    for f_ in srcs + shared + own + [x1, g]:
        f_.close()


def test_multi_rhs_full_size_24x48(ctx):
    """The benchmark's multi-RHS workload at full size: 24^3x48, kappa 0.15, eps 0.5 (seed
    1001), Section 4's 12 point sources at the seeded site, FP32-12 inner and FP64-class
    outer, solved together: every solution meets 1e-10 by the oracle's FP64 residual."""
    dims = (24, 24, 24, 48)
    U = synth.random_links(dims, 0.5, seed=synth.SEED_LINKS)
    site = synth.point_site(dims)
    g = ctx.gauge(dims, U, prec="f64")
    srcs_h = _point_sources(dims, site)
    srcs = [ctx.field(dims, "f64", lqcd.FULL, data=s_) for s_ in srcs_h]
    xs = [ctx.field(dims, "f64", lqcd.FULL) for _ in srcs_h]
    infos = lqcd.solve_multi(g, srcs, 0.15, 1e-10, xs, lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=12))
    for k, (inf, s_, x_) in enumerate(zip(infos, srcs_h, xs)):
        assert inf["status"] == 0, (k, inf)
        assert oracle.true_residual(dims, U, 0.15, s_, x_.download()) <= 1e-10, k
    for o in srcs + xs + [g]:
        o.close()


def test_engine_uneven_lattices_same_alone_and_in_mix(ctx):
    """Several lattices of different sizes and kappas in one engine: each result equals its
    solo solve bit for bit."""
    cases = [((4, 4, 4, 4), 0.12, 11), ((6, 4, 4, 6), 0.15, 12), ((4, 4, 2, 8), 0.14, 13),
             ((8, 4, 4, 4), 0.155, 14)]
    opts = lqcd.solve_opts(sloppy_prec="f16")
    eng = lqcd.Engine(ctx, opts, max_slots=8)
    items = []
    for dims, kappa, seed in cases:
        U = synth.random_links(dims, 0.5, seed=seed)
        b = synth.gaussian_spinor(dims, seed=seed + 100)
        g = ctx.gauge(dims, U, prec="f64")
        src = ctx.field(dims, "f64", lqcd.FULL, data=b)
        rid = eng.submit(g, src, kappa, 1e-10)
        items.append((rid, dims, kappa, U, b, g, src))
    while eng.step() > 0:
        pass
    done = set(eng.completed())
    assert done == {it[0] for it in items}
    for rid, dims, kappa, U, b, g, src in items:
        x = ctx.field(dims, "f64", lqcd.FULL)
        info = eng.result(rid, x)
        assert info["status"] == 0 and info["true_resid"] <= 1e-10
        xm = x.download()
        assert oracle.true_residual(dims, U, kappa, b, xm) <= 1e-10
        xs = ctx.field(dims, "f64", lqcd.FULL)
        lqcd.solve_fields(g, src, kappa, 1e-10, xs, opts)
        assert np.array_equal(xs.download(), xm)
    eng.close()


@pytest.mark.parametrize("nslots", [100, 140])
def test_engine_many_slots_same_alone_and_in_mix(ctx, nslots):
    """An engine holding more slots than the per-CTA slot view takes (128: the launches then
    stride over all tiles and read slot states from global memory) and one holding fewer
    (the view compacts the running slots): slots that converge and update at different
    iterations each give their solo result bit for bit."""
    shapes = [(4, 4, 4, 4), (4, 4, 2, 4), (2, 4, 4, 4)]
    opts = lqcd.solve_opts(sloppy_prec="f32")
    eng = lqcd.Engine(ctx, opts, max_slots=nslots)
    items = []
    for k in range(nslots):
        dims = shapes[k % 3]
        kappa = 0.12 + 0.03 * (k % 7) / 6
        U = synth.random_links(dims, 0.5, seed=3000 + k)
        g = ctx.gauge(dims, U, prec="f64")
        src = ctx.field(dims, "f64", lqcd.FULL, data=synth.gaussian_spinor(dims, seed=5000 + k))
        items.append((eng.submit(g, src, kappa, 1e-10), dims, kappa, g, src))
    while eng.step() > 0:
        pass
    iters = set()
    for rid, dims, kappa, g, src in items:
        x = ctx.field(dims, "f64", lqcd.FULL)
        info = eng.result(rid, x)
        assert info["status"] == 0 and info["true_resid"] <= 1e-10, info
        iters.add(info["iters"])
        xs = ctx.field(dims, "f64", lqcd.FULL)
        lqcd.solve_fields(g, src, kappa, 1e-10, xs, opts)
        assert np.array_equal(xs.download(), x.download()), (rid, dims, kappa)
        x.close()
        xs.close()
    assert len(iters) > 1  # the slots ran different iteration counts
    eng.close()
    for _, _, _, g, src in items:
        g.close()
        src.close()


def test_multi_group_reduction_alone_and_in_mix(ctx):
    """A slot of more than 1024 tiles has its reductions summed by several CTAs (a count
    fixed by its own tiles); in a batch with a small lattice it still gives its solo
    result bit for bit, and so does the small one."""
    big, small = (20, 20, 20, 40), (4, 4, 4, 8)  # V/2 = 160000 sites: 2500 tiles, 3 groups
    opts = lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=12)
    fields = []
    for dims, seed in ((big, 31), (small, 32)):
        g = ctx.gauge(dims, synth.random_links(dims, 0.4, seed=seed), prec="f64")
        src = ctx.field(dims, "f64", lqcd.FULL, data=synth.gaussian_spinor(dims, seed=seed + 1))
        fields.append((dims, g, src))
    eng = lqcd.Engine(ctx, opts, max_slots=4)
    ids = [eng.submit(g, src, 0.13, 1e-10) for _, g, src in fields]
    while eng.step() > 0:
        pass
    for rid, (dims, g, src) in zip(ids, fields):
        x = ctx.field(dims, "f64", lqcd.FULL)
        info = eng.result(rid, x)
        assert info["status"] == 0 and info["true_resid"] <= 1e-10, info
        solo = ctx.field(dims, "f64", lqcd.FULL)
        lqcd.solve_fields(g, src, 0.13, 1e-10, solo, opts)
        assert np.array_equal(solo.download(), x.download()), dims
    eng.close()


def test_solve_batch_matches_solo(ctx):
    """lqcd_solve_batch: systems on different lattices, gauges, kappas and tolerances (two
    sharing one gauge field) give each its solo result bit for bit; BiCGStab runs them in
    turn; bad arguments are refused."""
    opts = lqcd.solve_opts(sloppy_prec="f16", sloppy_compress=12)
    specs = [((6, 4, 4, 6), 0.15, 1e-10, 41), ((4, 4, 4, 8), 0.13, 1e-9, 42), ((8, 4, 4, 4), 0.14, 1e-10, 43)]
    gauges, srcs, kappas, tols = [], [], [], []
    for dims, kappa, tol, seed in specs:
        g = ctx.gauge(dims, synth.random_links(dims, 0.5, seed=seed), prec="f64")
        gauges.append(g)
        srcs.append(ctx.field(dims, "f64", lqcd.FULL, data=synth.gaussian_spinor(dims, seed=seed + 1)))
        kappas.append(kappa)
        tols.append(tol)
    # a second source on the first gauge field (multi-RHS inside the batch)
    gauges.append(gauges[0])
    srcs.append(ctx.field(specs[0][0], "f64", lqcd.FULL, data=synth.gaussian_spinor(specs[0][0], seed=49)))
    kappas.append(specs[0][1])
    tols.append(specs[0][2])
    for o in (opts, lqcd.solve_opts(sloppy_prec="f32", sloppy_compress=12, solver=lqcd.BICGSTAB)):
        xs = [ctx.field(g.dims, "f64", lqcd.FULL) for g in gauges]
        infos = lqcd.solve_batch(gauges, srcs, kappas, tols, xs, o)
        for g, src, kappa, tol, x, info in zip(gauges, srcs, kappas, tols, xs, infos):
            assert info["status"] == 0 and info["true_resid"] <= tol, info
            solo = ctx.field(g.dims, "f64", lqcd.FULL)
            lqcd.solve_fields(g, src, kappa, tol, solo, o)
            assert np.array_equal(solo.download(), x.download()), g.dims
    with pytest.raises(ValueError):
        lqcd.solve_batch(gauges, srcs[:2], kappas, tols, xs, opts)
    other = lqcd.Context(0)
    try:
        g2 = other.gauge(specs[1][0], synth.unit_links(specs[1][0]))
        with pytest.raises(lqcd.LqcdError):
            lqcd.solve_batch([gauges[0], g2], srcs[:2], kappas[:2], tols[:2], xs[:2], opts)
    finally:
        other.close()


def test_nonconvergence_reports_status(ctx):
    dims = (4, 4, 4, 4)
    U = synth.random_links(dims, 0.5, seed=3)
    b = synth.gaussian_spinor(dims, seed=4)
    g = ctx.gauge(dims, U)
    x, info = lqcd.solve(g, b, 0.15, 1e-10, lqcd.solve_opts(sloppy_prec="f32", maxiter=5))
    assert info["status"] == lqcd.ENOCONV
    assert info["iters"] >= 5 and info["true_resid"] > 1e-10


def test_nan_source_reports_nonfinite(ctx):
    dims = (4, 4, 4, 4)
    g = ctx.gauge(dims, synth.random_links(dims, 0.3, seed=5))
    b = synth.gaussian_spinor(dims, seed=6)
    b[17, 2, 1] = np.nan
    x, info = lqcd.solve(g, b, 0.12, 1e-10, lqcd.solve_opts(sloppy_prec="f32"))
    assert info["status"] == lqcd.ENONFINITE


def test_zero_source(ctx):
    dims = (4, 4, 4, 4)
    g = ctx.gauge(dims, synth.random_links(dims, 0.3, seed=5))
    x, info = lqcd.solve(g, np.zeros((256, 4, 3), complex), 0.12, 1e-10)
    assert info["status"] == 0 and np.all(x == 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_bicgstab_breakdown_on_singular_system(ctx, prec):
    """A singular system makes BiCGStab break down, reported as LQCD_EBREAKDOWN. With unit
    links, periodic t and kappa = 1/8, D_eo D_oe maps a constant spinor to 64 times itself,
    so Mhat = 1 - D_eo D_oe / 64 annihilates it. One real component equal to 1 on each of
    the 256 even sites of 4x4x4x8 gives |bhat| = 16, so the restart vector r = bhat / 16 and
    every hop sum are small integers over 16: the first <r0, Mhat p> is exactly zero."""
    dims = (4, 4, 4, 8)
    g = ctx.gauge(dims, synth.unit_links(dims), t_bc=+1)
    even = synth.parity_of_sites(dims) == 0
    b = np.zeros((synth.volume(dims), 4, 3), complex)
    b[even, 0, 0] = 1.0
    x, info = lqcd.solve(g, b, 0.125, 1e-10, lqcd.solve_opts(sloppy_prec=prec, solver=lqcd.BICGSTAB))
    assert info["status"] == lqcd.EBREAKDOWN, info
    assert info["iters"] == 0, info
    g.close()


def test_engine_budget_and_cancel(ctx):
    dims = (4, 4, 4, 4)
    g = ctx.gauge(dims, synth.random_links(dims, 0.3, seed=7))
    src = ctx.field(dims, "f64", lqcd.FULL, data=synth.gaussian_spinor(dims, seed=8))
    probe = lqcd.Engine(ctx, lqcd.solve_opts(sloppy_prec="f32"))
    need = probe.request_bytes(dims)
    probe.close()
    tiny = lqcd.Engine(ctx, lqcd.solve_opts(sloppy_prec="f32"), hbm_budget=need // 2)
    with pytest.raises(lqcd.LqcdError) as e:
        tiny.submit(g, src, 0.12, 1e-10)
    assert e.value.code == lqcd.ENOMEM
    tiny.close()
    one = lqcd.Engine(ctx, lqcd.solve_opts(sloppy_prec="f32"), hbm_budget=need + need // 2)
    r1 = one.submit(g, src, 0.12, 1e-10)
    assert r1 is not None
    assert one.submit(g, src, 0.12, 1e-10) is None  # busy: budget holds one request
    one.cancel(r1, lqcd.ETIMEOUT)
    one.step()
    assert one.completed() == [r1]
    x = ctx.field(dims, "f64", lqcd.FULL)
    with pytest.raises(lqcd.LqcdError) as e:
        one.result(r1, x)
    assert e.value.code == lqcd.ETIMEOUT
    assert one.submit(g, src, 0.12, 1e-10) is not None  # slot and budget freed
    one.close()


@pytest.mark.slow
def test_near_critical_16x32_mixed_f16(ctx):
    """16^3 x 32, kappa 0.155, eps 0.8 (the ill-conditioned workload at reduced volume):
    FP16 sloppy CG with FP64 reliable updates reaches 1e-10 (oracle-measured residual)."""
    dims = (16, 16, 16, 32)
    U = synth.random_links(dims, 0.8)
    b = synth.gaussian_spinor(dims)
    g = ctx.gauge(dims, U, prec="f64")
    x, info = lqcd.solve(g, b, 0.155, 1e-10, lqcd.solve_opts(sloppy_prec="f16", sloppy_compress=12))
    assert info["status"] == 0, info
    assert oracle.true_residual(dims, U, 0.155, b, x) <= 1e-10


def test_full_size_solves_32x64(ctx):
    """The bench's solve workload at full size (32^3x64, kappa 0.155, eps 0.8, seeds 1001 /
    2002): mixed FP16-12 CG, Wilson and twisted mass (mu 0.01), each meets 1e-10 on the full
    operator as measured by the oracle on the returned solution. The Wilson solution is also
    compared element by element with the oracle's own FP64 even-odd CG solution (to 1e-12,
    computed once per machine): both solve the same system to a residual of 1e-10 or
    below, so they differ by at most cond(M) times that; 1e-8 allows cond(M) up to 100."""
    import oracle_cache
    dims, kappa, mu = (32, 32, 32, 64), 0.155, 0.01
    U, b, xo = oracle_cache.eo_solution(dims, 0.8, kappa, 0.0, synth.SEED_LINKS, synth.SEED_SOURCE, 1e-12)
    g = ctx.gauge(dims, U, prec="f64")
    for m in (0.0, mu):
        x, info = lqcd.solve(g, b, kappa, 1e-10, lqcd.solve_opts(sloppy_prec="f16", mu=m))
        assert info["status"] == 0, (m, info)
        assert oracle.true_residual(dims, U, kappa, b, x, mu=m) <= 1e-10, m
        if m == 0.0:
            err = np.linalg.norm(x - xo) / np.linalg.norm(xo)
            assert err < 1e-8, err
    g.close()
