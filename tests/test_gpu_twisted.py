"""GPU parity of the twisted-mass operators and solves against the FP64 oracle.

Paper Section 3: the N_f = 2 twisted-mass fermion matrix M = 1 - kappa D +
2 i kappa mu g5 (one flavour; the other has -mu), even-odd preconditioned with
the site-diagonal A = 1 + 2 i kappa mu g5: Mhat = A - kappa^2 D_eo A^-1 D_oe.
The bars are those of the Wilson operator (the twist adds one complex multiply
per component): FP64 and DF64 1e-12, FP32 1e-5, FP16 4e-3, BF16 3e-2 (max
|gpu - oracle| / max |oracle|); solves reach ||b - M x|| <= tol ||b|| measured by
the oracle with the same mu.
"""
import numpy as np
import pytest

import oracle
from paper_1112_5280_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "df64": 1e-12, "f32": 1e-5, "f16": 4e-3, "bf16": 3e-2}


@pytest.fixture(scope="module")
def ctx():
    c = lqcd.Context(0)
    yield c
    c.close()


def _rel_err(a, b, mask=None):
    if mask is not None:
        a, b = a[mask], b[mask]
    return np.abs(a - b).max() / np.abs(b).max()


def _even(dims):
    return synth.parity_of_sites(dims) == 0


@pytest.mark.parametrize("dims", [(6, 6, 4, 10), (4, 4, 4, 4)])
@pytest.mark.parametrize("prec,compress", [("f64", 18), ("df64", 18), ("f32", 12), ("f16", 12),
                                           ("bf16", 12)])
@pytest.mark.parametrize("mu", [0.3, -0.05])
def test_apply_M_and_Mhat_twisted(ctx, dims, prec, compress, mu):
    kappa = 0.155
    U = synth.random_links(dims, 0.5, seed=21)
    psi = synth.gaussian_spinor(dims, seed=22)
    g = ctx.gauge(dims, U, prec=prec, compress=compress)
    fin = ctx.field(dims, prec, lqcd.FULL, data=psi)
    fout = ctx.field(dims, prec, lqcd.FULL)
    ev = _even(dims)
    psi_e = psi * ev[:, None, None]
    for dag in (False, True):
        lqcd.apply_M(g, kappa, fin, fout, dagger=dag, mu=mu)
        ref = oracle.apply_M(dims, U, kappa, psi, dagger=dag, mu=mu)
        assert _rel_err(fout.download(), ref) < TOL[prec], ("M", dag)
        fe = ctx.field(dims, prec, lqcd.EVEN, data=psi)
        fo = ctx.field(dims, prec, lqcd.EVEN)
        lqcd.apply_Mhat(g, kappa, fe, fo, dagger=dag, mu=mu)
        ref = oracle.apply_Mhat(dims, U, kappa, psi_e, dagger=dag, mu=mu)
        assert _rel_err(fo.download(), ref, ev) < TOL[prec], ("Mhat", dag)


def test_mu_zero_entry_points_equal_wilson(ctx):
    """The twisted entry points at mu = 0 are the Wilson operator bit for bit."""
    dims = (4, 4, 2, 6)
    U = synth.random_links(dims, 0.5, seed=23)
    psi = synth.gaussian_spinor(dims, seed=24)
    g = ctx.gauge(dims, U, prec="f32")
    lib = lqcd.load()
    fin = ctx.field(dims, "f32", lqcd.FULL, data=psi)
    a, b = ctx.field(dims, "f32", lqcd.FULL), ctx.field(dims, "f32", lqcd.FULL)
    lqcd.apply_M(g, 0.14, fin, a)
    assert lib.lqcd_apply_M_tm(g.h, 0.14, 0.0, fin.h, b.h, 0) == 0
    assert np.array_equal(a.download(), b.download())
    assert lib.lqcd_apply_Mhat_tm(g.h, 0.14, 0.0, fin.h, b.h, 1) == 0
    lqcd.apply_Mhat(g, 0.14, fin, a, dagger=True)
    ev = _even(dims)
    assert np.array_equal(a.download()[ev], b.download()[ev])


def test_twisted_flavour_hermiticity_on_gpu(ctx):
    """<phi, M(mu) psi> = <g5 M(-mu) g5 phi, psi> with both sides from the GPU."""
    dims = (6, 4, 4, 6)
    U = synth.random_links(dims, 0.5, seed=25)
    phi, psi = synth.gaussian_spinor(dims, seed=26), synth.gaussian_spinor(dims, seed=27)
    g5 = np.array([1, 1, -1, -1])[None, :, None]
    g = ctx.gauge(dims, U, prec="f64")
    out = ctx.field(dims, "f64", lqcd.FULL)
    lqcd.apply_M(g, 0.15, ctx.field(dims, "f64", lqcd.FULL, data=psi), out, mu=0.2)
    lhs = np.vdot(phi, out.download())
    lqcd.apply_M(g, 0.15, ctx.field(dims, "f64", lqcd.FULL, data=g5 * phi), out, mu=-0.2)
    rhs = np.vdot(g5 * out.download(), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _tm_solve_check(ctx, dims, kappa, mu, prec, compress=12, solver=lqcd.CG, tol=1e-10, seed=31):
    U = synth.random_links(dims, 0.5, seed=seed)
    b = synth.gaussian_spinor(dims, seed=seed + 1)
    g = ctx.gauge(dims, U, prec="f64")
    opts = lqcd.solve_opts(sloppy_prec=prec, sloppy_compress=compress, solver=solver, mu=mu)
    x, info = lqcd.solve(g, b, kappa, tol, opts)
    assert info["status"] == 0, info
    assert oracle.true_residual(dims, U, kappa, b, x, mu=mu) <= tol
    assert oracle.true_residual(dims, U, kappa, b, x) > 10 * tol  # the twist was applied
    xo, st, _, _ = oracle.solve(dims, U, kappa, b, tol=tol * 1e-2, method=oracle.METHOD_CG_EO, mu=mu)
    assert st == 0
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-8
    return x, info


@pytest.mark.parametrize("prec,compress", [("f64", 18), ("df64", 18), ("f32", 12), ("f16", 12),
                                           ("bf16", 12)])
def test_twisted_cg(ctx, prec, compress):
    """CG on Mhat^dag Mhat with the twisted Schur operator, every sloppy precision."""
    _tm_solve_check(ctx, (6, 4, 4, 6), 0.16, 0.05, prec, compress)


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_twisted_bicgstab(ctx, prec):
    _tm_solve_check(ctx, (6, 4, 4, 6), 0.16, 0.05, prec, 12, solver=lqcd.BICGSTAB)
    _tm_solve_check(ctx, (4, 4, 4, 4), 0.14, -0.2, prec, 18, solver=lqcd.BICGSTAB, seed=41)


def test_engine_mixes_flavours_and_kappas(ctx):
    """+mu, -mu and Wilson requests in one engine: each result equals its solo solve bit
    for bit and meets the oracle's residual with its own mu."""
    opts = lqcd.solve_opts(sloppy_prec="f16")
    eng = lqcd.Engine(ctx, opts, max_slots=8)
    cases = [((6, 4, 4, 6), 0.16, 0.05, 51), ((6, 4, 4, 6), 0.16, -0.05, 51),
             ((4, 4, 4, 8), 0.15, 0.0, 52), ((4, 4, 2, 8), 0.14, 0.3, 53)]
    items = []
    for dims, kappa, mu, seed in cases:
        U = synth.random_links(dims, 0.5, seed=seed)
        b = synth.gaussian_spinor(dims, seed=seed + 100)
        g = ctx.gauge(dims, U, prec="f64")
        src = ctx.field(dims, "f64", lqcd.FULL, data=b)
        items.append((eng.submit(g, src, kappa, 1e-10, mu=mu), dims, kappa, mu, U, b, g, src))
    while eng.step() > 0:
        pass
    for rid, dims, kappa, mu, U, b, g, src in items:
        x = ctx.field(dims, "f64", lqcd.FULL)
        info = eng.result(rid, x)
        assert info["status"] == 0, info
        xm = x.download()
        assert oracle.true_residual(dims, U, kappa, b, xm, mu=mu) <= 1e-10
        xs = ctx.field(dims, "f64", lqcd.FULL)
        o = lqcd.solve_opts(sloppy_prec="f16", mu=mu)
        lqcd.solve_fields(g, src, kappa, 1e-10, xs, o)
        assert np.array_equal(xs.download(), xm)
    eng.close()


def test_twisted_rejects_nonfinite_mu(ctx):
    dims = (4, 4, 4, 4)
    g = ctx.gauge(dims, synth.random_links(dims, 0.3, seed=5))
    f = ctx.field(dims, "f64", lqcd.FULL, data=synth.gaussian_spinor(dims, seed=6))
    out = ctx.field(dims, "f64", lqcd.FULL)
    with pytest.raises(lqcd.LqcdError):
        lqcd.apply_M(g, 0.12, f, out, mu=float("nan"))
    with pytest.raises(lqcd.LqcdError):
        lqcd.solve(g, synth.gaussian_spinor(dims, seed=6), 0.12, 1e-10,
                   lqcd.solve_opts(sloppy_prec="f32", mu=float("inf")))
