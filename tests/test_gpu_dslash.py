"""GPU parity of the even-odd Wilson Dslash, Mhat and M against the FP64 oracle.

DF64 (double-float storage and arithmetic, 48-bit significand) is held to the
FP64 bar.

Paper Section 3: the even-odd preconditioned hopping term "dslash" is the hot
kernel. Every precision / compression / dagger / parity combination is
compared element by element with the oracle on the same seeded inputs.
Tolerance (max |gpu - oracle| / max |oracle|): FP64 1e-12, FP32 1e-5 (the
stated bars); FP16 4e-3 and BF16 3e-2, derived from the unit roundoff of the
storage (2^-11, 2^-8) times the ~8-term sums per output component.
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


def _par(dims, p):
    return synth.parity_of_sites(dims) == p


# ragged: Vh = 720 -> 5.6 tiles of 128; 2^4: coinciding neighbours; 4^4: small workload
LATTICES = [(6, 6, 4, 10), (2, 2, 2, 2), (4, 4, 4, 4), (2, 4, 6, 4)]


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("compress", [18, 12])
def test_dslash_eo_parity(ctx, dims, prec, compress):
    U = synth.random_links(dims, 0.5, seed=1001)
    psi = synth.gaussian_spinor(dims, seed=2002)
    g = ctx.gauge(dims, U, prec=prec, compress=compress, t_bc=-1)
    fin = ctx.field(dims, prec, lqcd.FULL, data=psi)
    for p in (0, 1):
        for dag in (False, True):
            fout = ctx.field(dims, prec, p)
            lqcd.dslash_eo(g, fin, fout, p, dagger=dag)
            got = fout.download()
            ref = oracle.hop_eo(dims, U, psi, p, dagger=dag)
            err = _rel_err(got, ref, _par(dims, p))
            assert err < TOL[prec], (prec, compress, p, dag, err)


@pytest.mark.parametrize("t_bc", [1, -1])
def test_dslash_boundary_conditions(ctx, t_bc):
    dims = (4, 2, 2, 6)
    U = synth.random_links(dims, 0.8, seed=5)
    psi = synth.gaussian_spinor(dims, seed=6)
    g = ctx.gauge(dims, U, prec="f64", t_bc=t_bc)
    fin = ctx.field(dims, "f64", lqcd.FULL, data=psi)
    fout = ctx.field(dims, "f64", lqcd.FULL)
    for p in (0, 1):
        lqcd.dslash_eo(g, fin, fout, p)
    got = fout.download()
    ref = oracle.hop(dims, U, psi, t_bc=t_bc)
    assert _rel_err(got, ref) < 1e-12


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_apply_M_and_Mhat(ctx, prec):
    dims = (6, 4, 4, 6)
    kappa = 0.15
    U = synth.random_links(dims, 0.5, seed=11)
    psi = synth.gaussian_spinor(dims, seed=12)
    g = ctx.gauge(dims, U, prec=prec, compress=12)
    fin = ctx.field(dims, prec, lqcd.FULL, data=psi)
    fout = ctx.field(dims, prec, lqcd.FULL)
    for dag in (False, True):
        lqcd.apply_M(g, kappa, fin, fout, dagger=dag)
        assert _rel_err(fout.download(), oracle.apply_M(dims, U, kappa, psi, dagger=dag)) < TOL[prec]
        fe = ctx.field(dims, prec, lqcd.EVEN, data=psi)
        fo = ctx.field(dims, prec, lqcd.EVEN)
        lqcd.apply_Mhat(g, kappa, fe, fo, dagger=dag)
        psi_e = psi * _par(dims, 0)[:, None, None]
        ref = oracle.apply_Mhat(dims, U, kappa, psi_e, dagger=dag)
        assert _rel_err(fo.download(), ref, _par(dims, 0)) < TOL[prec]


def test_kappa_zero_is_identity(ctx):
    dims = (4, 4, 2, 2)
    U = synth.random_links(dims, 0.5, seed=3)
    psi = synth.gaussian_spinor(dims, seed=4)
    g = ctx.gauge(dims, U, prec="f64")
    fin = ctx.field(dims, "f64", lqcd.FULL, data=psi)
    fout = ctx.field(dims, "f64", lqcd.FULL)
    lqcd.apply_M(g, 0.0, fin, fout)
    assert np.array_equal(fout.download(), psi)


def test_gauge_covariance_on_gpu(ctx):
    """M[U^g](g psi) = g M[U] psi evaluated entirely on the GPU (FP64)."""
    from oracle import dense
    dims = (4, 4, 4, 6)
    U = synth.random_links(dims, 0.5, seed=31)
    gt = synth.gauge_transform_field(dims, seed=32)
    psi = synth.gaussian_spinor(dims, seed=33)
    kappa = 0.14
    outs = []
    for links, src in ((U, psi), (dense.gauge_transform_links(dims, U, gt),
                                  dense.gauge_transform_spinor(gt, psi))):
        g = ctx.gauge(dims, links, prec="f64")
        fin = ctx.field(dims, "f64", lqcd.FULL, data=src)
        fout = ctx.field(dims, "f64", lqcd.FULL)
        lqcd.apply_M(g, kappa, fin, fout)
        outs.append(fout.download())
    assert _rel_err(outs[1], dense.gauge_transform_spinor(gt, outs[0])) < 1e-12


def test_norm_copy_and_device_io(ctx):
    import torch
    dims = (4, 2, 4, 4)
    psi = synth.gaussian_spinor(dims, seed=9)
    f64 = ctx.field(dims, "f64", lqcd.FULL, data=psi)
    assert abs(f64.norm2() - np.vdot(psi, psi).real) < 1e-10 * np.vdot(psi, psi).real
    f32 = ctx.field(dims, "f32", lqcd.FULL)
    f32.copy_from(f64, 2.0)
    assert _rel_err(f32.download(), 2 * psi) < 1e-6
    t = torch.from_numpy(psi).cuda()
    fd = ctx.field(dims, "f64", lqcd.FULL)
    fd.upload(t)
    out = torch.zeros_like(t)
    fd.download(out)
    ctx.sync()
    assert np.array_equal(out.cpu().numpy(), psi)


def test_half_field_download_leaves_other_parity(ctx):
    dims = (4, 4, 2, 2)
    psi = synth.gaussian_spinor(dims, seed=19)
    f = ctx.field(dims, "f64", lqcd.ODD, data=psi)
    host = np.full_like(psi, 7.0 + 1j)
    f.download(host)
    odd = _par(dims, 1)
    assert np.array_equal(host[odd], psi[odd])
    assert np.all(host[~odd] == 7.0 + 1j)


def test_invalid_arguments_fail_loudly(ctx):
    with pytest.raises(lqcd.LqcdError):
        ctx.field((3, 4, 4, 4), "f64")
    dims = (4, 4, 4, 4)
    g = ctx.gauge(dims, synth.unit_links(dims), prec="f64")
    fe = ctx.field(dims, "f64", lqcd.EVEN)
    fo = ctx.field(dims, "f64", lqcd.EVEN)
    with pytest.raises(lqcd.LqcdError):
        lqcd.dslash_eo(g, fe, fo, 0)  # input must hold the odd parity


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
def test_dslash_sampled_sites_16x32(ctx, prec):
    """Benchmark workload shape (16^3 x 32, eps = 0.5): sampled output sites vs the oracle."""
    dims = (16, 16, 16, 32)
    U = synth.random_links(dims, 0.5, seed=1001)
    psi = synth.gaussian_spinor(dims, seed=2002)
    g = ctx.gauge(dims, U, prec=prec, compress=18 if prec != "f16" else 12)
    fin = ctx.field(dims, prec, lqcd.FULL, data=psi)
    fout = ctx.field(dims, prec, lqcd.FULL)
    for p in (0, 1):
        lqcd.dslash_eo(g, fin, fout, p)
    got = fout.download()
    rng = np.random.default_rng(5)
    sites = np.concatenate([rng.integers(0, synth.volume(dims), 3000),
                            [0, synth.volume(dims) - 1]])
    ref = oracle.hop_sites(dims, U, psi, sites)
    assert _rel_err(got[sites], ref) < TOL[prec]


def test_objects_outlive_context_handle():
    """Destroying the context handle first is safe: its fields and gauge keep it alive."""
    c = lqcd.Context(0)
    dims = (4, 4, 4, 4)
    psi = synth.gaussian_spinor(dims, seed=1)
    g = c.gauge(dims, synth.random_links(dims, 0.3, seed=2), prec="f64")
    f = c.field(dims, "f64", lqcd.FULL, data=psi)
    o = c.field(dims, "f64", lqcd.FULL)
    c.close()
    for p in (0, 1):
        lqcd.dslash_eo(g, f, o, p)
    assert np.abs(o.download() - oracle.hop(dims, synth.random_links(dims, 0.3, seed=2), psi)).max() < 1e-12 * 100
    f.close()
    o.close()
    g.close()


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16"])
@pytest.mark.parametrize("same_size", [False, True])
def test_dslash_batch_matches_oracle(ctx, prec, same_size):
    """n independent applications in one launch (mixed lattice sizes, or equal sizes in the
    interleaved tile order) each equal the oracle's hopping term."""
    shapes = [(6, 6, 4, 10)] * 3 if same_size else [(4, 4, 4, 4), (6, 6, 4, 10), (2, 4, 6, 4)]
    gs, fins, fouts, refs = [], [], [], []
    for k, dims in enumerate(shapes):
        U = synth.random_links(dims, 0.5, seed=300 + k)
        psi = synth.gaussian_spinor(dims, seed=400 + k)
        gs.append(ctx.gauge(dims, U, prec=prec, compress=12 if prec == "f16" else 18))
        fins.append(ctx.field(dims, prec, lqcd.ODD, data=psi))
        fouts.append(ctx.field(dims, prec, lqcd.EVEN))
        refs.append((dims, oracle.hop_eo(dims, U, psi, 0, dagger=True)))
    b = lqcd.DslashBatch(gs, fins, fouts, 0, dagger=True)
    b.apply()
    b.apply()
    for f, (dims, ref) in zip(fouts, refs):
        assert _rel_err(f.download(), ref, _par(dims, 0)) < TOL[prec]
    b.close()


def _nan_spinor(dims):
    return np.full((synth.volume(dims), 4, 3), complex(np.nan, np.nan))


@pytest.mark.parametrize("prec", ["f64", "df64", "f32", "f16", "bf16"])
def test_outputs_fully_written(ctx, prec):
    """Coverage check with poisoned outputs: every output field is filled with NaN before the
    kernel, and every site of the parity the kernel writes must come back finite. Ragged
    lattices (partial last tiles), single launches of both parities, a batch of mixed
    sizes, Mhat into an even field, and a solve into a poisoned solution field."""
    shapes = [(6, 6, 4, 10), (2, 4, 6, 4), (4, 4, 4, 4)]
    nr = 12 if prec in ("f16", "bf16") else 18
    gs, fins, fouts = [], [], []
    for k, dims in enumerate(shapes):
        gs.append(ctx.gauge(dims, synth.random_links(dims, 0.5, seed=500 + k), prec=prec, compress=nr))
        fins.append(ctx.field(dims, prec, lqcd.FULL, data=synth.gaussian_spinor(dims, seed=600 + k)))
        fouts.append(ctx.field(dims, prec, lqcd.FULL, data=_nan_spinor(dims)))
    for g, fi, fo in zip(gs, fins, fouts):
        for p in (0, 1):
            lqcd.dslash_eo(g, fi, fo, p)
        assert np.isfinite(fo.download()).all()
    for fo, dims in zip(fouts, shapes):
        fo.upload(_nan_spinor(dims))
    b = lqcd.DslashBatch(gs, fins, fouts, 1, dagger=True)
    b.apply()
    for fo, dims in zip(fouts, shapes):
        assert np.isfinite(fo.download()[_par(dims, 1)]).all(), dims
    b.close()
    for g, fi, fo, dims in zip(gs, fins, fouts, shapes):
        fo.upload(_nan_spinor(dims))
        lqcd.apply_Mhat(g, 0.13, fi, fo)
        assert np.isfinite(fo.download()[_par(dims, 0)]).all(), dims
    dims = shapes[0]
    g64 = ctx.gauge(dims, synth.random_links(dims, 0.5, seed=500), prec="f64")
    src = ctx.field(dims, "f64", lqcd.FULL, data=synth.gaussian_spinor(dims, seed=610))
    x = ctx.field(dims, "f64", lqcd.FULL, data=_nan_spinor(dims))
    sp = prec if prec != "f64" else "f64"
    info = lqcd.solve_fields(g64, src, 0.13, 1e-10, x, lqcd.solve_opts(sloppy_prec=sp, sloppy_compress=nr))
    assert info["status"] == 0 and np.isfinite(x.download()).all()
    for o in gs + fins + fouts + [g64, src, x]:
        o.close()


@pytest.fixture(scope="module")
def bench_sets():
    """The benchmark's 10 field sets: 16^3x32 links exp(i 0.5 H) and Gaussian spinors, seeds
    1001 + k and 2002 + k (bench.py's generator)."""
    dims = (16, 16, 16, 32)
    return dims, [(synth.random_links(dims, 0.5, seed=synth.SEED_LINKS + k),
                   synth.gaussian_spinor(dims, seed=synth.SEED_SOURCE + k)) for k in range(10)]


@pytest.mark.parametrize("prec", ["f32", "f64", "df64"])
def test_bench_launch_configuration(ctx, bench_sets, prec):
    """The launch the benchmark times, at full size: one batch of the 10 field sets (10 slots
    of 16^3x32, 18-real links, antiperiodic t, out parity 0) applied twice; 500 sampled even
    output sites of every set against the oracle's hopping term at those sites."""
    dims, sets = bench_sets
    gs = [ctx.gauge(dims, U, prec=prec, compress=18, t_bc=-1) for U, _ in sets]
    fins = [ctx.field(dims, prec, lqcd.ODD, data=psi) for _, psi in sets]
    fouts = [ctx.field(dims, prec, lqcd.EVEN) for _ in sets]
    b = lqcd.DslashBatch(gs, fins, fouts, 0)
    b.apply()
    b.apply()
    even = np.flatnonzero(synth.parity_of_sites(dims) == 0)
    rng = np.random.default_rng(11)
    for k, ((U, psi), fo) in enumerate(zip(sets, fouts)):
        sites = np.concatenate([rng.choice(even, 500, replace=False), even[[0, -1]]])
        ref = oracle.hop_sites(dims, U, psi, sites)
        assert _rel_err(fo.download()[sites], ref) < TOL[prec], k
    b.close()
    for o in gs + fins + fouts:
        o.close()


@pytest.mark.parametrize("form", [0, 1])
def test_df64_both_forms(ctx, form):
    """Both Dslash forms of double-float (one thread per site, three per site) meet the FP64 bar."""
    dims = (6, 6, 4, 10)
    U = synth.random_links(dims, 0.5, seed=77)
    psi = synth.gaussian_spinor(dims, seed=78)
    lqcd.set_dslash_form("df64", form)
    try:
        g = ctx.gauge(dims, U, prec="df64", compress=18)
        fin = ctx.field(dims, "df64", lqcd.FULL, data=psi)
        fout = ctx.field(dims, "df64", lqcd.FULL)
        for p in (0, 1):
            for dag in (False, True):
                lqcd.dslash_eo(g, fin, fout, p, dagger=dag)
                ref = oracle.hop_eo(dims, U, psi, p, dagger=dag)
                assert _rel_err(fout.download(), ref, _par(dims, p)) < 1e-12
    finally:
        lqcd.set_dslash_form("df64", 1)
