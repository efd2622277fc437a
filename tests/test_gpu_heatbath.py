"""GPU SU(3) heatbath and plaquette against the FP64 oracle (paper Section 3: the pure-gauge
SU(3) heatbath, citing Creutz).

Both sides draw the same Philox4x64-10 numbers (counter per link, sweep, subgroup and
attempt), so a GPU sweep equals the oracle's sweep link by link up to rounding: FMA
contraction, the order of the staple sum, CUDA's and the C library's log1p / expm1 /
sqrt / sin / cos, the GPU's V <- R V update against the oracle's V = U W.

The sweep itself amplifies rounding: the SU(2) rotation v = c / |c| is ill-conditioned
where |c| is small, and at beta = 0 a 1e-15 relative perturbation of the input links
grows to ~1e-12 after one sweep and ~1e-10 after two (measured on the oracle). So the
bar is relative to the oracle's own spread: each case perturbs the oracle's input by
1e-15 (relative), takes the largest change d of its output, and requires
max |gpu - oracle| <= 100 d + 1e-13 on every link element. An accept decision flipped
by rounding (probability ~1e-16 per draw) would give an O(1) difference and fail.
"""
import numpy as np
import pytest

from oracle import gauge as ogauge
from paper_1112_5280_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = lqcd.Context(0)
    yield c
    c.close()


def _oracle_spread(dims, U0, beta, **kw):
    """Oracle output and the largest change of it under a 1e-15 relative input perturbation."""
    ref, fails = ogauge.heatbath(dims, U0, beta, **kw)
    rng = np.random.default_rng(123)
    pert, _ = ogauge.heatbath(dims, U0 * (1 + 1e-15 * rng.standard_normal(U0.shape)), beta, **kw)
    return ref, fails, np.abs(pert - ref).max()


# ragged: V/2 = 720 is 5.6 CTAs of 128; 2^4: coinciding neighbours
@pytest.mark.parametrize("dims", [(6, 6, 4, 10), (2, 2, 2, 2), (4, 4, 4, 8)])
@pytest.mark.parametrize("beta", [0.0, 2.3, 6.0, 40.0])  # 40: alpha up to ~40, span = 1 in FP32
def test_heatbath_matches_oracle(ctx, dims, beta):
    U0 = synth.random_links(dims, 0.8, seed=1001)
    g = ctx.gauge(dims, U0, prec="f64")
    fails = g.heatbath(beta, nsweeps=2, seed=17, sweep0=5)
    ref, ofails, spread = _oracle_spread(dims, U0, beta, seed=17, sweep0=5, nsweeps=2)
    assert fails == ofails == 0
    got = g.download()
    err = np.abs(got - ref).max()
    assert err <= 100 * spread + 1e-13, (err, spread)
    assert abs(g.plaquette() - ogauge.plaquette(dims, got)) < 1e-13
    g.close()


def test_heatbath_without_reunit_and_in_pieces(ctx):
    """Two sweeps in one call equal one sweep per call with consecutive sweep numbers."""
    dims = (4, 4, 2, 6)
    U0 = synth.random_links(dims, 0.5, seed=7)
    a = ctx.gauge(dims, U0)
    b = ctx.gauge(dims, U0)
    a.heatbath(5.7, nsweeps=2, seed=3, sweep0=0, reunit=False)
    b.heatbath(5.7, nsweeps=1, seed=3, sweep0=0, reunit=False)
    b.heatbath(5.7, nsweeps=1, seed=3, sweep0=1, reunit=False)
    assert np.array_equal(a.download(), b.download())
    ref, _, spread = _oracle_spread(dims, U0, 5.7, seed=3, nsweeps=2, reunit=False)
    assert np.abs(a.download() - ref).max() <= 100 * spread + 1e-13


def test_plaquette_and_download(ctx):
    dims = (6, 4, 4, 8)
    U = synth.random_links(dims, 0.7, seed=9)
    g = ctx.gauge(dims, U, prec="f64")
    assert np.array_equal(g.download(), U)
    assert abs(g.plaquette() - ogauge.plaquette(dims, U)) < 1e-13
    gu = ctx.gauge(dims, synth.unit_links(dims))
    assert gu.plaquette() == 1.0


def test_derived_copies_follow_the_update(ctx):
    """After a heatbath the FP32 / FP16-12 copies used by the Dslash hold the new links."""
    import oracle
    dims = (4, 4, 4, 4)
    U0 = synth.random_links(dims, 0.5, seed=11)
    g = ctx.gauge(dims, U0, prec="f32", compress=18)
    g.add_copy("f16", 12)
    g.heatbath(5.5, nsweeps=1, seed=1)
    U1 = g.download()
    psi = synth.gaussian_spinor(dims, seed=12)
    for prec, tol in (("f32", 1e-5), ("f16", 4e-3)):
        fin = ctx.field(dims, prec, lqcd.FULL, data=psi)
        fout = ctx.field(dims, prec, lqcd.EVEN)
        lqcd.dslash_eo(g, fin, fout, 0)
        ref = oracle.hop_eo(dims, U1, psi, 0)
        ev = synth.parity_of_sites(dims) == 0
        assert np.abs(fout.download()[ev] - ref[ev]).max() / np.abs(ref[ev]).max() < tol, prec


def test_heatbath_rejects_bad_beta(ctx):
    dims = (2, 2, 2, 2)
    g = ctx.gauge(dims, synth.unit_links(dims))
    for beta in (-1.0, float("nan"), float("inf")):
        with pytest.raises(lqcd.LqcdError):
            g.heatbath(beta)
