"""The CUDA path against the golden fixtures (tests/golden), without running the oracle's
solvers, sweeps or integrators (the trajectory's pseudofermion input is built by the oracle).

Bars as in the parity tests: FP64 operators 1e-12 of the largest entry; the mixed FP16
solve within 1e-8 relative of the solution's norm (tol 1e-10 times the condition of this
small system); two heatbath sweeps within 1e-10 (double-float algebra, chaotic
amplification of 1e-15 input differences stays below 1e-12 at beta 2.3 over two sweeps);
the trajectory within 1e-8 (its forces come from solves to 1e-12) and dH within 1e-7.
"""
import os
import sys

import numpy as np
import pytest

from paper_1112_5280_gb300 import lqcd, synth

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_golden as mg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = lqcd.Context(0)
    yield c
    c.close()


def _even(dims):
    return synth.parity_of_sites(dims) == 0


def test_hop_and_mhat(ctx):
    dims = (2, 2, 2, 4)
    U = synth.random_links(dims, 0.5, seed=1001)
    psi = synth.gaussian_spinor(dims, seed=2002)
    g = ctx.gauge(dims, U, prec="f64", t_bc=-1)
    fin = ctx.field(dims, "f64", lqcd.FULL, data=psi)
    fout = ctx.field(dims, "f64", lqcd.FULL)
    for p in (0, 1):
        lqcd.dslash_eo(g, fin, fout, p)
    want = mg.read(mg.HOP[0])
    got = fout.download().ravel()
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()
    fe = ctx.field(dims, "f64", lqcd.EVEN, data=psi)
    fo = ctx.field(dims, "f64", lqcd.EVEN)
    lqcd.apply_Mhat(g, 0.15, fe, fo, mu=0.1)
    want = mg.read(mg.MHAT[0])
    got = fo.download()[_even(dims)].ravel()
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def test_solve(ctx):
    dims = (4, 4, 4, 4)
    g = ctx.gauge(dims, synth.random_links(dims, 0.3, seed=1001), prec="f64")
    x, info = lqcd.solve(g, synth.gaussian_spinor(dims, seed=2002), 0.12, 1e-10,
                         lqcd.solve_opts(sloppy_prec="f16", sloppy_compress=12))
    assert info["status"] == 0
    want = mg.read(mg.SOLVE[0])
    norm = np.sqrt(want[0].real)
    got = np.concatenate([x[s].ravel() for s in mg.SOLVE_SITES])
    assert np.abs(got - want[1:]).max() < 1e-8 * norm


def test_heatbath(ctx):
    dims = (2, 2, 2, 2)
    g = ctx.gauge(dims, synth.random_links(dims, 0.8, seed=1001), prec="f64")
    assert g.heatbath(2.3, nsweeps=2, seed=17, sweep0=5) == 0
    want = mg.read(mg.HEATBATH[0])
    assert abs(g.plaquette() - want[0].real) < 1e-10
    assert np.abs(g.download()[0].ravel() - want[1:]).max() < 1e-10


def test_trajectory(ctx):
    from oracle import hmc as ohmc  # the pseudofermion phi = Mhat^dag eta is an input here
    dims, beta, kappa, mu = (2, 2, 2, 4), 5.0, 0.12, 0.1
    U = synth.random_links(dims, 0.5, seed=231)
    P = synth.gaussian_momenta(dims, 232)
    eta = synth.gaussian_spinor(dims, seed=233) * _even(dims)[:, None, None]
    phi = ohmc.pseudofermion(dims, U, kappa, mu, eta)
    g = ctx.gauge(dims, U)
    m = ctx.mom(dims, P)
    f = ctx.field(dims, "f64", lqcd.FULL, data=phi)
    p = lqcd.hmc_params(beta=beta, kappa=kappa, mu=mu, tau=0.2, nsteps=2, ngauge=2, scheme=lqcd.LEAPFROG,
                        tol=1e-12)
    info = lqcd.hmc_trajectory(g, p, m, f, lqcd.solve_opts(sloppy_prec="f64"))
    want = mg.read(mg.HMC[0])
    assert abs(info["H0"] - want[0].real) < 1e-7 and abs(info["dH"] - want[1].real) < 1e-7, info
    assert np.abs(m.download()[0].ravel() - want[2:]).max() < 1e-8
