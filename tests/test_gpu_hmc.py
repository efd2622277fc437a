"""GPU HMC pieces against the FP64 oracle (paper Section 3: HMC with even-odd
preconditioning and the 2MN integrator for N_f = 2 twisted-mass Wilson fermions).

Bars:
  * the normal-equation solve meets its tolerance on the oracle's operator, and agrees
    with the oracle's CG within cond * tol (1e-8 here);
  * forces computed from the same solution X: 1e-12 of max|G| (FP64 both sides, the
    same arithmetic up to summation order);
  * gauge force 1e-12 (staples in double-float, unit roundoff 2^-48 = 3.6e-15);
    exp(eps P) U (2^s * 10 + 4) u per link, u = 2^-48, s the number of squarings (the
    Taylor stage and the product with U leave a few u, each squaring doubles the error);
    kinetic energy 1e-13 relative;
  * a short trajectory: links and momenta within 1e-8 of the oracle's (the force solves
    stop at 1e-12, so the forces differ by ~1e-10 and the trajectory inherits that),
    dH within 1e-7; reversibility on the GPU within 1e-8.
"""
import numpy as np
import pytest

from oracle import hmc as ohmc
from paper_1112_5280_gb300 import lqcd, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = lqcd.Context(0)
    yield c
    c.close()


def _even(dims):
    return (synth.parity_of_sites(dims) == 0)[:, None, None]


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 6)])
@pytest.mark.parametrize("mu", [0.0, 0.15])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_solve_normal_matches_oracle(ctx, dims, mu, prec):
    kappa = 0.14
    U = synth.random_links(dims, 0.6, seed=201)
    phi = synth.gaussian_spinor(dims, seed=202) * _even(dims)
    g = ctx.gauge(dims, U)
    src = ctx.field(dims, "f64", lqcd.FULL, data=phi)
    x = ctx.field(dims, "f64", lqcd.FULL)
    info = lqcd.solve_normal(g, src, kappa, 1e-12, x, lqcd.solve_opts(sloppy_prec=prec, mu=mu))
    assert info["status"] == 0 and info["true_resid"] <= 1e-12, info
    X = x.download()
    assert np.abs(X[~_even(dims)[:, 0, 0]]).max() == 0.0
    Xo, _ = ohmc.solve_normal(dims, U, kappa, mu, phi, tol=1e-14)
    assert np.linalg.norm(X - Xo) / np.linalg.norm(Xo) < 1e-8


@pytest.mark.parametrize("mu", [0.0, 0.2])
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_fermion_force_matches_oracle(ctx, mu, t_bc):
    dims, kappa = (4, 4, 2, 6), 0.13
    U = synth.random_links(dims, 0.6, seed=211)
    phi = synth.gaussian_spinor(dims, seed=212) * _even(dims)
    g = ctx.gauge(dims, U, t_bc=t_bc)
    X, _ = ohmc.solve_normal(dims, U, kappa, mu, phi, tol=1e-14, t_bc=t_bc)
    x = ctx.field(dims, "f64", lqcd.FULL, data=X)
    m = ctx.mom(dims)
    sf = lqcd.fermion_force(g, kappa, mu, x, 1.0, m)
    ref = ohmc.fermion_force_from_X(dims, U, kappa, mu, X, t_bc=t_bc)
    got = m.download()
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()
    assert abs(sf - np.vdot(phi, X).real) < 1e-10 * abs(sf)
    # accumulation: coeff scales and adds
    lqcd.fermion_force(g, kappa, mu, x, -0.5, m)
    assert np.abs(m.download() - 0.5 * ref).max() < 1e-12 * np.abs(ref).max()


def _expm_bar(P, eps):
    """Per-link bar for exp(eps P) U in double-float (unit roundoff u = 2^-48): the Taylor
    stage and the product with U each leave a few u; each of the s squarings (|eps P|_F
    halved s times to reach 1/2) doubles the relative error and adds one product's
    rounding, so the bound is (2^s * 10 + 4) u."""
    nrm = eps * np.sqrt((np.abs(P) ** 2).sum(axis=(-1, -2)))
    s = np.maximum(0, np.ceil(np.log2(np.maximum(nrm, 1e-300) / 0.5)))
    return (2.0 ** s * 10 + 4) * 2.0 ** -48


def test_gauge_force_update_kinetic(ctx):
    dims, beta = (6, 4, 4, 4), 5.7
    U = synth.random_links(dims, 0.7, seed=221)
    g = ctx.gauge(dims, U)
    m = ctx.mom(dims)
    lqcd.gauge_force(g, beta, 2.0, m)
    ref = 2.0 * ohmc.gauge_force(dims, U, beta)
    assert np.abs(m.download() - ref).max() < 1e-12 * np.abs(ref).max()
    P = synth.gaussian_momenta(dims, 222)
    m.upload(P)
    assert np.array_equal(m.download(), P)
    assert abs(m.kinetic() - ohmc.kinetic(P)) < 1e-13 * ohmc.kinetic(P)
    for eps in (0.05, 0.7):  # 0.7 |P| > 1/2: exercises the scaling and squaring
        g2 = ctx.gauge(dims, U)
        lqcd.gauge_update(g2, m, eps)
        err = np.abs(g2.download() - ohmc.expm_update(U, P, eps)).max(axis=(-1, -2))
        assert (err <= _expm_bar(P, eps)).all(), (err / _expm_bar(P, eps)).max()


@pytest.mark.parametrize("scheme", [lqcd.LEAPFROG, lqcd.TWO_MN])
def test_trajectory_matches_oracle(ctx, scheme):
    dims, beta, kappa, mu = (4, 4, 4, 4), 5.0, 0.12, 0.1
    U = synth.random_links(dims, 0.5, seed=231)
    P = synth.gaussian_momenta(dims, 232)
    eta = synth.gaussian_spinor(dims, seed=233) * _even(dims)
    phi = ohmc.pseudofermion(dims, U, kappa, mu, eta)
    g = ctx.gauge(dims, U)
    m = ctx.mom(dims, P)
    f = ctx.field(dims, "f64", lqcd.FULL, data=phi)
    p = lqcd.hmc_params(beta=beta, kappa=kappa, mu=mu, tau=0.2, nsteps=2, ngauge=2, scheme=scheme, tol=1e-12)
    info = lqcd.hmc_trajectory(g, p, m, f, lqcd.solve_opts(sloppy_prec="f64"))
    name = "leapfrog" if scheme == lqcd.LEAPFROG else "2mn"
    U1, P1 = ohmc.integrate(dims, U, P, phi, beta, kappa, mu, 0.2, 2, scheme=name, ngauge=2)
    assert np.abs(g.download() - U1).max() < 1e-8
    assert np.abs(m.download() - P1).max() < 1e-8
    H0 = ohmc.hamiltonian(dims, U, P, phi, beta, kappa, mu)
    H1 = ohmc.hamiltonian(dims, U1, P1, phi, beta, kappa, mu)
    assert abs(info["H0"] - H0) < 1e-7 and abs(info["dH"] - (H1 - H0)) < 1e-7, (info, H0, H1)
    assert abs(info["fermion0"] - np.vdot(eta, eta).real) < 1e-8
    assert info["force_evals"] == (3 if scheme == lqcd.LEAPFROG else 5)
    assert info["accepted"] == 1


def test_trajectory_reversible_and_metropolis(ctx):
    dims, beta, kappa, mu = (4, 4, 4, 4), 5.5, 0.13, 0.05
    U = synth.random_links(dims, 0.4, seed=241)
    P = synth.gaussian_momenta(dims, 242)
    phi = ohmc.pseudofermion(dims, U, kappa, mu, synth.gaussian_spinor(dims, seed=243) * _even(dims))
    g = ctx.gauge(dims, U)
    m = ctx.mom(dims, P)
    f = ctx.field(dims, "f64", lqcd.FULL, data=phi)
    opts = lqcd.solve_opts(sloppy_prec="f32")
    p = lqcd.hmc_params(beta=beta, kappa=kappa, mu=mu, tau=0.3, nsteps=3, ngauge=3, tol=1e-12)
    i1 = lqcd.hmc_trajectory(g, p, m, f, opts)
    m.upload(-m.download())
    i2 = lqcd.hmc_trajectory(g, p, m, f, opts)
    assert np.abs(g.download() - U).max() < 1e-8 and np.abs(m.download() + P).max() < 1e-8
    assert abs(i1["dH"] + i2["dH"]) < 1e-6
    # Metropolis: accept_u = 1 accepts only dH <= 0; a rejection restores the links
    g2 = ctx.gauge(dims, U)
    m.upload(P)
    p.accept_u = 1.0
    i3 = lqcd.hmc_trajectory(g2, p, m, f, opts)
    assert i3["accepted"] == (1 if i3["dH"] <= 0 else 0)
    if not i3["accepted"]:
        assert np.array_equal(g2.download(), U)


@pytest.mark.parametrize("chrono", [1, 2])
def test_chronological_guess_keeps_the_trajectory(ctx, chrono):
    """Force solves that start from the last solution (chrono 1) or from its linear
    extrapolation (chrono 2) still converge to the same tolerance, so the trajectory matches
    the oracle's to the same 1e-8 as the solves from zero, and dH to 1e-7; the solves take
    fewer iterations in total."""
    dims, beta, kappa, mu = (4, 4, 4, 4), 5.0, 0.12, 0.1
    U = synth.random_links(dims, 0.5, seed=251)
    P = synth.gaussian_momenta(dims, 252)
    phi = ohmc.pseudofermion(dims, U, kappa, mu, synth.gaussian_spinor(dims, seed=253) * _even(dims))
    U1, P1 = ohmc.integrate(dims, U, P, phi, beta, kappa, mu, 0.4, 4, scheme="2mn", ngauge=2)
    H0 = ohmc.hamiltonian(dims, U, P, phi, beta, kappa, mu)
    H1 = ohmc.hamiltonian(dims, U1, P1, phi, beta, kappa, mu)
    iters = {}
    for ch in (0, chrono):
        g = ctx.gauge(dims, U)
        m = ctx.mom(dims, P)
        f = ctx.field(dims, "f64", lqcd.FULL, data=phi)
        p = lqcd.hmc_params(beta=beta, kappa=kappa, mu=mu, tau=0.4, nsteps=4, ngauge=2,
                            scheme=lqcd.TWO_MN, tol=1e-12, chrono=ch)
        info = lqcd.hmc_trajectory(g, p, m, f, lqcd.solve_opts(sloppy_prec="f32"))
        assert np.abs(g.download() - U1).max() < 1e-8, ch
        assert np.abs(m.download() - P1).max() < 1e-8, ch
        assert abs(info["dH"] - (H1 - H0)) < 1e-7, (ch, info["dH"], H1 - H0)
        iters[ch] = info["solver_iters"]
        assert info["force_evals"] == 9
        for o in (g, m, f):
            o.close()
    assert iters[chrono] < iters[0], iters


def test_bad_hmc_arguments(ctx):
    dims = (2, 2, 2, 2)
    g = ctx.gauge(dims, synth.unit_links(dims))
    m = ctx.mom(dims)
    f = ctx.field(dims, "f64", lqcd.FULL)
    for kw in ({"nsteps": 0}, {"ngauge": 0}, {"tau": -1.0}, {"scheme": 7}, {"tol": 0.0}, {"chrono": 3}):
        with pytest.raises(lqcd.LqcdError):
            lqcd.hmc_trajectory(g, lqcd.hmc_params(**kw), m, f)
    with pytest.raises(lqcd.LqcdError):
        lqcd.hmc_trajectory(g, lqcd.hmc_params(), m, ctx.field(dims, "f32", lqcd.FULL))


def test_engine_mixes_normal_and_plain_requests(ctx):
    """Normal-equation and M x = b requests (Wilson and twisted) share one engine, each on its
    own reliable-update path, and each result equals its solo solve bit for bit."""
    opts = lqcd.solve_opts(sloppy_prec="f32")
    eng = lqcd.Engine(ctx, opts, max_slots=8)
    dims = (6, 4, 4, 6)
    U = synth.random_links(dims, 0.5, seed=251)
    g = ctx.gauge(dims, U)
    ev = _even(dims)
    cases = [(True, 0.0, 252), (False, 0.0, 253), (True, 0.1, 254), (False, 0.1, 255)]
    items = []
    for normal, mu, seed in cases:
        b = synth.gaussian_spinor(dims, seed=seed)
        if normal:
            b = b * ev
        src = ctx.field(dims, "f64", lqcd.FULL, data=b)
        items.append((eng.submit(g, src, 0.14, 1e-11, mu=mu, normal=normal), normal, mu, b, src))
    while eng.step() > 0:
        pass
    for rid, normal, mu, b, src in items:
        x = ctx.field(dims, "f64", lqcd.FULL)
        info = eng.result(rid, x)
        assert info["status"] == 0, (normal, mu, info)
        xm = x.download()
        solo = ctx.field(dims, "f64", lqcd.FULL)
        o = lqcd.solve_opts(sloppy_prec="f32", mu=mu)
        if normal:
            lqcd.solve_normal(g, src, 0.14, 1e-11, solo, o)
            Xo, _ = ohmc.solve_normal(dims, U, 0.14, mu, b, tol=1e-14)
            assert np.linalg.norm(xm - Xo) / np.linalg.norm(Xo) < 1e-7
        else:
            lqcd.solve_fields(g, src, 0.14, 1e-11, solo, o)
        assert np.array_equal(solo.download(), xm), (normal, mu)
    eng.close()
