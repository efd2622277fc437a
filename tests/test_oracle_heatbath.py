"""Pins of the heatbath oracle (CPU only): each check compares the oracle with something
other than itself, so that a plausible mistake (a dropped 1/3 in beta, a transposed or
daggered staple, a wrong subgroup block, a missing rotation by v, a wrong acceptance)
fails at least one of them; the planted mutants at the end confirm that.

  * Philox4x64-10 against numpy's independent Philox bit generator.
  * The SU(2) draw against its exact density exp(alpha b0) sqrt(1 - b0^2) on [-1, 1]
    (moments by quadrature, Kolmogorov-Smirnov) and a uniform direction.
  * One link in equilibrium with fixed neighbours: the chain average of Re Tr(U W)/3
    against a brute-force Haar-measure integral, W written out here from the definition.
  * beta = 0 gives Haar links: <Re Tr U> = 0, <|Tr U|^2> = 1 for SU(3).
  * Strong coupling: <P> = beta/18 + beta^2/216 + O(beta^4), from the SU(3) Haar moments
    <(Re Tr U)^2> = 1/2, <(Re Tr U)^3> = 1/4, <(Re Tr U)^4> = 3/4 (the beta^3 term cancels).
  * The staple against the plaquette: sum_{x,mu} Re Tr(U W) = 4 sum_P Re Tr U_P; the
    plaquette of unit links is 1 and gauge invariant; links stay in SU(3).
"""
import os
import subprocess

import numpy as np
import pytest
from scipy import integrate, special, stats

from oracle import build as obuild
from oracle import dense, gauge, wilson
from paper_1112_5280_gb300 import synth

# ------------------------------------------------------------ Philox


def test_philox_matches_numpy():
    rng = np.random.default_rng(5)
    for _ in range(20):
        ctr = [int(x) for x in rng.integers(0, 2**63, 4, dtype=np.int64)]
        ctr[0] = max(ctr[0], 1)
        key = [int(x) for x in rng.integers(0, 2**63, 2, dtype=np.int64)]
        # numpy's Philox advances the counter before each block: counter - 1 gives block `ctr`
        prev = list(ctr)
        prev[0] -= 1
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
        assert gauge.philox4x64(ctr, key) == [int(x) for x in bg.random_raw(4)]


# ------------------------------------------------------------ SU(2) draw


def _density_moments(alpha):
    f = lambda x, k: x**k * np.sqrt(1 - x * x) * np.exp(alpha * (x - 1))  # noqa: E731
    z = integrate.quad(f, -1, 1, args=(0,), epsabs=0, epsrel=1e-12)[0]
    return [integrate.quad(f, -1, 1, args=(k,), epsabs=0, epsrel=1e-12)[0] / z for k in (1, 2)]


@pytest.mark.parametrize("alpha", [0.0, 0.7, 3.0, 12.0])
def test_su2_draw_distribution(alpha):
    n = 200_000
    b, fails = gauge.su2_draws(alpha, seed=11, n=n)
    assert fails == 0
    assert np.abs(np.sum(b * b, axis=1) - 1).max() < 1e-14
    m1, m2 = _density_moments(alpha)
    if alpha > 0:  # closed form of the mean: I2(alpha) / I1(alpha)
        assert abs(m1 - special.iv(2, alpha) / special.iv(1, alpha)) < 1e-9
    b0 = b[:, 0]
    sd = np.sqrt(m2 - m1 * m1)
    assert abs(b0.mean() - m1) < 5 * sd / np.sqrt(n)
    assert abs((b0 * b0).mean() - m2) < 5 * np.sqrt(np.var(b0 * b0) / n)

    def cdf(x):
        f = lambda t: np.sqrt(1 - t * t) * np.exp(alpha * (t - 1))  # noqa: E731
        z = integrate.quad(f, -1, 1, limit=200)[0]
        return np.array([integrate.quad(f, -1, xi)[0] / z for xi in np.atleast_1d(x)])

    sub = np.sort(b0[:4000])
    assert stats.kstest(sub, cdf).pvalue > 1e-3
    # direction uniform on the 2-sphere of radius sqrt(1 - b0^2)
    vec = b[:, 1:]
    for k in range(3):
        assert abs(vec[:, k].mean()) < 5 * np.sqrt((1 - m2) / 3 / n)
        assert abs((vec[:, k] ** 2).mean() - (1 - m2) / 3) < 5 * np.sqrt(np.var(vec[:, k] ** 2) / n)


# ------------------------------------------------------------ single link in equilibrium


def _link(U, dims, c, mu):
    return U[synth.site_index(dims, *c), mu]


def _staple_by_definition(U, dims, c, mu):
    """W = sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+ + U_nu(x+mu-nu)^+ U_mu(x-nu)^+ U_nu(x-nu)."""
    def sh(cc, m, d):
        cc = list(cc)
        cc[m] = (cc[m] + d) % dims[m]
        return cc
    H = lambda a: a.conj().T  # noqa: E731
    W = np.zeros((3, 3), dtype=np.complex128)
    for nu in range(4):
        if nu == mu:
            continue
        W += _link(U, dims, sh(c, mu, 1), nu) @ H(_link(U, dims, sh(c, nu, 1), mu)) @ H(_link(U, dims, c, nu))
        W += (H(_link(U, dims, sh(sh(c, mu, 1), nu, -1), nu)) @ H(_link(U, dims, sh(c, nu, -1), mu))
              @ _link(U, dims, sh(c, nu, -1), nu))
    return W


def _haar_su3(n, rng):
    z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=1, axis2=2)
    q = q * (d / np.abs(d))[:, None, :]  # Haar on U(3)
    root = np.linalg.det(q) ** (1 / 3) * np.exp(2j * np.pi * rng.integers(0, 3, n) / 3)
    return q / root[:, None, None]  # a uniformly chosen cube root of det: Haar on SU(3)


def test_haar_sampler_of_this_test():
    s = _haar_su3(200_000, np.random.default_rng(1))
    t = np.trace(s, axis1=1, axis2=2)
    assert np.abs(np.linalg.det(s) - 1).max() < 1e-12
    assert abs(np.mean(np.abs(t) ** 2) - 1) < 0.02 and abs(np.mean(t)) < 0.01
    assert abs(np.mean(t ** 3) - 1) < 0.05  # the SU(3) (not U(3)) invariant


@pytest.mark.parametrize("beta,mu", [(1.0, 1), (2.5, 3)])
def test_single_link_equilibrium(beta, mu):
    dims = (2, 2, 2, 4)
    U = np.ascontiguousarray(synth.random_links(dims, 0.8, seed=21))
    c = (1, 0, 1, 2)
    s = synth.site_index(dims, *c)
    W = _staple_by_definition(U, dims, c, mu)
    assert np.abs(gauge.staple(dims, U, s, mu) - W).max() < 1e-13
    f = []
    for sweep in range(6000):
        assert gauge.heatbath_link(dims, U, beta, 77, sweep, s, mu) == 0
        f.append(np.real(np.trace(U[s, mu] @ W)) / 3)
    f = np.array(f[200:])
    nb = 40  # batch means for the autocorrelated chain
    bm = f[: len(f) // nb * nb].reshape(nb, -1).mean(axis=1)
    chain, chain_err = bm.mean(), bm.std(ddof=1) / np.sqrt(nb)
    h = _haar_su3(400_000, np.random.default_rng(3))
    g = np.real(np.einsum("nij,ji->n", h, W)) / 3
    w = np.exp(beta * (g - g.max()))
    exact = np.sum(w * g) / np.sum(w)
    exact_err = np.sqrt(np.sum(w * w * (g - exact) ** 2)) / np.sum(w)
    assert abs(chain - exact) < 5 * np.hypot(chain_err, exact_err), (chain, exact, chain_err, exact_err)


# ------------------------------------------------------------ whole-lattice pins


def test_beta_zero_gives_haar_links():
    dims = (4, 4, 4, 4)
    U, fails = gauge.heatbath(dims, synth.unit_links(dims), 0.0, seed=5, nsweeps=1)
    assert fails == 0
    t = np.trace(U, axis1=2, axis2=3).reshape(-1)
    n = t.size
    assert abs(np.mean(t.real)) < 4 * np.sqrt(0.5 / n)
    assert abs(np.mean(np.abs(t) ** 2) - 1) < 4 * np.sqrt(1.0 / n)


def test_strong_coupling_plaquette():
    dims = (8, 8, 8, 8)
    beta = 0.5
    U, _ = gauge.heatbath(dims, synth.unit_links(dims), beta, seed=9, nsweeps=5)
    p = []
    for k in range(40):
        U, fails = gauge.heatbath(dims, U, beta, seed=9, sweep0=5 + k, nsweeps=1)
        assert fails == 0
        p.append(gauge.plaquette(dims, U))
    p = np.array(p)
    expect = beta / 18 + beta**2 / 216
    assert abs(p.mean() - expect) < 4 * p.std(ddof=1) / np.sqrt(len(p)) + 2e-5, (p.mean(), expect)


def test_staple_sum_equals_four_plaquettes():
    dims = (4, 2, 4, 2)
    U = synth.random_links(dims, 0.9, seed=31)
    V = synth.volume(dims)
    tot = sum(np.real(np.trace(U[s, mu] @ gauge.staple(dims, U, s, mu))) for s in range(V) for mu in range(4))
    assert abs(tot - 4 * 18 * V * gauge.plaquette(dims, U)) < 1e-10 * abs(tot)


def test_plaquette_unit_and_gauge_invariant():
    dims = (4, 4, 2, 6)
    assert abs(gauge.plaquette(dims, synth.unit_links(dims)) - 1) < 1e-15
    U = synth.random_links(dims, 0.7, seed=41)
    gt = synth.gauge_transform_field(dims, seed=42)
    p0 = gauge.plaquette(dims, U)
    assert abs(gauge.plaquette(dims, dense.gauge_transform_links(dims, U, gt)) - p0) < 1e-13


@pytest.mark.parametrize("reunit", [True, False])
def test_links_stay_su3(reunit):
    dims = (4, 4, 4, 4)
    U, _ = gauge.heatbath(dims, synth.random_links(dims, 0.5, seed=51), 5.7, seed=3, nsweeps=3,
                          reunit=reunit)
    eye = np.eye(3)
    assert np.abs(np.einsum("smji,smjk->smik", U.conj(), U) - eye).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13


def test_reunitarise_fixes_drift():
    dims = (2, 2, 2, 2)
    U = synth.random_links(dims, 0.5, seed=61)
    U2 = gauge.reunitarise(dims, U * (1 + 1e-6))
    assert np.abs(U2 - U).max() < 1e-12


# ------------------------------------------------------------ planted mistakes

HB_SRC = os.path.join(os.path.dirname(obuild.__file__), "heatbath.c")
MUTANTS = {
    "beta_without_third": ("beta * kk / 3.0", "beta * kk"),
    # (a = v b would be no mistake: Haar measure is bi-invariant and a.v = b0 either way)
    "missing_v_rotation": ("B[r * 2 + 0] * Vm[0 * 2 + q] + B[r * 2 + 1] * Vm[1 * 2 + q]",
                           "B[r * 2 + q] + 0.0 * Vm[0]"),
    "subgroup_c1_sign": ("c[1] = -cimag(x01 + x10);", "c[1] = cimag(x01 + x10);"),
    "no_acceptance": ("if (u1 * u1 <= s2) {", "if (s2 >= 0.0) {"),
    "upper_staple_undaggered": ("mul_nd(link(U, sp, nu), link(U, spn, mu), T);",
                                "mul_nn(link(U, sp, nu), link(U, spn, mu), T);"),
    "lower_staple_wrong_site": ("mul_dn(A, link(U, smn, nu), T2);", "mul_dn(A, link(U, s, nu), T2);"),
}


def _fast_pins():
    out = {}
    try:
        test_single_link_equilibrium(1.0, 1)
        out["single_link"] = True
    except AssertionError:
        out["single_link"] = False
    try:
        test_su2_draw_distribution(3.0)
        out["su2"] = True
    except AssertionError:
        out["su2"] = False
    return out


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_heatbath_mutant_is_caught(name, tmp_path):
    src = open(HB_SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, old
    (tmp_path / "heatbath.c").write_text(src.replace(old, new))
    hdir = os.path.dirname(HB_SRC)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", f"-I{hdir}", "-o", str(so),
                    os.path.join(hdir, "wilson_oracle.c"), str(tmp_path / "heatbath.c"), "-lm"], check=True)
    saved_lib, saved_ready = wilson._lib, gauge._ready
    real_build = obuild.build
    wilson._lib, gauge._ready = None, False
    obuild.build = lambda force=False: str(so)
    try:
        res = _fast_pins()
    finally:
        obuild.build = real_build
        wilson._lib, gauge._ready = saved_lib, saved_ready
    assert not all(res.values()), f"mutant {name} passed: {res}"
