"""Pins of the HMC oracle (CPU only).

  * Forces against central finite differences of the actions: for U -> exp(e H) U with H a
    random su(3) field, (S(+h) - S(-h)) / 2h equals -sum Tr(H G) (gauge and fermion, Wilson
    and twisted mass, both boundary conditions). The difference is independent of the
    force formula, so a wrong sign, factor, boundary sign, shift or dagger fails.
  * Gauge covariance: G[U^g] = g G[U] g^dag (the fermion field transformed with it).
  * The integrators: reversibility (forward, flip P, forward again returns (U, -P)) and
    second order (dH shrinks ~4x when the step halves).
  * Planted mistakes in a copy of hmc.py are caught by the finite-difference pin.
"""
import types

import numpy as np
import pytest

from oracle import dense, hmc
from paper_1112_5280_gb300 import synth

DIMS = (4, 2, 2, 4)


def _direction(dims, seed):
    return synth.gaussian_momenta(dims, seed)


def _fd(action, U, H, h=2e-4):
    """Central difference with one Richardson step (error O(h^4))."""
    def cd(e):
        return (action(hmc.expm_update(U, H, e)) - action(hmc.expm_update(U, H, -e))) / (2 * e)
    return (4 * cd(h / 2) - cd(h)) / 3


def _pairing(H, G):
    return float(np.sum(np.conj(H) * G).real)  # -Tr(H G) summed, for anti-Hermitian H, G


def test_momenta_are_su3_algebra():
    P = synth.gaussian_momenta(DIMS, 1)
    assert np.abs(P + np.conj(np.swapaxes(P, -1, -2))).max() < 1e-15
    assert np.abs(np.trace(P, axis1=-2, axis2=-1)).max() < 1e-14
    big = synth.gaussian_momenta((8, 8, 8, 8), 2)
    # density exp(-sum|P_ij|^2/2) on the 8 real dimensions of su(3): <sum|P_ij|^2> = 8 per link
    assert abs(np.mean(np.sum(np.abs(big) ** 2, axis=(-2, -1))) - 8) < 0.1


@pytest.mark.parametrize("beta", [5.5, 1.0])
def test_gauge_force_is_gradient(beta):
    U = synth.random_links(DIMS, 0.6, seed=3)
    H = _direction(DIMS, 4)
    fd = _fd(lambda u: hmc.gauge_action(DIMS, u, beta), U, H)
    an = _pairing(H, hmc.gauge_force(DIMS, U, beta))
    assert abs(fd - an) < 1e-7 * max(1.0, abs(an)), (fd, an)


@pytest.mark.parametrize("mu", [0.0, 0.25])
@pytest.mark.parametrize("t_bc", [-1, 1])
def test_fermion_force_is_gradient(mu, t_bc):
    kappa = 0.13
    U = synth.random_links(DIMS, 0.6, seed=5)
    eta = synth.gaussian_spinor(DIMS, seed=6)
    phi = hmc.pseudofermion(DIMS, U, kappa, mu, eta, t_bc=t_bc)
    H = _direction(DIMS, 7)
    fd = _fd(lambda u: hmc.fermion_action(DIMS, u, kappa, mu, phi, t_bc=t_bc, tol=1e-14), U, H)
    an = _pairing(H, hmc.fermion_force(DIMS, U, kappa, mu, phi, t_bc=t_bc, tol=1e-14))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (fd, an)


def test_fermion_action_at_start_is_eta_norm():
    """phi = Mhat^dag eta gives S_f = |eta_e|^2 (checks the solve and the pseudofermion)."""
    kappa, mu = 0.14, 0.1
    U = synth.random_links(DIMS, 0.6, seed=8)
    eta = synth.gaussian_spinor(DIMS, seed=9) * (dense.parity_mask(DIMS) == 0)[:, None, None]
    phi = hmc.pseudofermion(DIMS, U, kappa, mu, eta)
    assert abs(hmc.fermion_action(DIMS, U, kappa, mu, phi) - np.vdot(eta, eta).real) < 1e-9


def test_forces_gauge_covariant():
    kappa, mu, beta = 0.13, 0.2, 5.0
    U = synth.random_links(DIMS, 0.6, seed=10)
    g = synth.gauge_transform_field(DIMS, seed=11)
    Ug = dense.gauge_transform_links(DIMS, U, g)
    rot = lambda F: np.einsum("sab,smbc,sdc->smad", g, F, np.conj(g))  # noqa: E731
    assert np.abs(hmc.gauge_force(DIMS, Ug, beta) - rot(hmc.gauge_force(DIMS, U, beta))).max() < 1e-12
    phi = hmc.pseudofermion(DIMS, U, kappa, mu, synth.gaussian_spinor(DIMS, seed=12))
    F = hmc.fermion_force(DIMS, U, kappa, mu, phi)
    Fg = hmc.fermion_force(DIMS, Ug, kappa, mu, dense.gauge_transform_spinor(g, phi))
    assert np.abs(Fg - rot(F)).max() < 1e-10


@pytest.mark.parametrize("scheme", ["leapfrog", "2mn"])
def test_integrator_reversible(scheme):
    beta, kappa, mu = 5.0, 0.12, 0.1
    U = synth.random_links(DIMS, 0.5, seed=13)
    P = synth.gaussian_momenta(DIMS, 14)
    phi = hmc.pseudofermion(DIMS, U, kappa, mu, synth.gaussian_spinor(DIMS, seed=15))
    U1, P1 = hmc.integrate(DIMS, U, P, phi, beta, kappa, mu, 0.3, 3, scheme=scheme, ngauge=2)
    U2, P2 = hmc.integrate(DIMS, U1, -P1, phi, beta, kappa, mu, 0.3, 3, scheme=scheme, ngauge=2)
    assert np.abs(U2 - U).max() < 1e-10 and np.abs(P2 + P).max() < 1e-10


@pytest.mark.parametrize("scheme", ["leapfrog", "2mn"])
def test_integrator_second_order(scheme):
    beta, kappa, mu = 5.0, 0.12, 0.1
    U = synth.random_links(DIMS, 0.5, seed=16)
    P = synth.gaussian_momenta(DIMS, 17)
    phi = hmc.pseudofermion(DIMS, U, kappa, mu, synth.gaussian_spinor(DIMS, seed=18))
    H0 = hmc.hamiltonian(DIMS, U, P, phi, beta, kappa, mu)
    dh = []
    for n in (4, 8):
        U1, P1 = hmc.integrate(DIMS, U, P, phi, beta, kappa, mu, 0.5, n, scheme=scheme)
        dh.append(abs(hmc.hamiltonian(DIMS, U1, P1, phi, beta, kappa, mu) - H0))
    assert 3.0 < dh[0] / dh[1] < 5.5, dh


# ------------------------------------------------------------ planted mistakes

MUTANTS = {
    "boundary_sign_dropped": ("eta[lt - 1] = t_bc", "eta[lt - 1] = 1"),
    "factor_two_dropped": ("-2.0 * kappa * kappa * eta", "-1.0 * kappa * kappa * eta"),
    "backward_term_at_x": ('np.einsum("...sa,...sb->...ab", fwd_psi,', 'np.einsum("...sa,...sb->...ab", Gpsi,'),
    "projector_sign": ("one - g[m], fwd_phi", "one + g[m], fwd_phi"),
    "odd_field_untwisted": ("Xo = twist(wilson.hop_eo(dims, U, X, 1, t_bc=t_bc), s, -a)",
                            "Xo = wilson.hop_eo(dims, U, X, 1, t_bc=t_bc)"),
    "gauge_force_sign": ("return (beta / 3.0) * ta(", "return -(beta / 3.0) * ta("),
}


def _mutant_module(name):
    src = open(hmc.__file__).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, old
    mod = types.ModuleType("hmc_mutant", None)
    mod.__dict__["__package__"] = "oracle"
    exec(compile(src.replace(old, new), "hmc_mutant.py", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_hmc_mutant_is_caught(name):
    m = _mutant_module(name)
    kappa, mu, beta, t_bc = 0.13, 0.25, 5.0, -1
    U = synth.random_links(DIMS, 0.6, seed=5)
    phi = m.pseudofermion(DIMS, U, kappa, mu, synth.gaussian_spinor(DIMS, seed=6), t_bc=t_bc)
    H = _direction(DIMS, 7)
    fd_f = _fd(lambda u: m.fermion_action(DIMS, u, kappa, mu, phi, t_bc=t_bc, tol=1e-14), U, H)
    an_f = _pairing(H, m.fermion_force(DIMS, U, kappa, mu, phi, t_bc=t_bc, tol=1e-14))
    fd_g = _fd(lambda u: m.gauge_action(DIMS, u, beta), U, H)
    an_g = _pairing(H, m.gauge_force(DIMS, U, beta))
    ok = abs(fd_f - an_f) < 1e-6 * max(1, abs(an_f)) and abs(fd_g - an_g) < 1e-7 * max(1, abs(an_g))
    assert not ok, name
