"""HMC for N_f = 2 (twisted-mass) Wilson fermions with even-odd preconditioning: actions,
forces and molecular-dynamics integrators (test infrastructure only).

The paper (Section 3) asks for an HMC with even-odd preconditioning, the 2MN integrator
and multiple integration timescales for N_f = 2 twisted-mass Wilson fermions; it writes
none of it down. Readings, stated here once:

  Actions     S_g = beta sum_P (1 - Re Tr U_P / 3);  S_f = phi^dag (Mhat^dag Mhat)^-1 phi on
              the even sites, Mhat = A - kappa^2 D_eo A^-1 D_oe (A = 1 + 2 i kappa mu g5;
              A = 1 for mu = 0). det M = det A_oo det Mhat and A_oo does not depend on U, so
              S_f carries the whole gauge dependence of det(M^dag M) for the doublet.
  Momenta     P_mu(x) traceless anti-Hermitian, kinetic energy -sum Tr(P^2) / 2.
  Gradient    G_mu(x) in su(3) with dS/de = -sum Tr(H G) for U -> exp(e H) U. For a term
              c Re Tr(U B) (B independent of U) that is G = -c TA(U B), with
              TA(M) = (M - M^dag)/2 - Tr(M - M^dag)/6.
              Gauge: G_g = (beta/3) TA(U W), W the staple sum.
              Fermion: with X = (Mhat^dag Mhat)^-1 phi and Y = Mhat X,
              dS_f = 2 kappa^2 Re[Psi^dag dD Phi], Phi = X_e + A^-1 D_oe X_e,
              Psi = Y_e + A^-dag (D^dag)_oe Y_e (D the hopping term, D^dag = g5 D g5), and the
              terms of D holding U_mu(x) give
              G_f = -2 kappa^2 eta TA(U [ ((1 - g_mu) Phi(x+mu))^T conj(Psi(x))
                                          + Psi(x+mu)^T conj((1 + g_mu) Phi(x)) ]),
              the products taken over spin, the 3 x 3 result indexed by colour, eta the
              t-boundary sign of the link.
  MD          dU/dt = P U, dP/dt = -G. Leapfrog; the second-order minimum-norm (2MN,
              Omelyan-Mryglod-Folk) integrator with lambda = 0.1931833275037836; a
              two-level nesting with the gauge force on the inner level (Sexton-Weingarten).
  Hamiltonian H = -sum Tr(P^2) / 2 + S_g + S_f.

Pins (tests/test_oracle_hmc.py): central finite differences of S_g and S_f along random
su(3) directions against sum -Tr(H G); gauge covariance of the forces; reversibility of
the integrators; dH ~ eps^2 for both second-order integrators.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import dense, gauge, wilson

LAMBDA_2MN = 0.1931833275037836


def ta(m):
    """Traceless anti-Hermitian part of [..., 3, 3] matrices."""
    a = 0.5 * (m - np.conj(np.swapaxes(m, -1, -2)))
    return a - (np.trace(a, axis1=-2, axis2=-1) / 3)[..., None, None] * np.eye(3)


def kinetic(P):
    """-sum Tr(P^2) / 2 = sum |P_ij|^2 / 2 for anti-Hermitian P."""
    return 0.5 * float(np.sum(np.abs(P) ** 2))


def expm_update(U, P, eps):
    """U_mu(x) <- exp(eps P_mu(x)) U_mu(x)."""
    return sla.expm(eps * P) @ U


# ------------------------------------------------------------ lattice helpers


def _grid(dims, a):
    lx, ly, lz, lt = dims
    return a.reshape((lt, lz, ly, lx) + a.shape[1:])


_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}  # direction mu -> axis of the (t, z, y, x) grid


def _fwd(a, mu):
    """a(x + mu) on the (t, z, y, x, ...) grid."""
    return np.roll(a, -1, axis=_AXIS[mu])


def _bwd(a, mu):
    return np.roll(a, 1, axis=_AXIS[mu])


def _dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def staples(dims, U):
    """W[V, 4, 3, 3]: sum_{nu != mu} U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    + U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu)."""
    G = _grid(dims, U)
    W = np.zeros_like(G)
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            Umu, Unu = G[..., mu, :, :], G[..., nu, :, :]
            W[..., mu, :, :] += _fwd(Unu, mu) @ _dag(_fwd(Umu, nu)) @ _dag(Unu)
            W[..., mu, :, :] += _dag(_bwd(_fwd(Unu, mu), nu)) @ _dag(_bwd(Umu, nu)) @ _bwd(Unu, nu)
    return W.reshape(U.shape)


def gauge_action(dims, U, beta):
    V = int(np.prod(dims))
    return beta * 6 * V * (1.0 - gauge.plaquette(dims, U))


def gauge_force(dims, U, beta):
    return (beta / 3.0) * ta(U @ staples(dims, U))


# ------------------------------------------------------------ fermions


def _g5(v):
    return v * np.array([1, 1, -1, -1])[None, :, None]


def twist(v, s, t):
    """s (1 + i t g5) v on spinors [V, 4, 3]."""
    return s * (v + 1j * t * _g5(v))


def solve_normal(dims, U, kappa, mu, phi, tol=1e-13, maxiter=20000, t_bc=-1):
    """X = (Mhat^dag Mhat)^-1 phi on the even sites: textbook CG, x0 = 0, stopping at
    |phi - Mhat^dag Mhat X| <= tol |phi|."""
    ev = (dense.parity_mask(dims) == 0)[:, None, None]
    phi = phi * ev
    A = lambda v: wilson.apply_Mhat(dims, U, kappa, wilson.apply_Mhat(dims, U, kappa, v, t_bc=t_bc, mu=mu),  # noqa: E731
                                    t_bc=t_bc, dagger=True, mu=mu)
    x = np.zeros_like(phi)
    r = phi.copy()
    p = r.copy()
    rr = np.vdot(r, r).real
    stop = tol * tol * np.vdot(phi, phi).real
    for it in range(maxiter):
        if rr <= stop:
            return x, it
        q = A(p)
        alpha = rr / np.vdot(p, q).real
        x = x + alpha * p
        r = r - alpha * q
        rr_new = np.vdot(r, r).real
        p = r + (rr_new / rr) * p
        rr = rr_new
    raise RuntimeError("solve_normal: no convergence")


def fermion_fields(dims, U, kappa, mu, X, t_bc=-1):
    """(Phi, Psi, Y): Phi = X_e + A^-1 D_oe X_e, Psi = Y_e + A^-dag (D^dag)_oe Y_e, Y = Mhat X."""
    a = 2.0 * kappa * mu
    s = 1.0 / (1.0 + a * a)
    Y = wilson.apply_Mhat(dims, U, kappa, X, t_bc=t_bc, mu=mu)
    Xo = twist(wilson.hop_eo(dims, U, X, 1, t_bc=t_bc), s, -a)
    Yo = twist(wilson.hop_eo(dims, U, Y, 1, t_bc=t_bc, dagger=True), s, a)
    return X + Xo, Y + Yo, Y


def fermion_action(dims, U, kappa, mu, phi, t_bc=-1, tol=1e-13):
    X, _ = solve_normal(dims, U, kappa, mu, phi, tol=tol, t_bc=t_bc)
    return float(np.vdot(phi, X).real)


def fermion_force_from_X(dims, U, kappa, mu, X, t_bc=-1):
    """G_f for the solution X = (Mhat^dag Mhat)^-1 phi (see the module text)."""
    g, _ = dense.gammas()
    Phi, Psi, _ = fermion_fields(dims, U, kappa, mu, X, t_bc=t_bc)
    Gphi, Gpsi = _grid(dims, Phi), _grid(dims, Psi)
    GU = _grid(dims, U)
    lt = dims[3]
    F = np.zeros_like(GU)
    one = np.eye(4)
    for m in range(4):
        fwd_phi = _fwd(Gphi, m)                   # Phi(x + mu)   [..., 4, 3]
        fwd_psi = _fwd(Gpsi, m)
        v1 = np.einsum("st,...tc->...sc", one - g[m], fwd_phi)   # (1 - g_mu) Phi(x+mu)
        v2 = np.einsum("st,...tc->...sc", one + g[m], Gphi)      # (1 + g_mu) Phi(x)
        B = np.einsum("...sb,...sa->...ba", v1, np.conj(Gpsi)) + np.einsum("...sa,...sb->...ab", fwd_psi,
                                                                             np.conj(v2))
        eta = np.ones(GU.shape[:4])
        if m == 3:
            eta[lt - 1] = t_bc  # the t link from t = Lt - 1 crosses the boundary
        F[..., m, :, :] = -2.0 * kappa * kappa * eta[..., None, None] * ta(GU[..., m, :, :] @ B)
    return F.reshape(U.shape)


def fermion_force(dims, U, kappa, mu, phi, t_bc=-1, tol=1e-13):
    X, _ = solve_normal(dims, U, kappa, mu, phi, tol=tol, t_bc=t_bc)
    return fermion_force_from_X(dims, U, kappa, mu, X, t_bc=t_bc)


def pseudofermion(dims, U, kappa, mu, eta, t_bc=-1):
    """phi = Mhat^dag eta (even sites): S_f = |eta|^2 at the start of a trajectory."""
    ev = (dense.parity_mask(dims) == 0)[:, None, None]
    return wilson.apply_Mhat(dims, U, kappa, eta * ev, t_bc=t_bc, dagger=True, mu=mu)


# ------------------------------------------------------------ molecular dynamics


def hamiltonian(dims, U, P, phi, beta, kappa, mu, t_bc=-1):
    return kinetic(P) + gauge_action(dims, U, beta) + fermion_action(dims, U, kappa, mu, phi, t_bc=t_bc)


def integrate(dims, U, P, phi, beta, kappa, mu, tau, nsteps, scheme="2mn", ngauge=1, t_bc=-1):
    """One MD trajectory of length tau in nsteps outer steps; the gauge force runs ngauge
    inner steps per outer step (same scheme). Returns (U, P)."""
    eps = tau / nsteps

    def f_ferm(U):
        return fermion_force(dims, U, kappa, mu, phi, t_bc=t_bc)

    def f_gauge(U):
        return gauge_force(dims, U, beta)

    def inner(U, P, h):
        """Gauge level of length h: ngauge steps of the scheme with exact link updates."""
        e = h / ngauge
        for _ in range(ngauge):
            if scheme == "leapfrog":
                P = P - 0.5 * e * f_gauge(U)
                U = expm_update(U, P, e)
                P = P - 0.5 * e * f_gauge(U)
            else:
                P = P - LAMBDA_2MN * e * f_gauge(U)
                U = expm_update(U, P, 0.5 * e)
                P = P - (1 - 2 * LAMBDA_2MN) * e * f_gauge(U)
                U = expm_update(U, P, 0.5 * e)
                P = P - LAMBDA_2MN * e * f_gauge(U)
        return U, P

    for _ in range(nsteps):
        if scheme == "leapfrog":
            P = P - 0.5 * eps * f_ferm(U)
            U, P = inner(U, P, eps)
            P = P - 0.5 * eps * f_ferm(U)
        else:
            P = P - LAMBDA_2MN * eps * f_ferm(U)
            U, P = inner(U, P, 0.5 * eps)
            P = P - (1 - 2 * LAMBDA_2MN) * eps * f_ferm(U)
            U, P = inner(U, P, 0.5 * eps)
            P = P - LAMBDA_2MN * eps * f_ferm(U)
    return U, P
