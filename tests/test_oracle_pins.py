"""Pins of the FP64 oracle to facts outside itself (CPU only).

The paper (Section 3) names the even-odd Wilson "dslash" and the fermion-matrix
inversion but prints no worked example, so every pin here is mathematical:
closed-form free-field spectrum and solution, gamma5-hermiticity, adjointness,
gauge covariance, a dense brute-force matrix, dense LAPACK solves and the
Schur-complement identity. Each pin targets a class of plausible mistakes
(named in its docstring).
"""
import numpy as np
import pytest

import oracle
from oracle import dense
from paper_1112_5280_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _vdot(a, b):
    return np.vdot(a.reshape(-1), b.reshape(-1))


def _g5(psi):
    out = psi.copy()
    out[:, 2:, :] *= -1
    return out


# ---------------------------------------------------------------- gamma algebra

def test_gamma_algebra():
    """Clifford algebra, hermiticity and g5 = g1 g2 g3 g4 = diag(1,1,-1,-1) (chiral basis)."""
    g, g5 = dense.gammas()
    for mu in range(4):
        assert np.allclose(g[mu], g[mu].conj().T)
        for nu in range(4):
            anti = g[mu] @ g[nu] + g[nu] @ g[mu]
            assert np.allclose(anti, 2 * (mu == nu) * np.eye(4))
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


# ---------------------------------------------------------------- free field

def test_constant_field_periodic():
    """U = 1, all-periodic, constant psi: D psi = sum_mu [(1-g)+(1+g)] psi = 8 psi.
    Catches a dropped hop or a wrong relative sign between forward and backward terms."""
    dims = (4, 2, 6, 4)
    U = synth.unit_links(dims)
    chi = synth.gaussian_spinor((1, 1, 1, 1), seed=5)[0]
    psi = np.broadcast_to(chi, (synth.volume(dims), 4, 3)).copy()
    out = oracle.hop(dims, U, psi, t_bc=+1)
    assert np.abs(out - 8 * psi).max() < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 8), (6, 4, 2, 6)])
def test_free_plane_wave_eigenvectors(dims):
    """At U = 1 a plane wave exp(ipx) chi, with chi an eigenvector of sum g_mu sin p_mu, is
    an eigenvector of M with eigenvalue 1 - 2k sum cos p +- 2ik |sin p| (antiperiodic t:
    p_t = (2 pi n + pi)/L_t). Catches wrong gamma matrices, hop directions and t signs."""
    kappa = 0.13
    U = synth.unit_links(dims)
    g, _ = dense.gammas()
    rng = np.random.default_rng(7)
    for _ in range(6):
        n = [int(rng.integers(0, L)) for L in dims]
        _, p = synth.plane_wave(dims, n, np.zeros((4, 3)))
        s = sum(np.sin(p[mu]) * g[mu] for mu in range(4))
        w, vecs = np.linalg.eigh(s)
        for k in (0, 3):
            chi = np.outer(vecs[:, k], rng.standard_normal(3) + 1j * rng.standard_normal(3))
            psi, _ = synth.plane_wave(dims, n, chi)
            lam = 1 - 2 * kappa * np.sum(np.cos(p)) + 2j * kappa * w[k]
            out = oracle.apply_M(dims, U, kappa, psi)
            assert np.abs(out - lam * psi).max() < 1e-13


def test_free_spectrum_dense():
    """Eigenvalues of M assembled from oracle applications to unit vectors on 2x2x2x4 equal
    the closed-form free spectrum (each 6-fold)."""
    dims = (2, 2, 2, 4)
    kappa = 0.12
    U = synth.unit_links(dims)
    V = synth.volume(dims)
    M = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    for j in range(12 * V):
        e = np.zeros(12 * V, dtype=np.complex128)
        e[j] = 1
        M[:, j] = oracle.apply_M(dims, U, kappa, e.reshape(V, 4, 3)).reshape(-1)
    ev = np.linalg.eigvals(M)
    ref = dense.free_eigenvalues(dims, kappa)
    key = lambda a: np.lexsort((np.round(a.imag, 9), np.round(a.real, 9)))  # noqa: E731
    assert np.abs(ev[key(ev)] - ref[key(ref)]).max() < 1e-12


# ---------------------------------------------------------------- structure with random links

@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 6), (2, 2, 2, 2)])
def test_gamma5_hermiticity(dims):
    """<phi, M psi> = <g5 M g5 phi, psi>. Catches a wrong link dagger/placement on the backward
    hop or a projector sign that breaks the g5 structure."""
    U = synth.random_links(dims, 0.3, seed=11)
    phi = synth.gaussian_spinor(dims, seed=12)
    psi = synth.gaussian_spinor(dims, seed=13)
    kappa = 0.12
    lhs = _vdot(phi, oracle.apply_M(dims, U, kappa, psi))
    rhs = _vdot(_g5(oracle.apply_M(dims, U, kappa, _g5(phi))), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 6)])
def test_dagger_is_adjoint(dims):
    """<phi, M psi> = <M^dag phi, psi> and M^dag = g5 M g5 (the dagger path flips the projectors)."""
    U = synth.random_links(dims, 0.5, seed=21)
    phi = synth.gaussian_spinor(dims, seed=22)
    psi = synth.gaussian_spinor(dims, seed=23)
    kappa = 0.15
    lhs = _vdot(phi, oracle.apply_M(dims, U, kappa, psi))
    rhs = _vdot(oracle.apply_M(dims, U, kappa, phi, dagger=True), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    md = oracle.apply_M(dims, U, kappa, phi, dagger=True)
    assert np.abs(md - _g5(oracle.apply_M(dims, U, kappa, _g5(phi)))).max() < 1e-13


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_gauge_covariance(dims):
    """M[U^g](g psi) = g M[U] psi with U'_mu(x) = g(x) U_mu(x) g(x+mu)^dag. Catches a link on
    the wrong site, a missing dagger or a transposed link product."""
    U = synth.random_links(dims, 0.5, seed=31)
    g = synth.gauge_transform_field(dims, seed=32)
    psi = synth.gaussian_spinor(dims, seed=33)
    kappa = 0.14
    Ug = dense.gauge_transform_links(dims, U, g)
    lhs = oracle.apply_M(dims, Ug, kappa, dense.gauge_transform_spinor(g, psi))
    rhs = dense.gauge_transform_spinor(g, oracle.apply_M(dims, U, kappa, psi))
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max() * 10


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4), (2, 4, 2, 2)])
def test_dense_brute_force(dims):
    """The matrix assembled from oracle applications equals the dense matrix built block by
    block in pure Python (independent gamma construction, independent indexing); L = 2
    directions exercise coinciding forward and backward neighbours."""
    U = synth.random_links(dims, 0.3, seed=41)
    kappa = 0.12
    V = synth.volume(dims)
    M = dense.dense_wilson(dims, U, kappa)
    Mo = np.zeros_like(M)
    for j in range(12 * V):
        e = np.zeros(12 * V, dtype=np.complex128)
        e[j] = 1
        Mo[:, j] = oracle.apply_M(dims, U, kappa, e.reshape(V, 4, 3)).reshape(-1)
    assert np.abs(M - Mo).max() < 1e-15


# ---------------------------------------------------------------- even-odd

def test_eo_blocks_and_schur():
    """hop_eo(p) equals the parity-p rows of the full hop applied to the parity-(1-p) part, and
    Mhat = 1 - k^2 D_eo D_oe equals the Schur complement M_ee - M_eo M_oo^-1 M_oe of the dense M."""
    dims = (2, 2, 2, 4)
    U = synth.random_links(dims, 0.5, seed=51)
    psi = synth.gaussian_spinor(dims, seed=52)
    kappa = 0.15
    par = synth.parity_of_sites(dims)
    for p in (0, 1):
        masked = psi * (par == 1 - p)[:, None, None]
        full = oracle.hop(dims, U, masked) * (par == p)[:, None, None]
        assert np.abs(oracle.hop_eo(dims, U, psi, p) - full).max() < 1e-15
    M = dense.dense_wilson(dims, U, kappa)
    e = np.repeat(par == 0, 12)
    o = ~e
    schur = M[np.ix_(e, e)] - M[np.ix_(e, o)] @ np.linalg.solve(M[np.ix_(o, o)], M[np.ix_(o, e)])
    psi_e = psi * (par == 0)[:, None, None]
    out = oracle.apply_Mhat(dims, U, kappa, psi_e)
    assert np.abs(out.reshape(-1)[e] - schur @ psi_e.reshape(-1)[e]).max() < 1e-13
    assert np.abs(out.reshape(-1)[o]).max() == 0.0
    outd = oracle.apply_Mhat(dims, U, kappa, psi_e, dagger=True)
    assert np.abs(outd.reshape(-1)[e] - schur.conj().T @ psi_e.reshape(-1)[e]).max() < 1e-13


# ---------------------------------------------------------------- solvers

@pytest.mark.parametrize("method", [oracle.METHOD_CG_FULL, oracle.METHOD_CG_EO,
                                    oracle.METHOD_BICGSTAB_EO])
def test_solvers_vs_lapack_4x4x4x4(method):
    """4^4, kappa = 0.12, eps = 0.3 (the small workload): every solver reaches ||b - Mx|| <= 1e-10
    ||b|| and agrees with numpy.linalg.solve on the dense M."""
    dims = (4, 4, 4, 4)
    U = synth.random_links(dims, 0.3)
    b = synth.gaussian_spinor(dims)
    kappa = 0.12
    x, status, iters, res = oracle.solve(dims, U, kappa, b, tol=1e-10, method=method)
    assert status == 0 and res <= 1e-10 and iters > 0
    M = dense.dense_wilson(dims, U, kappa)
    xd = np.linalg.solve(M, b.reshape(-1)).reshape(x.shape)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


def test_solve_free_field_fft():
    """At U = 1 the EO CG solution equals the exact Fourier solution (8^3 x 16, kappa = 0.124)."""
    dims = (8, 8, 8, 16)
    U = synth.unit_links(dims)
    b = synth.gaussian_spinor(dims, seed=61)
    kappa = 0.124
    x, status, iters, res = oracle.solve(dims, U, kappa, b, tol=1e-11, method=oracle.METHOD_CG_EO)
    assert status == 0 and res <= 1e-11
    xf = dense.free_solve_fft(dims, kappa, b)
    assert np.linalg.norm(x - xf) / np.linalg.norm(xf) < 1e-9


def test_solve_gauge_covariance():
    """M[U^g]^-1 (g b) = g M[U]^-1 b."""
    dims = (4, 4, 2, 6)
    U = synth.random_links(dims, 0.5, seed=71)
    g = synth.gauge_transform_field(dims, seed=72)
    b = synth.gaussian_spinor(dims, seed=73)
    kappa = 0.13
    x, st, _, _ = oracle.solve(dims, U, kappa, b, tol=1e-12)
    xg, st2, _, _ = oracle.solve(dims, dense.gauge_transform_links(dims, U, g), kappa,
                                 dense.gauge_transform_spinor(g, b), tol=1e-12)
    assert st == 0 and st2 == 0
    ref = dense.gauge_transform_spinor(g, x)
    assert np.linalg.norm(xg - ref) / np.linalg.norm(ref) < 1e-10


def test_cg_and_bicgstab_agree():
    dims = (6, 4, 4, 6)
    U = synth.random_links(dims, 0.5, seed=81)
    b = synth.gaussian_spinor(dims, seed=82)
    kappa = 0.15
    x1, s1, _, r1 = oracle.solve(dims, U, kappa, b, tol=1e-11, method=oracle.METHOD_CG_EO)
    x2, s2, _, r2 = oracle.solve(dims, U, kappa, b, tol=1e-11, method=oracle.METHOD_BICGSTAB_EO)
    assert s1 == 0 and s2 == 0 and r1 <= 1e-11 and r2 <= 1e-11
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x1) < 1e-9


def test_hop_sites_matches_full():
    dims = (4, 6, 4, 8)
    U = synth.random_links(dims, 0.8, seed=91)
    psi = synth.gaussian_spinor(dims, seed=92)
    full = oracle.hop(dims, U, psi)
    sites = np.array([0, 5, 17, synth.volume(dims) - 1, 333])
    for dag in (False, True):
        fd = oracle.hop(dims, U, psi, dagger=dag)
        assert np.abs(oracle.hop_sites(dims, U, psi, sites, dagger=dag) - fd[sites]).max() == 0.0
    assert np.abs(full[sites] - oracle.hop_sites(dims, U, psi, sites)).max() == 0.0


# ---------------------------------------------------------------- inputs

def test_link_generator_is_su3_and_twelve_real_exact():
    """Generated links are unitary with det 1, so row 2 = conj(row0 x row1): the identity the
    12-real (RECONSTRUCT TWELVE, Section 3) storage relies on."""
    dims = (4, 4, 4, 8)
    for eps in (0.3, 0.5, 0.8):
        U = synth.random_links(dims, eps, seed=101).reshape(-1, 3, 3)
        assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
        assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - np.eye(3)).max() < 1e-14
        r2 = np.conj(np.cross(U[:, 0, :], U[:, 1, :]))
        assert np.abs(r2 - U[:, 2, :]).max() < 1e-15


# ---------------------------------------------------------------- twisted mass (Section 3: N_f = 2)

@pytest.mark.parametrize("mu", [0.05, 0.4])
def test_tm_gamma5_hermiticity_flips_mu(mu):
    """M(mu)^dag = g5 M(-mu) g5 for M = 1 - k D + 2 i k mu g5, and the dagger path is the adjoint."""
    dims = (4, 4, 2, 4)
    U = synth.random_links(dims, 0.5, seed=201)
    phi = synth.gaussian_spinor(dims, seed=202)
    psi = synth.gaussian_spinor(dims, seed=203)
    kappa = 0.14
    lhs = _vdot(phi, oracle.apply_M(dims, U, kappa, psi, mu=mu))
    rhs = _vdot(_g5(oracle.apply_M(dims, U, kappa, _g5(phi), mu=-mu)), psi)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    rhs2 = _vdot(oracle.apply_M(dims, U, kappa, phi, mu=mu, dagger=True), psi)
    assert abs(lhs - rhs2) < 1e-12 * abs(lhs)


def test_tm_free_spectrum():
    """At U = 1 the twisted operator has eigenvalues 1 - 2k sum cos p +- 2ik sqrt(sum sin^2 p + mu^2)."""
    dims = (2, 2, 2, 4)
    kappa, mu = 0.12, 0.3
    V = synth.volume(dims)
    U = synth.unit_links(dims)
    M = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    for j in range(12 * V):
        e = np.zeros(12 * V, dtype=np.complex128)
        e[j] = 1
        M[:, j] = oracle.apply_M(dims, U, kappa, e.reshape(V, 4, 3), mu=mu).reshape(-1)
    ev = np.linalg.eigvals(M)
    ref = dense.free_eigenvalues(dims, kappa, mu=mu)
    key = lambda a: np.lexsort((np.round(a.imag, 9), np.round(a.real, 9)))  # noqa: E731
    assert np.abs(ev[key(ev)] - ref[key(ref)]).max() < 1e-12


def test_tm_dense_and_schur():
    dims = (2, 2, 2, 4)
    U = synth.random_links(dims, 0.5, seed=204)
    kappa, mu = 0.15, 0.2
    V = synth.volume(dims)
    M = dense.dense_wilson(dims, U, kappa, mu=mu)
    cols = []
    for j in range(12 * V):
        e = np.zeros(12 * V, dtype=np.complex128)
        e[j] = 1
        cols.append(oracle.apply_M(dims, U, kappa, e.reshape(V, 4, 3), mu=mu).reshape(-1))
    assert np.abs(M - np.stack(cols, axis=1)).max() < 1e-15
    par = synth.parity_of_sites(dims)
    ev = np.repeat(par == 0, 12)
    od = ~ev
    schur = M[np.ix_(ev, ev)] - M[np.ix_(ev, od)] @ np.linalg.solve(M[np.ix_(od, od)], M[np.ix_(od, ev)])
    psi = synth.gaussian_spinor(dims, seed=205) * (par == 0)[:, None, None]
    out = oracle.apply_Mhat(dims, U, kappa, psi, mu=mu)
    assert np.abs(out.reshape(-1)[ev] - schur @ psi.reshape(-1)[ev]).max() < 1e-13
    outd = oracle.apply_Mhat(dims, U, kappa, psi, mu=mu, dagger=True)
    assert np.abs(outd.reshape(-1)[ev] - schur.conj().T @ psi.reshape(-1)[ev]).max() < 1e-13


@pytest.mark.parametrize("method", [oracle.METHOD_CG_FULL, oracle.METHOD_CG_EO,
                                    oracle.METHOD_BICGSTAB_EO])
def test_tm_solvers_vs_lapack(method):
    dims = (4, 4, 2, 4)
    U = synth.random_links(dims, 0.4, seed=206)
    b = synth.gaussian_spinor(dims, seed=207)
    kappa, mu = 0.15, 0.1
    x, status, _, res = oracle.solve(dims, U, kappa, b, tol=1e-11, method=method, mu=mu)
    assert status == 0 and res <= 1e-11
    xd = np.linalg.solve(dense.dense_wilson(dims, U, kappa, mu=mu), b.reshape(-1)).reshape(x.shape)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9


# ---------------------------------------------------------------- true residual (the solves' arbiter)

@pytest.mark.parametrize("dims,t_bc,mu", [((2, 2, 2, 2), -1, 0.0), ((2, 2, 2, 4), -1, 0.0),
                                          ((2, 2, 2, 4), 1, 0.0), ((2, 2, 2, 4), -1, 0.3),
                                          ((2, 2, 2, 2), 1, -0.2)])
def test_true_residual_against_dense(dims, t_bc, mu):
    """oracle.true_residual is the arbiter of every GPU solve, so it is pinned on its own:
    ||b - M x|| / ||b|| with M the dense matrix built block by block (dense.py), for a random
    x where the value is O(1) (Wilson and twisted, both t boundaries). x = 0 gives 1,
    the LAPACK solution gives rounding level, and the value is invariant under a common
    scale of b and x (x = 0 gives 1 up to the rounding of the norm's OpenMP reduction,
    whose order may differ between the two sums). Catches Mhat in place of M, the dagger operator, a dropped square
    root, a wrong denominator and a wrong sign in b - M x."""
    U = synth.random_links(dims, 0.5, seed=301)
    b = synth.gaussian_spinor(dims, seed=302)
    x = 0.7 * synth.gaussian_spinor(dims, seed=303)
    kappa = 0.13
    M = dense.dense_wilson(dims, U, kappa, t_bc=t_bc, mu=mu)
    ref = np.linalg.norm(b.reshape(-1) - M @ x.reshape(-1)) / np.linalg.norm(b.reshape(-1))
    assert 0.3 < ref < 10.0
    got = oracle.true_residual(dims, U, kappa, b, x, t_bc=t_bc, mu=mu)
    assert abs(got - ref) <= 1e-13 * ref, (got, ref)
    assert abs(oracle.true_residual(dims, U, kappa, b, np.zeros_like(b), t_bc=t_bc, mu=mu) - 1.0) <= 1e-15
    xd = np.linalg.solve(M, b.reshape(-1)).reshape(b.shape)
    assert oracle.true_residual(dims, U, kappa, b, xd, t_bc=t_bc, mu=mu) < 1e-13
    got2 = oracle.true_residual(dims, U, kappa, 2.5 * b, 2.5 * x, t_bc=t_bc, mu=mu)
    assert abs(got2 - got) <= 1e-14 * got


def test_true_residual_of_perturbed_solution():
    """x = x* + e with x* the exact solution: the residual is |M e| / |b| for any e, so it
    grows linearly in the size of e (checked at e ~ 1e-4 and 1e-7 of |x*|, against the dense
    matrix). This is the regime the GPU tests read (residuals near 1e-10)."""
    dims = (2, 2, 2, 4)
    U = synth.random_links(dims, 0.5, seed=311)
    b = synth.gaussian_spinor(dims, seed=312)
    kappa = 0.14
    M = dense.dense_wilson(dims, U, kappa)
    xs = np.linalg.solve(M, b.reshape(-1))
    e = synth.gaussian_spinor(dims, seed=313).reshape(-1)
    for scale in (1e-4, 1e-7):
        ee = e * scale * np.linalg.norm(xs) / np.linalg.norm(e)
        ref = np.linalg.norm(M @ ee) / np.linalg.norm(b.reshape(-1))
        got = oracle.true_residual(dims, U, kappa, b, (xs + ee).reshape(b.shape))
        assert abs(got - ref) <= 1e-6 * ref, (scale, got, ref)
