"""Pins of the oracle's meson contraction (paper Section 4, eq. 4.1), CPU only.

- gauge invariance of C_Gamma(t) for every Gamma (catches colour-index errors);
- Gamma = g5 reduces to the Frobenius norm: sum_t C_g5(t) = - sum over the 12
  solutions of |x|^2 (catches a missing dagger, a sign or a transposed S);
- free field: C_g5(t0 + tau) = C_g5(t0 - tau) (time reflection of the free action);
- the matrix form equals an explicit loop over spin and colour indices on 2^4.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import contract, dense
from paper_1112_5280_gb300 import synth

CODES = list(range(10))


def _solutions(dims, U, kappa, site, tol=1e-12):
    sols = []
    for s in range(4):
        for c in range(3):
            x, st, _, _ = oracle.solve(dims, U, kappa, synth.point_source(dims, site, s, c), tol=tol)
            assert st == 0
            sols.append(x)
    return sols


def test_gauge_invariance():
    dims = (4, 4, 2, 6)
    U = synth.random_links(dims, 0.5, seed=5)
    g = synth.gauge_transform_field(dims, seed=6)
    site = 37
    c1 = contract.meson_correlator(dims, _solutions(dims, U, 0.13, site), CODES)
    c2 = contract.meson_correlator(dims, _solutions(dims, dense.gauge_transform_links(dims, U, g), 0.13, site),
                                   CODES)
    assert np.abs(c1 - c2).max() < 1e-9 * np.abs(c1).max()


def test_g5_is_frobenius_norm():
    dims = (4, 2, 4, 4)
    U = synth.random_links(dims, 0.5, seed=7)
    sols = _solutions(dims, U, 0.14, 9)
    c = contract.meson_correlator(dims, sols, [1])[0]
    assert abs(c.sum() + sum(np.vdot(x, x).real for x in sols)) < 1e-12 * abs(c.sum())
    assert np.all(c.real < 0) and np.abs(c.imag).max() < 1e-12 * np.abs(c.real).max()


def test_free_field_time_reflection():
    dims = (4, 4, 4, 8)
    kappa = 0.12
    site = synth.site_index(dims, 1, 2, 3, 2)
    t0 = 2
    sols = [dense.free_solve_fft(dims, kappa, synth.point_source(dims, site, s, c))
            for s in range(4) for c in range(3)]
    c = contract.meson_correlator(dims, sols, [1])[0].real
    lt = dims[3]
    for tau in range(1, lt // 2):
        assert abs(c[(t0 + tau) % lt] - c[(t0 - tau) % lt]) < 1e-10 * abs(c).max()


@pytest.mark.parametrize("code", CODES)
def test_matrix_form_equals_index_loops(code):
    dims = (2, 2, 2, 2)
    V = synth.volume(dims)
    rng = np.random.default_rng(code)
    sols = [rng.standard_normal((V, 4, 3)) + 1j * rng.standard_normal((V, 4, 3)) for _ in range(12)]
    G = contract.gamma_matrix(code)
    g5 = contract.gamma_matrix(1)
    A, B = g5 @ G, G @ g5
    ref = np.zeros(V, dtype=np.complex128)
    for x in range(V):
        tot = 0.0
        for be, b, al, a, al2, be2 in itertools.product(range(4), range(3), range(4), range(3),
                                                        range(4), range(4)):
            s_dag = np.conj(sols[3 * be + b][x, al, a])
            tot += s_dag * A[al, al2] * sols[3 * be2 + b][x, al2, a] * B[be2, be]
        ref[x] = -tot
    assert np.abs(contract.meson_correlator_sites(sols, code) - ref).max() < 1e-12 * np.abs(ref).max()
