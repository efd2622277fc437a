"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of the C oracle (a textual patch of
oracle/wilson_oracle.c compiled into a temporary directory), loads it in
place of the real oracle and runs the pin checks: at least one must fail.
The real oracle must pass all of them.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle
from oracle import build as obuild
from oracle import dense, wilson
from paper_1112_5280_gb300 import synth

SRC = os.path.join(os.path.dirname(obuild.__file__), "wilson_oracle.c")

MUTANTS = {
    "backward_link_not_daggered": ("conj(link[b * 3 + a])", "link[a * 3 + b]"),
    "forward_link_transposed": ("(dir == 0) ? link[a * 3 + b]", "(dir == 0) ? link[b * 3 + a]"),
    "projector_sign_swapped": ("(dir == 0) ? -sgn : sgn", "(dir == 0) ? sgn : -sgn"),
    "t_boundary_sign_dropped": ("if (mu == 3 && c[3] == g->L[3] - 1) eta = (double)t_bc;",
                                "if (mu == 3 && c[3] == g->L[3] - 1) eta = 1.0;"),
    "backward_link_on_wrong_site": ("link = U + (index_of(g, n) * 4 + mu) * 9;",
                                    "link = U + (s * 4 + mu) * 9;"),
    "dropped_backward_z_hop": ("for (int dir = 0; dir < 2; ++dir)",
                               "for (int dir = 0; dir < 2 - (mu == 2); ++dir)"),
    "gamma_lower_block_sign": ("GAMMA[k][2 + a][b] = I * sig[k][a][b];",
                               "GAMMA[k][2 + a][b] = -I * sig[k][a][b];"),
    "kappa_sign_in_M": ("o[i] = p[i] - kappa * o[i] +", "o[i] = p[i] + kappa * o[i] +"),
    "schur_sign": ("apsi[s * 12 + k] - kappa * kappa * o[s * 12 + k]",
                   "apsi[s * 12 + k] + kappa * kappa * o[s * 12 + k]"),
    "bhat_sign": ("bhat[s * 12 + k] = parity_of(cc) == 0 ? bb[s * 12 + k] + kappa * tmp[s * 12 + k]",
                  "bhat[s * 12 + k] = parity_of(cc) == 0 ? bb[s * 12 + k] - kappa * tmp[s * 12 + k]"),
    "odd_reconstruction_sign": ("tmp[s * 12 + k] = parity_of(cc) == 1 ? bb[s * 12 + k] + kappa * tmp",
                                "tmp[s * 12 + k] = parity_of(cc) == 1 ? bb[s * 12 + k] - kappa * tmp"),
    "twisted_term_sign": ("+ I * tm * g5_sign(sp) * p[i]", "- I * tm * g5_sign(sp) * p[i]"),
    "twisted_term_no_g5": ("+ I * tm * g5_sign(sp) * p[i]", "+ I * tm * p[i]"),
    "schur_inverse_twist_sign": ("twist(&g, 1.0 / (1.0 + a * a), -a, tmp, tmp2, 1);",
                                 "twist(&g, 1.0 / (1.0 + a * a), a, tmp, tmp2, 1);"),
    "odd_reconstruction_missing_inverse": ("    twist(&g, 1.0 / (1.0 + a * a), -a, tmp, tmp, 1);",
                                           "    twist(&g, 1.0, 0.0, tmp, tmp, 1);"),
    "t_neighbour_off_by_one": ("n[mu] = (c[mu] + 1) % g->L[mu];",
                               "n[mu] = (c[mu] + 1 + (mu == 3)) % g->L[mu];"),
    # the true residual ||b - M x|| / ||b||, the arbiter of every GPU solve
    "true_residual_uses_Mhat": ("oracle_apply_M(dims, t_bc, U, kappa, mu, x, (double*)y, 0);",
                                "oracle_apply_Mhat(dims, t_bc, U, kappa, mu, x, (double*)y, 0);"),
    "true_residual_uses_dagger": ("oracle_apply_M(dims, t_bc, U, kappa, mu, x, (double*)y, 0);",
                                  "oracle_apply_M(dims, t_bc, U, kappa, mu, x, (double*)y, 1);"),
    "true_residual_no_sqrt": ("double res = sqrt(vnorm2(y, n)) / sqrt(vnorm2(bb, n));",
                              "double res = vnorm2(y, n) / sqrt(vnorm2(bb, n));"),
    "true_residual_wrong_denominator": ("double res = sqrt(vnorm2(y, n)) / sqrt(vnorm2(bb, n));",
                                        "double res = sqrt(vnorm2(y, n)) / sqrt(vnorm2((const cplx*)x, n));"),
    "true_residual_sign": ("y[i] = bb[i] - y[i];", "y[i] = bb[i] + y[i];"),
}


def _pin_checks():
    """Each returns True when the pin holds."""
    checks = {}

    def plane_wave():
        dims, kappa = (4, 4, 2, 6), 0.13
        U = synth.unit_links(dims)
        g, _ = dense.gammas()
        n = (1, 2, 1, 4)
        _, p = synth.plane_wave(dims, n, np.zeros((4, 3)))
        w, vecs = np.linalg.eigh(sum(np.sin(p[m]) * g[m] for m in range(4)))
        ok = True
        for k in (0, 3):
            chi = np.outer(vecs[:, k], [1.0, 0.5j, -0.25])
            psi, _ = synth.plane_wave(dims, n, chi)
            lam = 1 - 2 * kappa * np.sum(np.cos(p)) + 2j * kappa * w[k]
            ok &= np.abs(oracle.apply_M(dims, U, kappa, psi) - lam * psi).max() < 1e-12
        return bool(ok)

    def hermiticity():
        dims = (4, 2, 4, 4)
        U = synth.random_links(dims, 0.5, seed=1)
        phi, psi = synth.gaussian_spinor(dims, 2), synth.gaussian_spinor(dims, 3)
        g5 = lambda v: v * np.array([1, 1, -1, -1])[None, :, None]  # noqa: E731
        lhs = np.vdot(phi, oracle.apply_M(dims, U, 0.12, psi))
        rhs = np.vdot(g5(oracle.apply_M(dims, U, 0.12, g5(phi))), psi)
        return bool(abs(lhs - rhs) < 1e-12 * abs(lhs))

    def covariance():
        dims = (4, 2, 2, 4)
        U = synth.random_links(dims, 0.5, seed=4)
        g = synth.gauge_transform_field(dims, 5)
        psi = synth.gaussian_spinor(dims, 6)
        lhs = oracle.apply_M(dims, dense.gauge_transform_links(dims, U, g), 0.14,
                             dense.gauge_transform_spinor(g, psi))
        rhs = dense.gauge_transform_spinor(g, oracle.apply_M(dims, U, 0.14, psi))
        return bool(np.abs(lhs - rhs).max() < 1e-12)

    def brute_force():
        dims = (2, 2, 2, 4)
        U = synth.random_links(dims, 0.3, seed=7)
        V = synth.volume(dims)
        M = dense.dense_wilson(dims, U, 0.12)
        cols = []
        for j in range(12 * V):
            e = np.zeros(12 * V, dtype=np.complex128)
            e[j] = 1
            cols.append(oracle.apply_M(dims, U, 0.12, e.reshape(V, 4, 3)).reshape(-1))
        return bool(np.abs(M - np.stack(cols, axis=1)).max() < 1e-14)

    def eo_solve_vs_lapack():
        dims = (2, 2, 2, 4)
        U = synth.random_links(dims, 0.3, seed=8)
        b = synth.gaussian_spinor(dims, 9)
        x, st, _, _ = oracle.solve(dims, U, 0.12, b, tol=1e-11, maxiter=500,
                                   method=oracle.METHOD_CG_EO)
        xd = np.linalg.solve(dense.dense_wilson(dims, U, 0.12), b.reshape(-1))
        return bool(st == 0 and np.linalg.norm(x.reshape(-1) - xd) < 1e-9 * np.linalg.norm(xd))

    def tm_hermiticity():
        dims = (4, 2, 2, 4)
        U = synth.random_links(dims, 0.5, seed=10)
        phi, psi = synth.gaussian_spinor(dims, 11), synth.gaussian_spinor(dims, 12)
        g5 = lambda v: v * np.array([1, 1, -1, -1])[None, :, None]  # noqa: E731
        lhs = np.vdot(phi, oracle.apply_M(dims, U, 0.13, psi, mu=0.3))
        rhs = np.vdot(g5(oracle.apply_M(dims, U, 0.13, g5(phi), mu=-0.3)), psi)
        return bool(abs(lhs - rhs) < 1e-12 * abs(lhs))

    def tm_solve_vs_lapack():
        dims = (2, 2, 2, 4)
        U = synth.random_links(dims, 0.3, seed=13)
        b = synth.gaussian_spinor(dims, 14)
        ok = True
        for method in (oracle.METHOD_CG_EO, oracle.METHOD_BICGSTAB_EO):
            x, st, _, _ = oracle.solve(dims, U, 0.14, b, tol=1e-11, maxiter=500, method=method, mu=0.4)
            xd = np.linalg.solve(dense.dense_wilson(dims, U, 0.14, mu=0.4), b.reshape(-1))
            ok &= st == 0 and np.linalg.norm(x.reshape(-1) - xd) < 1e-9 * np.linalg.norm(xd)
        return bool(ok)

    def tm_brute_force():
        dims = (2, 2, 2, 2)
        U = synth.random_links(dims, 0.3, seed=15)
        V = synth.volume(dims)
        M = dense.dense_wilson(dims, U, 0.12, mu=0.25)
        cols = []
        for j in range(12 * V):
            e = np.zeros(12 * V, dtype=np.complex128)
            e[j] = 1
            cols.append(oracle.apply_M(dims, U, 0.12, e.reshape(V, 4, 3), mu=0.25).reshape(-1))
        return bool(np.abs(M - np.stack(cols, axis=1)).max() < 1e-14)

    def true_residual_dense():
        ok = True
        for dims, mu in (((2, 2, 2, 4), 0.0), ((2, 2, 2, 2), 0.3)):
            U = synth.random_links(dims, 0.5, seed=16)
            b, x = synth.gaussian_spinor(dims, 17), 0.7 * synth.gaussian_spinor(dims, 18)
            M = dense.dense_wilson(dims, U, 0.13, mu=mu)
            ref = np.linalg.norm(b.reshape(-1) - M @ x.reshape(-1)) / np.linalg.norm(b.reshape(-1))
            ok &= abs(oracle.true_residual(dims, U, 0.13, b, x, mu=mu) - ref) <= 1e-13 * ref
        return bool(ok)

    checks.update(plane_wave=plane_wave, true_residual_dense=true_residual_dense, hermiticity=hermiticity, covariance=covariance,
                  brute_force=brute_force, eo_solve_vs_lapack=eo_solve_vs_lapack,
                  tm_hermiticity=tm_hermiticity, tm_solve_vs_lapack=tm_solve_vs_lapack,
                  tm_brute_force=tm_brute_force)
    return checks


def _run_checks():
    out = {}
    for name, fn in _pin_checks().items():
        try:
            out[name] = fn()
        except Exception:
            out[name] = False
    return out


def _load_mutant(tmp_path, patch):
    src = open(SRC).read()
    old, new = patch
    assert src.count(old) >= 1, f"mutation anchor not found: {old}"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new, 1))
    hdr = os.path.join(os.path.dirname(SRC), "wilson_oracle.h")
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-std=c11", "-O1", "-fopenmp", "-fPIC", "-shared", f"-I{os.path.dirname(hdr)}",
                    "-o", str(so), str(mut), "-lm"], check=True)
    return str(so)


def _with_lib(path):
    saved = wilson._lib
    wilson._lib = None
    real_build = obuild.build
    obuild.build = lambda force=False: path
    try:
        wilson._load()
        return _run_checks()
    finally:
        obuild.build = real_build
        wilson._lib = saved


def test_real_oracle_passes_all_pins():
    res = _run_checks()
    assert all(res.values()), res


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    path = _load_mutant(tmp_path, MUTANTS[name])
    res = _with_lib(path)
    assert not all(res.values()), f"mutant {name} passed every pin: {res}"
