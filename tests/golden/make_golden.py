"""Writes the golden fixtures of tests/golden from the FP64 oracle (test infrastructure).

The paper prints no worked example (its only numbers are timings), so every stored value
here comes from the oracle alone, on the seeded synthetic inputs of
paper_1112_5280_gb300.synth. The fixtures freeze the oracle's results: tests/test_golden.py
recomputes them on the CPU (a change to the oracle's arithmetic shows up there and must
name its justification), and tests/test_gpu_golden.py holds the CUDA path against them
without running the oracle.

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import gauge as ogauge  # noqa: E402
from oracle import hmc as ohmc  # noqa: E402
from paper_1112_5280_gb300 import synth  # noqa: E402

# (name, what, paper passage)
HOP = ("hop_2x2x2x4.txt", "D psi (hopping term, both parities) on 2x2x2x4, links eps 0.5 seed 1001, "
       "spinor seed 2002, antiperiodic t", "Section 3, the dslash")
MHAT = ("mhat_tm_2x2x2x4.txt", "Mhat(kappa 0.15, mu 0.1) on the even sites of the same inputs",
        "Section 3, even-odd preconditioned twisted-mass fermion matrix")
SOLVE = ("solve_4x4x4x4.txt", "x = M^-1 b on 4^4, kappa 0.12, links eps 0.3 seed 1001, source seed 2002 "
         "(EO CG to 1e-13): |x|^2 and x at sites 0, 77, 255", "Section 3, the fermion-matrix inversion")
HEATBATH = ("heatbath_2x2x2x2.txt", "two heatbath sweeps at beta 2.3 (seed 17, sweeps 5-6) from links eps 0.8 "
            "seed 1001 on 2^4: plaquette, then the 4 links of site 0", "Section 3, the SU(3) heatbath")
HMC = ("hmc_2x2x2x4.txt", "one leapfrog trajectory (tau 0.2, 2 steps x 2 gauge steps), beta 5.0, kappa 0.12, "
       "mu 0.1, links eps 0.5 seed 231, momenta seed 232, eta seed 233 on 2x2x2x4: H0, dH, then P at site 0",
       "Section 3, the HMC")
SOLVE_SITES = (0, 77, 255)


def _write(spec, values):
    name, what, passage = spec
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# {what}\n# written by tests/golden/make_golden.py from the FP64 oracle; paper: {passage}\n")
        for v in np.asarray(values, dtype=complex).ravel():
            f.write(f"{v.real:.17e} {v.imag:.17e}\n")


def hop_values():
    dims = (2, 2, 2, 4)
    U = synth.random_links(dims, 0.5, seed=1001)
    psi = synth.gaussian_spinor(dims, seed=2002)
    return oracle.hop(dims, U, psi)


def mhat_values():
    dims = (2, 2, 2, 4)
    U = synth.random_links(dims, 0.5, seed=1001)
    psi = synth.gaussian_spinor(dims, seed=2002) * (synth.parity_of_sites(dims) == 0)[:, None, None]
    out = oracle.apply_Mhat(dims, U, 0.15, psi, mu=0.1)
    return out[synth.parity_of_sites(dims) == 0]


def solve_values():
    dims = (4, 4, 4, 4)
    U = synth.random_links(dims, 0.3, seed=1001)
    b = synth.gaussian_spinor(dims, seed=2002)
    x, status, _, _ = oracle.solve(dims, U, 0.12, b, tol=1e-13, method=oracle.METHOD_CG_EO)
    assert status == 0
    return np.concatenate([[np.vdot(x, x)], np.concatenate([x[s].ravel() for s in SOLVE_SITES])])


def heatbath_values():
    dims = (2, 2, 2, 2)
    U0 = synth.random_links(dims, 0.8, seed=1001)
    U, fails = ogauge.heatbath(dims, U0, 2.3, seed=17, sweep0=5, nsweeps=2)
    assert fails == 0
    return np.concatenate([[ogauge.plaquette(dims, U)], U[0].ravel()])


def hmc_values():
    dims, beta, kappa, mu = (2, 2, 2, 4), 5.0, 0.12, 0.1
    U = synth.random_links(dims, 0.5, seed=231)
    P = synth.gaussian_momenta(dims, 232)
    eta = synth.gaussian_spinor(dims, seed=233) * (synth.parity_of_sites(dims) == 0)[:, None, None]
    phi = ohmc.pseudofermion(dims, U, kappa, mu, eta)
    U1, P1 = ohmc.integrate(dims, U, P, phi, beta, kappa, mu, 0.2, 2, scheme="leapfrog", ngauge=2)
    h0 = ohmc.hamiltonian(dims, U, P, phi, beta, kappa, mu)
    h1 = ohmc.hamiltonian(dims, U1, P1, phi, beta, kappa, mu)
    return np.concatenate([[h0, h1 - h0], P1[0].ravel()])


GOLDEN = [(HOP, hop_values), (MHAT, mhat_values), (SOLVE, solve_values), (HEATBATH, heatbath_values),
          (HMC, hmc_values)]


def read(name):
    vals = np.loadtxt(os.path.join(HERE, name), comments="#")
    return vals[:, 0] + 1j * vals[:, 1]


if __name__ == "__main__":
    for spec, fn in GOLDEN:
        _write(spec, fn())
        print("wrote", spec[0])
