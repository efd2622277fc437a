"""Meson two-point functions from a point-source propagator (test infrastructure only).

Paper Section 4, eq. (4.1): for a propagator S(x0, x) ~ M^-1 b(x0) from a point
source at x0, the N_f = 2 flavour-doublet meson correlator with Dirac
structure Gamma is

    C_Gamma(x0, x) = - Tr[ S^dag(x0, x) g5 Gamma S(x0, x) Gamma g5 ],

with the trace over spin and colour. S(x) is the 12 x 12 matrix whose column
(beta, b) is the solution of M x = (point source at x0, spin beta, colour b),
read at site x, row (alpha, a). The time-slice correlator is
C_Gamma(t) = sum over spatial x of C_Gamma(x, t).

Here S is built as an explicit matrix per site and the trace is taken with
plain matrix products (numpy), the definition written out.
"""
from __future__ import annotations

import numpy as np

from .dense import gammas

# Dirac structures, in the order of the library's LQCD_G_* codes
GAMMA_NAMES = ("1", "g5", "gx", "gy", "gz", "gt", "g5gx", "g5gy", "g5gz", "g5gt")


def gamma_matrix(code: int) -> np.ndarray:
    g, g5 = gammas()
    if code == 0:
        return np.eye(4, dtype=np.complex128)
    if code == 1:
        return g5
    if 2 <= code <= 5:
        return g[code - 2]
    if 6 <= code <= 9:
        return g5 @ g[code - 6]
    raise ValueError(code)


def propagator_matrix(solutions) -> np.ndarray:
    """solutions[3*beta + b] is the [V, 4, 3] solution for source spin beta, colour b.
    Returns S[V, 12, 12] with S[x, 3*alpha + a, 3*beta + b]."""
    sols = np.asarray(solutions)  # [12, V, 4, 3]
    V = sols.shape[1]
    return np.transpose(sols.reshape(12, V, 12), (1, 2, 0))


def meson_correlator_sites(solutions, code: int) -> np.ndarray:
    """C_Gamma(x) for every site x (complex)."""
    S = propagator_matrix(solutions)
    G = gamma_matrix(code)
    g5 = gamma_matrix(1)
    A = np.kron(g5 @ G, np.eye(3))
    B = np.kron(G @ g5, np.eye(3))
    Sd = np.conj(np.swapaxes(S, -1, -2))
    prod = Sd @ A @ S @ B
    return -np.trace(prod, axis1=-2, axis2=-1)


def meson_correlator(dims, solutions, codes) -> np.ndarray:
    """C_Gamma(t) for each code: array [len(codes), Lt] complex."""
    lx, ly, lz, lt = dims
    out = np.zeros((len(codes), lt), dtype=np.complex128)
    for i, c in enumerate(codes):
        cx = meson_correlator_sites(solutions, c).reshape(lt, lz * ly * lx)
        out[i] = cx.sum(axis=1)
    return out
