"""Oracle solutions of large systems, computed once per machine (test infrastructure).

A 32^3 x 64 oracle solve takes a minute or more on the host cores, so its
solution is kept in the temporary directory, keyed by everything that
determines it: lattice, link width eps, kappa, mu, the input seeds, the
tolerance and a hash of the oracle's C sources. Nothing here computes; the
solution comes from oracle.solve alone.
"""
from __future__ import annotations

import hashlib
import os
import tempfile

import numpy as np

import oracle
from oracle import build as obuild
from paper_1112_5280_gb300 import synth

CACHE_DIR = os.path.join(tempfile.gettempdir(), "lqcd_oracle_cache")


def _oracle_hash() -> str:
    h = hashlib.sha256()
    for p in sorted(obuild.SOURCES + obuild.HEADERS):
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def eo_solution(dims, eps, kappa, mu, seed_links, seed_source, tol):
    """(U, b, x): seeded links and source and the oracle's even-odd CG solution of M x = b
    to ||b - M x|| <= tol ||b||."""
    U = synth.random_links(dims, eps, seed=seed_links)
    b = synth.gaussian_spinor(dims, seed=seed_source)
    key = f"{'x'.join(map(str, dims))}_e{eps}_k{kappa}_m{mu}_s{seed_links}_{seed_source}_t{tol}_{_oracle_hash()}"
    path = os.path.join(CACHE_DIR, key + ".npy")
    if os.path.exists(path):
        return U, b, np.load(path)
    x, status, _, res = oracle.solve(dims, U, kappa, b, tol=tol, method=oracle.METHOD_CG_EO, mu=mu)
    if status != 0 or not res <= tol:
        raise RuntimeError(f"oracle solve did not converge: status {status}, residual {res}")
    os.makedirs(CACHE_DIR, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npy"
    np.save(tmp, x)
    os.replace(tmp, path)
    return U, b, x
