"""ctypes bindings to the FP64 heatbath oracle (heatbath.c; test infrastructure only).

Links use the host layout of wilson_oracle.h: [V, 4, 3, 3] complex128.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import wilson

_ready = False


def _lib():
    global _ready
    lib = wilson._load()
    if not _ready:
        u64p = C.POINTER(C.c_uint64)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        lib.oracle_philox4x64.argtypes = [u64p, u64p, u64p]
        lib.oracle_philox4x64.restype = None
        lib.oracle_su2_draws.argtypes = [C.c_double, C.c_uint64, C.c_longlong, dp]
        lib.oracle_su2_draws.restype = C.c_longlong
        lib.oracle_plaquette.argtypes = [ip, dp]
        lib.oracle_plaquette.restype = C.c_double
        lib.oracle_staple.argtypes = [ip, dp, C.c_longlong, C.c_int, dp]
        lib.oracle_staple.restype = None
        lib.oracle_heatbath_link.argtypes = [ip, dp, C.c_double, C.c_uint64, C.c_uint64, C.c_longlong,
                                             C.c_int]
        lib.oracle_heatbath_link.restype = C.c_int
        lib.oracle_heatbath.argtypes = [ip, dp, C.c_double, C.c_uint64, C.c_uint64, C.c_int, C.c_int]
        lib.oracle_heatbath.restype = C.c_longlong
        lib.oracle_reunitarise.argtypes = [ip, dp]
        lib.oracle_reunitarise.restype = None
        _ready = True
    return lib


def _dims(dims):
    return (C.c_int * 4)(*[int(d) for d in dims])


def _links(U, dims):
    V = int(np.prod(dims))
    U = np.ascontiguousarray(U, dtype=np.complex128)
    if U.shape != (V, 4, 3, 3):
        raise ValueError(f"expected links [{V}, 4, 3, 3], got {U.shape}")
    return U


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def philox4x64(counter, key):
    ctr = (C.c_uint64 * 4)(*[int(c) for c in counter])
    k = (C.c_uint64 * 2)(*[int(c) for c in key])
    out = (C.c_uint64 * 4)()
    _lib().oracle_philox4x64(ctr, k, out)
    return [int(x) for x in out]


def su2_draws(alpha, seed, n):
    """Returns (draws [n, 4], number that hit the attempt limit)."""
    out = np.empty((int(n), 4), dtype=np.float64)
    fails = _lib().oracle_su2_draws(float(alpha), int(seed), int(n), _dp(out))
    return out, int(fails)


def plaquette(dims, U):
    U = _links(U, dims)
    return float(_lib().oracle_plaquette(_dims(dims), _dp(U)))


def staple(dims, U, site, mu):
    U = _links(U, dims)
    W = np.empty((3, 3), dtype=np.complex128)
    _lib().oracle_staple(_dims(dims), _dp(U), int(site), int(mu), _dp(W))
    return W


def heatbath_link(dims, U, beta, seed, sweep, site, mu):
    """Updates U[site, mu] in place (U must be a C-contiguous complex128 array)."""
    if not (isinstance(U, np.ndarray) and U.dtype == np.complex128 and U.flags.c_contiguous):
        raise ValueError("U must be a C-contiguous complex128 array (updated in place)")
    rc = _lib().oracle_heatbath_link(_dims(dims), _dp(U), float(beta), int(seed), int(sweep),
                                     int(site), int(mu))
    if rc < 0:
        raise ValueError("oracle_heatbath_link: bad arguments")
    return rc


def heatbath(dims, U, beta, seed, sweep0=0, nsweeps=1, reunit=True):
    """Returns (new links, number of subgroup updates that hit the attempt limit)."""
    U = _links(U, dims).copy()
    fails = _lib().oracle_heatbath(_dims(dims), _dp(U), float(beta), int(seed), int(sweep0),
                                   int(nsweeps), int(bool(reunit)))
    if fails < 0:
        raise ValueError("oracle_heatbath: bad arguments")
    return U, int(fails)


def reunitarise(dims, U):
    U = _links(U, dims).copy()
    _lib().oracle_reunitarise(_dims(dims), _dp(U))
    return U
