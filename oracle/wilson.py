"""ctypes bindings to the FP64 C oracle (test infrastructure only).

All arrays use the host layout of wilson_oracle.h: links [V, 4, 3, 3] and
spinors [V, 4, 3], complex128, site s = x + Lx*(y + Ly*(z + Lz*t)).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

METHOD_CG_FULL = 0
METHOD_CG_EO = 1
METHOD_BICGSTAB_EO = 2

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        lib.oracle_hop.argtypes = [ip, C.c_int, dp, dp, dp, C.c_int]
        lib.oracle_hop_eo.argtypes = [ip, C.c_int, dp, dp, dp, C.c_int, C.c_int]
        lib.oracle_hop_sites.argtypes = [ip, C.c_int, dp, dp, C.POINTER(C.c_longlong),
                                         C.c_longlong, dp, C.c_int]
        lib.oracle_apply_M.argtypes = [ip, C.c_int, dp, C.c_double, C.c_double, dp, dp, C.c_int]
        lib.oracle_apply_Mhat.argtypes = [ip, C.c_int, dp, C.c_double, C.c_double, dp, dp, C.c_int]
        lib.oracle_solve.argtypes = [ip, C.c_int, dp, C.c_double, C.c_double, dp, dp, C.c_double,
                                     C.c_int, C.c_int, dp]
        lib.oracle_true_residual.argtypes = [ip, C.c_int, dp, C.c_double, C.c_double, dp, dp]
        lib.oracle_true_residual.restype = C.c_double
        lib.oracle_set_threads.argtypes = [C.c_int]
        lib.oracle_get_threads.restype = C.c_int
        for f in (lib.oracle_hop, lib.oracle_hop_eo, lib.oracle_hop_sites, lib.oracle_apply_M,
                  lib.oracle_apply_Mhat, lib.oracle_solve):
            f.restype = C.c_int
        _lib = lib
    return _lib


def _dims(dims):
    return (C.c_int * 4)(*[int(d) for d in dims])


def _c128(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _vol(dims):
    return int(np.prod([int(d) for d in dims]))


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def hop(dims, U, psi, t_bc=-1, dagger=False):
    V = _vol(dims)
    U = _c128(U, (V, 4, 3, 3))
    psi = _c128(psi, (V, 4, 3))
    out = np.empty_like(psi)
    rc = _load().oracle_hop(_dims(dims), int(t_bc), _ptr(U), _ptr(psi), _ptr(out), int(dagger))
    if rc:
        raise ValueError(f"oracle_hop failed: {rc}")
    return out


def hop_eo(dims, U, psi, out_parity, t_bc=-1, dagger=False):
    V = _vol(dims)
    U = _c128(U, (V, 4, 3, 3))
    psi = _c128(psi, (V, 4, 3))
    out = np.empty_like(psi)
    rc = _load().oracle_hop_eo(_dims(dims), int(t_bc), _ptr(U), _ptr(psi), _ptr(out),
                               int(out_parity), int(dagger))
    if rc:
        raise ValueError(f"oracle_hop_eo failed: {rc}")
    return out


def hop_sites(dims, U, psi, sites, t_bc=-1, dagger=False):
    V = _vol(dims)
    U = _c128(U, (V, 4, 3, 3))
    psi = _c128(psi, (V, 4, 3))
    sites = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(sites), 4, 3), dtype=np.complex128)
    rc = _load().oracle_hop_sites(_dims(dims), int(t_bc), _ptr(U), _ptr(psi),
                                  sites.ctypes.data_as(C.POINTER(C.c_longlong)),
                                  C.c_longlong(len(sites)), _ptr(out), int(dagger))
    if rc:
        raise ValueError(f"oracle_hop_sites failed: {rc}")
    return out


def apply_M(dims, U, kappa, psi, t_bc=-1, dagger=False, mu=0.0):
    V = _vol(dims)
    U = _c128(U, (V, 4, 3, 3))
    psi = _c128(psi, (V, 4, 3))
    out = np.empty_like(psi)
    rc = _load().oracle_apply_M(_dims(dims), int(t_bc), _ptr(U), float(kappa), float(mu),
                                _ptr(psi), _ptr(out), int(dagger))
    if rc:
        raise ValueError(f"oracle_apply_M failed: {rc}")
    return out


def apply_Mhat(dims, U, kappa, psi, t_bc=-1, dagger=False, mu=0.0):
    V = _vol(dims)
    U = _c128(U, (V, 4, 3, 3))
    psi = _c128(psi, (V, 4, 3))
    out = np.empty_like(psi)
    rc = _load().oracle_apply_Mhat(_dims(dims), int(t_bc), _ptr(U), float(kappa), float(mu),
                                   _ptr(psi), _ptr(out), int(dagger))
    if rc:
        raise ValueError(f"oracle_apply_Mhat failed: {rc}")
    return out


def solve(dims, U, kappa, b, tol=1e-10, maxiter=10000, method=METHOD_CG_EO, t_bc=-1, mu=0.0):
    """Returns (x, status, iterations, true_relative_residual)."""
    V = _vol(dims)
    U = _c128(U, (V, 4, 3, 3))
    b = _c128(b, (V, 4, 3))
    x = np.zeros_like(b)
    info = np.zeros(2, dtype=np.float64)
    rc = _load().oracle_solve(_dims(dims), int(t_bc), _ptr(U), float(kappa), float(mu), _ptr(b),
                              _ptr(x), float(tol), int(maxiter), int(method),
                              info.ctypes.data_as(C.POINTER(C.c_double)))
    if rc < 0:
        raise ValueError(f"oracle_solve failed: {rc}")
    return x, int(rc), int(info[0]), float(info[1])


def true_residual(dims, U, kappa, b, x, t_bc=-1, mu=0.0):
    V = _vol(dims)
    U = _c128(U, (V, 4, 3, 3))
    b = _c128(b, (V, 4, 3))
    x = _c128(x, (V, 4, 3))
    return float(_load().oracle_true_residual(_dims(dims), int(t_bc), _ptr(U), float(kappa),
                                              float(mu), _ptr(b), _ptr(x)))
