"""ctypes binding of liblqcd.so (include/lqcd.h). Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.

Host arrays use the library's host layout (complex128):
  links  [V, 4, 3, 3]   spinors [V, 4, 3],   site = x + Lx*(y + Ly*(z + Lz*t)).
Device arrays may be torch tensors (complex128 / float64, same layout); their
data pointers are passed to the *_dev entry points.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ENOCONV, EBREAKDOWN, ENONFINITE, ETIMEOUT, ECUDA, EBUSY = 0, -1, -2, -3, -4, -5, -6, -7, -8
F64, F32, F16, BF16, DF64 = 0, 1, 2, 3, 4
EVEN, ODD, FULL = 0, 1, 2
CG, BICGSTAB = 0, 1

PRECISIONS = {"f64": F64, "f32": F32, "f16": F16, "bf16": BF16, "df64": DF64}


class LqcdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"lqcd error {code}: {msg}")
        self.code = code


class SolveOpts(C.Structure):
    _fields_ = [("solver", C.c_int), ("sloppy_prec", C.c_int), ("sloppy_compress", C.c_int),
                ("maxiter", C.c_int), ("delta", C.c_double), ("chunk", C.c_int),
                ("use_graph", C.c_int), ("ru_interval", C.c_int), ("true_prec", C.c_int),
                ("multi_rhs_links", C.c_int), ("mu", C.c_double)]


class SolveInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("reliable_updates", C.c_int),
                ("pad", C.c_int), ("true_resid", C.c_double), ("ms", C.c_double)]

    def as_dict(self):
        return {"status": self.status, "iters": self.iters,
                "reliable_updates": self.reliable_updates, "true_resid": self.true_resid,
                "ms": self.ms}


class HmcParams(C.Structure):
    _fields_ = [("beta", C.c_double), ("kappa", C.c_double), ("mu", C.c_double), ("tau", C.c_double),
                ("nsteps", C.c_int), ("ngauge", C.c_int), ("scheme", C.c_int), ("chrono", C.c_int),
                ("tol", C.c_double), ("accept_u", C.c_double)]


class HmcInfo(C.Structure):
    _fields_ = [("dH", C.c_double), ("H0", C.c_double), ("H1", C.c_double), ("kinetic0", C.c_double),
                ("kinetic1", C.c_double), ("gauge0", C.c_double), ("gauge1", C.c_double),
                ("fermion0", C.c_double), ("fermion1", C.c_double), ("plaquette", C.c_double),
                ("accepted", C.c_int), ("force_evals", C.c_int), ("solver_iters", C.c_int), ("pad", C.c_int),
                ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


LEAPFROG, TWO_MN = 0, 1


class TuneResult(C.Structure):
    _fields_ = [("prec", C.c_int), ("nr", C.c_int), ("ntiles", C.c_int), ("ctas_per_sm", C.c_int),
                ("form", C.c_int), ("candidates", C.c_int), ("us_best", C.c_double),
                ("us_default", C.c_double), ("nrhs", C.c_int), ("group", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_VP = C.c_void_p
_IP = C.POINTER(C.c_int)


def _sig(lib, name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args


def load(build_if_missing: bool = True):
    """Load the library; builds it first when it is missing or stale and nvcc exists.
    With the environment variable LQCD_DEBUG_BOUNDS=1 the bounds-checked debug build is
    built and loaded instead (see lqcd_debug_bounds)."""
    global _lib
    if _lib is not None:
        return _lib
    debug = os.environ.get("LQCD_DEBUG_BOUNDS", "0") == "1"
    path = _build.lib_path(debug)
    if build_if_missing and not _build.up_to_date(debug):
        _build.build(debug=debug)
    if not os.path.exists(path):
        raise RuntimeError(f"liblqcd.so not built ({path}); run __graft_entry__.build()")
    lib = C.CDLL(path)
    i, d, sz, ll = C.c_int, C.c_double, C.c_size_t, C.c_longlong
    _sig(lib, "lqcd_status_string", C.c_char_p, [i])
    _sig(lib, "lqcd_last_error", C.c_char_p, [])
    _sig(lib, "lqcd_version", C.c_char_p, [])
    _sig(lib, "lqcd_ctx_create", i, [C.POINTER(_VP), i, _VP])
    _sig(lib, "lqcd_ctx_destroy", None, [_VP])
    _sig(lib, "lqcd_ctx_set_stream", i, [_VP, _VP])
    _sig(lib, "lqcd_ctx_stream", _VP, [_VP])
    _sig(lib, "lqcd_ctx_release_cache", i, [_VP])
    _sig(lib, "lqcd_ctx_sync", i, [_VP])
    _sig(lib, "lqcd_ctx_launch_count", ll, [_VP])
    _sig(lib, "lqcd_alu_peak", i, [_VP, i, C.POINTER(d)])
    _sig(lib, "lqcd_debug_bounds", i, [_VP, C.POINTER(C.c_ulonglong)])
    _sig(lib, "lqcd_set_grid_multiplier", None, [i, i])
    _sig(lib, "lqcd_set_dslash_form", i, [i, i])
    _sig(lib, "lqcd_gauge_upload", i, [_VP, _IP, _VP, i, i, i, C.POINTER(_VP)])
    _sig(lib, "lqcd_gauge_upload_dev", i, [_VP, _IP, _VP, i, i, i, C.POINTER(_VP)])
    _sig(lib, "lqcd_gauge_add_copy", i, [_VP, i, i])
    _sig(lib, "lqcd_gauge_bytes", sz, [_VP])
    _sig(lib, "lqcd_gauge_destroy", None, [_VP])
    _sig(lib, "lqcd_field_create", i, [_VP, _IP, i, i, C.POINTER(_VP)])
    _sig(lib, "lqcd_field_upload", i, [_VP, _VP])
    _sig(lib, "lqcd_field_download", i, [_VP, _VP])
    _sig(lib, "lqcd_field_upload_dev", i, [_VP, _VP])
    _sig(lib, "lqcd_field_download_dev", i, [_VP, _VP])
    _sig(lib, "lqcd_field_copy", i, [_VP, _VP, d])
    _sig(lib, "lqcd_field_norm2", i, [_VP, C.POINTER(d)])
    _sig(lib, "lqcd_field_zero", i, [_VP])
    _sig(lib, "lqcd_field_bytes", sz, [_VP])
    _sig(lib, "lqcd_field_destroy", None, [_VP])
    _sig(lib, "lqcd_dslash_eo", i, [_VP, _VP, _VP, i, i])
    _sig(lib, "lqcd_apply_Mhat", i, [_VP, d, _VP, _VP, i])
    _sig(lib, "lqcd_apply_M", i, [_VP, d, _VP, _VP, i])
    _sig(lib, "lqcd_apply_Mhat_tm", i, [_VP, d, d, _VP, _VP, i])
    _sig(lib, "lqcd_apply_M_tm", i, [_VP, d, d, _VP, _VP, i])
    _sig(lib, "lqcd_dslash_batch_create", i, [i, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(_VP), i, i,
                                              C.POINTER(_VP)])
    _sig(lib, "lqcd_dslash_batch_apply", i, [_VP])
    _sig(lib, "lqcd_dslash_batch_destroy", None, [_VP])
    _sig(lib, "lqcd_meson_correlator", i, [C.POINTER(_VP), i, C.POINTER(C.c_int), _VP])
    _sig(lib, "lqcd_gauge_download", i, [_VP, _VP])
    _sig(lib, "lqcd_mom_create", i, [_VP, _IP, C.POINTER(_VP)])
    _sig(lib, "lqcd_mom_upload", i, [_VP, _VP])
    _sig(lib, "lqcd_mom_download", i, [_VP, _VP])
    _sig(lib, "lqcd_mom_zero", i, [_VP])
    _sig(lib, "lqcd_mom_kinetic", i, [_VP, C.POINTER(d)])
    _sig(lib, "lqcd_mom_destroy", None, [_VP])
    _sig(lib, "lqcd_gauge_force", i, [_VP, d, d, _VP])
    _sig(lib, "lqcd_fermion_force", i, [_VP, d, d, _VP, d, _VP, C.POINTER(d)])
    _sig(lib, "lqcd_gauge_update", i, [_VP, _VP, d])
    _sig(lib, "lqcd_hmc_params_default", None, [C.POINTER(HmcParams)])
    _sig(lib, "lqcd_hmc_trajectory", i, [_VP, C.POINTER(HmcParams), _VP, _VP, C.POINTER(SolveOpts),
                                         C.POINTER(HmcInfo)])
    _sig(lib, "lqcd_heatbath", i, [_VP, d, i, C.c_ulonglong, C.c_ulonglong, i, C.POINTER(ll)])
    _sig(lib, "lqcd_plaquette", i, [_VP, C.POINTER(d)])
    _sig(lib, "lqcd_autotune_dslash", i, [i, C.POINTER(_VP), i, i, C.POINTER(TuneResult)])
    _sig(lib, "lqcd_tune_entries", i, [C.POINTER(TuneResult), i, _IP])
    _sig(lib, "lqcd_tune_clear", None, [])
    _sig(lib, "lqcd_tune_save", i, [C.c_char_p])
    _sig(lib, "lqcd_tune_load", i, [C.c_char_p])
    if hasattr(lib, "lqcd_apply_Mhat_noalloc"):
        _sig(lib, "lqcd_apply_Mhat_noalloc", i, [_VP, d, _VP, _VP, i])
    if hasattr(lib, "lqcd_solve"):
        _sig(lib, "lqcd_solve_opts_default", None, [C.POINTER(SolveOpts)])
        _sig(lib, "lqcd_solve", i, [_VP, _VP, d, d, C.POINTER(SolveOpts), _VP, C.POINTER(SolveInfo)])
        _sig(lib, "lqcd_solve_fields", i, [_VP, _VP, d, d, C.POINTER(SolveOpts), _VP,
                                           C.POINTER(SolveInfo)])
        _sig(lib, "lqcd_solve_multi", i, [_VP, i, C.POINTER(_VP), d, d, C.POINTER(SolveOpts),
                                          C.POINTER(_VP), C.POINTER(SolveInfo)])
        _sig(lib, "lqcd_solve_batch", i, [i, C.POINTER(_VP), C.POINTER(_VP), C.POINTER(d), C.POINTER(d),
                                          C.POINTER(SolveOpts), C.POINTER(_VP), C.POINTER(SolveInfo)])
        _sig(lib, "lqcd_engine_create", i, [_VP, C.POINTER(SolveOpts), sz, i, C.POINTER(_VP)])
        _sig(lib, "lqcd_engine_request_bytes", sz, [_VP, _IP])
        _sig(lib, "lqcd_engine_submit", i, [_VP, _VP, _VP, d, d, C.POINTER(ll)])
        _sig(lib, "lqcd_engine_submit_tm", i, [_VP, _VP, _VP, d, d, d, C.POINTER(ll)])
        _sig(lib, "lqcd_engine_submit_normal", i, [_VP, _VP, _VP, d, d, d, C.POINTER(ll)])
        _sig(lib, "lqcd_solve_normal", i, [_VP, _VP, d, d, C.POINTER(SolveOpts), _VP, C.POINTER(SolveInfo)])
        _sig(lib, "lqcd_engine_step", i, [_VP, _IP])
        _sig(lib, "lqcd_engine_completed", i, [_VP, C.POINTER(ll), i, _IP])
        _sig(lib, "lqcd_engine_result", i, [_VP, ll, _VP, C.POINTER(SolveInfo)])
        _sig(lib, "lqcd_engine_cancel", i, [_VP, ll, i])
        _sig(lib, "lqcd_engine_stats", i, [_VP, _IP, C.POINTER(sz)])
        _sig(lib, "lqcd_engine_destroy", None, [_VP])
    _lib = lib
    return lib


def _check(rc):
    if rc != OK:
        lib = load()
        raise LqcdError(rc, f"{lib.lqcd_status_string(rc).decode()}: {lib.lqcd_last_error().decode()}")
    return rc


def _dims(dims):
    return (C.c_int * 4)(*[int(d) for d in dims])


def _prec(p):
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _host_array(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


class Context:
    """A device + stream binding (lqcd_ctx)."""

    def __init__(self, device: int = 0, stream=None):
        self._lib = load()
        h = _VP()
        _check(self._lib.lqcd_ctx_create(C.byref(h), int(device), _stream_handle(stream)))
        self.h = h
        self.device = device
        self._stream = stream  # a borrowed stream must outlive the context's objects

    def close(self):
        if self.h:
            self._lib.lqcd_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        _check(self._lib.lqcd_ctx_set_stream(self.h, _stream_handle(stream)))

    @property
    def stream(self):
        return self._lib.lqcd_ctx_stream(self.h)

    def sync(self):
        _check(self._lib.lqcd_ctx_sync(self.h))

    def release_cache(self):
        """Frees the buffers the one-shot solves keep between calls (lqcd_ctx_release_cache)."""
        _check(self._lib.lqcd_ctx_release_cache(self.h))

    @property
    def launches(self) -> int:
        return int(self._lib.lqcd_ctx_launch_count(self.h))

    def debug_bounds(self):
        """(index, size) of the first out-of-range field access recorded since the last call by
        the bounds-checked build (LQCD_DEBUG_BOUNDS=1), or None; raises in the normal build."""
        w = C.c_ulonglong(0)
        _check(self._lib.lqcd_debug_bounds(self.h, C.byref(w)))
        if not w.value:
            return None
        return int(w.value & 0xFFFFFFFF), int((w.value >> 32) & 0x7FFFFFFF)

    def alu_peak(self, kind: str) -> float:
        """Measured FMA throughput of the device in TFLOP/s: kind "f64", "f32" or "f32x2" (packed
        FP32 pairs) (lqcd_alu_peak)."""
        out = C.c_double(0.0)
        _check(self._lib.lqcd_alu_peak(self.h, {"f64": 0, "f32": 1, "f32x2": 2}[kind], C.byref(out)))
        return float(out.value)

    def gauge(self, dims, U, prec="f64", compress=18, t_bc=-1):
        return Gauge(self, dims, U, prec, compress, t_bc)

    def mom(self, dims, data=None):
        return Mom(self, dims, data)

    def field(self, dims, prec="f64", subset=FULL, data=None):
        f = Field(self, dims, prec, subset)
        if data is not None:
            f.upload(data)
        return f


class Gauge:
    """SU(3) gauge field resident on the device (lqcd_gauge)."""

    def __init__(self, ctx: Context, dims, U, prec="f64", compress=18, t_bc=-1):
        self.ctx, self.dims, self.t_bc = ctx, tuple(int(d) for d in dims), t_bc
        self._lib = ctx._lib
        V = int(np.prod(self.dims))
        h = _VP()
        if hasattr(U, "data_ptr"):  # device tensor in the host layout
            if not U.is_cuda or not U.is_contiguous() or U.numel() * U.element_size() != V * 4 * 9 * 16:
                raise ValueError("device gauge tensor must be contiguous [V,4,3,3] complex128")
            _check(self._lib.lqcd_gauge_upload_dev(ctx.h, _dims(dims), U.data_ptr(), _prec(prec),
                                                   int(compress), int(t_bc), C.byref(h)))
        else:
            U = _host_array(U, (V, 4, 3, 3))
            _check(self._lib.lqcd_gauge_upload(ctx.h, _dims(dims), U.ctypes.data, _prec(prec),
                                               int(compress), int(t_bc), C.byref(h)))
        self.h = h

    def add_copy(self, prec, compress):
        _check(self._lib.lqcd_gauge_add_copy(self.h, _prec(prec), int(compress)))

    @property
    def nbytes(self) -> int:
        return int(self._lib.lqcd_gauge_bytes(self.h))

    def download(self, out=None):
        """FP64 master copy in the host layout [V, 4, 3, 3] complex128."""
        V = int(np.prod(self.dims))
        if out is None:
            out = np.empty((V, 4, 3, 3), dtype=np.complex128)
        if out.shape != (V, 4, 3, 3) or out.dtype != np.complex128 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous [V,4,3,3] complex128 array")
        _check(self._lib.lqcd_gauge_download(self.h, out.ctypes.data))
        return out

    def heatbath(self, beta, nsweeps=1, seed=0, sweep0=0, reunit=True) -> int:
        """SU(3) heatbath sweeps in place (Cabibbo-Marinari with Creutz's SU(2) draw);
        returns the number of subgroup draws that hit the attempt limit."""
        fails = C.c_longlong()
        _check(self._lib.lqcd_heatbath(self.h, float(beta), int(nsweeps), int(seed), int(sweep0),
                                       int(bool(reunit)), C.byref(fails)))
        return fails.value

    def plaquette(self) -> float:
        p = C.c_double()
        _check(self._lib.lqcd_plaquette(self.h, C.byref(p)))
        return p.value

    def close(self):
        if self.h:
            self._lib.lqcd_gauge_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mom:
    """HMC momentum / force field (lqcd_mom): traceless anti-Hermitian 3x3 per link, FP64."""

    def __init__(self, ctx: Context, dims, data=None):
        self.ctx, self.dims = ctx, tuple(int(d) for d in dims)
        self._lib = ctx._lib
        h = _VP()
        _check(self._lib.lqcd_mom_create(ctx.h, _dims(dims), C.byref(h)))
        self.h = h
        if data is not None:
            self.upload(data)

    def upload(self, P):
        V = int(np.prod(self.dims))
        P = _host_array(P, (V, 4, 3, 3))
        _check(self._lib.lqcd_mom_upload(self.h, P.ctypes.data))

    def download(self):
        V = int(np.prod(self.dims))
        out = np.empty((V, 4, 3, 3), dtype=np.complex128)
        _check(self._lib.lqcd_mom_download(self.h, out.ctypes.data))
        return out

    def zero(self):
        _check(self._lib.lqcd_mom_zero(self.h))

    def kinetic(self) -> float:
        e = C.c_double()
        _check(self._lib.lqcd_mom_kinetic(self.h, C.byref(e)))
        return e.value

    def close(self):
        if self.h:
            self._lib.lqcd_mom_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Field:
    """Spinor field on the device (lqcd_field): EVEN, ODD or FULL subset."""

    def __init__(self, ctx: Context, dims, prec="f64", subset=FULL):
        self.ctx, self.dims, self.prec, self.subset = ctx, tuple(int(d) for d in dims), _prec(prec), subset
        self._lib = ctx._lib
        self.V = int(np.prod(self.dims))
        h = _VP()
        _check(self._lib.lqcd_field_create(ctx.h, _dims(dims), self.prec, int(subset), C.byref(h)))
        self.h = h

    def upload(self, psi):
        if hasattr(psi, "data_ptr"):
            if not psi.is_cuda or not psi.is_contiguous() or psi.numel() * psi.element_size() != self.V * 12 * 16:
                raise ValueError("device spinor tensor must be contiguous [V,4,3] complex128")
            _check(self._lib.lqcd_field_upload_dev(self.h, psi.data_ptr()))
        else:
            psi = _host_array(psi, (self.V, 4, 3))
            _check(self._lib.lqcd_field_upload(self.h, psi.ctypes.data))
        return self

    def download(self, out=None):
        if out is not None and hasattr(out, "data_ptr"):
            _check(self._lib.lqcd_field_download_dev(self.h, out.data_ptr()))
            return out
        if out is None:
            out = np.zeros((self.V, 4, 3), dtype=np.complex128)
        _check(self._lib.lqcd_field_download(self.h, out.ctypes.data))
        return out

    def copy_from(self, src: "Field", scale=1.0):
        _check(self._lib.lqcd_field_copy(self.h, src.h, float(scale)))

    def norm2(self) -> float:
        v = C.c_double()
        _check(self._lib.lqcd_field_norm2(self.h, C.byref(v)))
        return v.value

    def zero(self):
        _check(self._lib.lqcd_field_zero(self.h))

    @property
    def nbytes(self) -> int:
        return int(self._lib.lqcd_field_bytes(self.h))

    def close(self):
        if self.h:
            self._lib.lqcd_field_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dslash_eo(gauge: Gauge, fin: Field, fout: Field, out_parity: int, dagger=False):
    _check(gauge._lib.lqcd_dslash_eo(gauge.h, fin.h, fout.h, int(out_parity), int(bool(dagger))))


class DslashBatch:
    """n independent even-odd Dslash applications in one launch (lqcd_dslash_batch)."""

    def __init__(self, gauges, fins, fouts, out_parity, dagger=False):
        n = len(gauges)
        if not (len(fins) == len(fouts) == n):
            raise ValueError("gauges, fins and fouts must have the same length")
        self._lib = gauges[0]._lib
        self._keep = (list(gauges), list(fins), list(fouts))
        h = _VP()
        _check(self._lib.lqcd_dslash_batch_create(
            n, (_VP * n)(*[g.h for g in gauges]), (_VP * n)(*[f.h for f in fins]),
            (_VP * n)(*[f.h for f in fouts]), int(out_parity), int(bool(dagger)), C.byref(h)))
        self.h = h

    def apply(self):
        _check(self._lib.lqcd_dslash_batch_apply(self.h))

    def close(self):
        if self.h:
            self._lib.lqcd_dslash_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apply_Mhat(gauge: Gauge, kappa: float, fin: Field, fout: Field, dagger=False, mu=0.0):
    """Even-odd Schur operator; mu != 0 gives the twisted-mass one, A - k^2 D_eo A^-1 D_oe."""
    if mu == 0.0:
        _check(gauge._lib.lqcd_apply_Mhat(gauge.h, float(kappa), fin.h, fout.h, int(bool(dagger))))
    else:
        _check(gauge._lib.lqcd_apply_Mhat_tm(gauge.h, float(kappa), float(mu), fin.h, fout.h,
                                             int(bool(dagger))))


def apply_Mhat_noalloc(gauge: Gauge, kappa: float, fin: Field, fout: Field, dagger=False):
    """Mhat without any device allocation by the library (fixed 16 MiB built-in
    scratch for the odd temporary; see include/lqcd.h for the limits)."""
    _check(gauge._lib.lqcd_apply_Mhat_noalloc(gauge.h, float(kappa), fin.h, fout.h,
                                              int(bool(dagger))))


def apply_M(gauge: Gauge, kappa: float, fin: Field, fout: Field, dagger=False, mu=0.0):
    """Full operator 1 - kappa D (+ 2 i kappa mu g5 for the twisted mass)."""
    if mu == 0.0:
        _check(gauge._lib.lqcd_apply_M(gauge.h, float(kappa), fin.h, fout.h, int(bool(dagger))))
    else:
        _check(gauge._lib.lqcd_apply_M_tm(gauge.h, float(kappa), float(mu), fin.h, fout.h,
                                          int(bool(dagger))))


def gauge_force(gauge: Gauge, beta, coeff, mom: Mom):
    """mom += coeff (beta/3) TA(U W)."""
    _check(gauge._lib.lqcd_gauge_force(gauge.h, float(beta), float(coeff), mom.h))


def fermion_force(gauge: Gauge, kappa, mu, x: Field, coeff, mom: Mom) -> float:
    """mom += coeff G_f for x = (Mhat^dag Mhat)^-1 phi; returns S_f = phi^dag x."""
    sf = C.c_double()
    _check(gauge._lib.lqcd_fermion_force(gauge.h, float(kappa), float(mu), x.h, float(coeff), mom.h,
                                         C.byref(sf)))
    return sf.value


def gauge_update(gauge: Gauge, mom: Mom, eps):
    """U <- exp(eps P) U."""
    _check(gauge._lib.lqcd_gauge_update(gauge.h, mom.h, float(eps)))


def solve_normal(gauge: Gauge, src: Field, kappa, tol, x: Field, opts: SolveOpts | None = None):
    """(Mhat^dag Mhat) x_e = src_e by CG; returns the info dict."""
    info = SolveInfo()
    o = opts if opts is not None else solve_opts()
    rc = gauge._lib.lqcd_solve_normal(gauge.h, src.h, float(kappa), float(tol), C.byref(o), x.h,
                                      C.byref(info))
    if rc not in (OK, ENOCONV, EBREAKDOWN, ENONFINITE):
        _check(rc)
    return info.as_dict()


def hmc_params(**kw) -> HmcParams:
    p = HmcParams()
    load().lqcd_hmc_params_default(C.byref(p))
    names = {f[0] for f in HmcParams._fields_}
    for k, v in kw.items():
        if k not in names or k == "pad":
            raise TypeError(f"unknown HMC parameter {k!r}")
        setattr(p, k, v)
    return p


def hmc_trajectory(gauge: Gauge, params: HmcParams, mom: Mom, phi: Field, opts: SolveOpts | None = None):
    """One MD trajectory (and Metropolis test when params.accept_u > 0); returns the info dict."""
    info = HmcInfo()
    o = opts if opts is not None else solve_opts()
    _check(gauge._lib.lqcd_hmc_trajectory(gauge.h, C.byref(params), mom.h, phi.h, C.byref(o),
                                          C.byref(info)))
    return info.as_dict()


def autotune_dslash(gauges, prec, compress=0) -> dict:
    """Times the batched Dslash over one slot per gauge (gauges may repeat) for every
    persistent grid and kernel form; later launches with the same key use the fastest.
    compress: 12 or 18 link reals (0: each gauge's default copy)."""
    gauges = list(gauges)
    if not gauges:
        raise ValueError("need at least one gauge")
    arr = (_VP * len(gauges))(*[g.h for g in gauges])
    r = TuneResult()
    _check(gauges[0]._lib.lqcd_autotune_dslash(len(gauges), arr, _prec(prec), int(compress),
                                               C.byref(r)))
    return r.as_dict()


def tune_entries() -> list:
    lib = load()
    n = C.c_int()
    _check(lib.lqcd_tune_entries(None, 0, C.byref(n)))
    buf = (TuneResult * max(1, n.value))()
    _check(lib.lqcd_tune_entries(buf, n.value, C.byref(n)))
    return [buf[k].as_dict() for k in range(n.value)]


def tune_clear() -> None:
    load().lqcd_tune_clear()


def tune_save(path) -> None:
    _check(load().lqcd_tune_save(os.fsencode(path)))


def tune_load(path) -> None:
    _check(load().lqcd_tune_load(os.fsencode(path)))


GAMMA_CODES = {"1": 0, "g5": 1, "gx": 2, "gy": 3, "gz": 4, "gt": 5,
               "g5gx": 6, "g5gy": 7, "g5gz": 8, "g5gt": 9}


def meson_correlator(props, gammas):
    """C_Gamma(t) for the 12 FULL FP64 propagator fields (source spin*3 + colour order).
    gammas: codes or names; returns complex array [len(gammas), Lt]."""
    if len(props) != 12:
        raise ValueError("need the 12 point-source solutions")
    codes = [GAMMA_CODES[g] if isinstance(g, str) else int(g) for g in gammas]
    lt = props[0].dims[3]
    out = np.zeros((len(codes), lt, 2), dtype=np.float64)
    _check(props[0]._lib.lqcd_meson_correlator((_VP * 12)(*[p.h for p in props]), len(codes),
                                               (C.c_int * len(codes))(*codes), out.ctypes.data))
    return out[..., 0] + 1j * out[..., 1]


def set_dslash_form(prec, form: int):
    """Dslash kernel form for DF64 fields: 0 one thread per site, 1 three per site."""
    _check(load().lqcd_set_dslash_form(_prec(prec), int(form)))


def set_grid_multiplier(family: int, mult: int):
    load().lqcd_set_grid_multiplier(int(family), int(mult))


def solve_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    load().lqcd_solve_opts_default(C.byref(o))
    names = {f[0] for f in SolveOpts._fields_}
    for k, v in kw.items():
        if k not in names or k == "pad":
            raise TypeError(f"unknown solve option {k!r}")
        if k in ("sloppy_prec", "true_prec") and isinstance(v, str):
            v = _prec(v)
        setattr(o, k, v)
    return o


def solve(gauge: Gauge, src, kappa, tol=1e-10, opts: SolveOpts | None = None):
    """Host solve: src full-lattice numpy spinor; returns (x, info dict)."""
    V = int(np.prod(gauge.dims))
    src = _host_array(src, (V, 4, 3))
    x = np.zeros_like(src)
    info = SolveInfo()
    o = opts if opts is not None else solve_opts()
    rc = gauge._lib.lqcd_solve(gauge.h, src.ctypes.data, float(kappa), float(tol), C.byref(o),
                               x.ctypes.data, C.byref(info))
    if rc not in (OK, ENOCONV, EBREAKDOWN, ENONFINITE):
        _check(rc)
    return x, info.as_dict()


def solve_fields(gauge: Gauge, src: Field, kappa, tol, x: Field, opts: SolveOpts | None = None):
    info = SolveInfo()
    o = opts if opts is not None else solve_opts()
    rc = gauge._lib.lqcd_solve_fields(gauge.h, src.h, float(kappa), float(tol), C.byref(o), x.h,
                                      C.byref(info))
    if rc not in (OK, ENOCONV, EBREAKDOWN, ENONFINITE):
        _check(rc)
    return info.as_dict()


def solve_multi(gauge: Gauge, srcs, kappa, tol, xs, opts: SolveOpts | None = None):
    n = len(srcs)
    sp = (_VP * n)(*[s.h for s in srcs])
    xp = (_VP * n)(*[x.h for x in xs])
    infos = (SolveInfo * n)()
    o = opts if opts is not None else solve_opts()
    rc = gauge._lib.lqcd_solve_multi(gauge.h, n, sp, float(kappa), float(tol), C.byref(o), xp, infos)
    if rc not in (OK, ENOCONV, EBREAKDOWN, ENONFINITE):
        _check(rc)
    return [infos[i].as_dict() for i in range(n)]


def solve_batch(gauges, srcs, kappas, tols, xs, opts: SolveOpts | None = None):
    """lqcd_solve_batch: n independent systems, each on its own gauge field (any lattice
    sizes), kappa and tolerance, solved together; returns the n info dicts."""
    n = len(gauges)
    if not (len(srcs) == len(xs) == n):
        raise ValueError("gauges, srcs and xs must have the same length")
    if isinstance(kappas, (int, float)):
        kappas = [kappas] * n
    if isinstance(tols, (int, float)):
        tols = [tols] * n
    if not (len(kappas) == len(tols) == n):
        raise ValueError("kappas and tols must have one entry per system")
    lib = gauges[0]._lib
    gp = (_VP * n)(*[g.h for g in gauges])
    sp = (_VP * n)(*[s.h for s in srcs])
    xp = (_VP * n)(*[x.h for x in xs])
    kp = (C.c_double * n)(*[float(k) for k in kappas])
    tp = (C.c_double * n)(*[float(t) for t in tols])
    infos = (SolveInfo * n)()
    o = opts if opts is not None else solve_opts()
    rc = lib.lqcd_solve_batch(n, gp, sp, kp, tp, C.byref(o), xp, infos)
    if rc not in (OK, ENOCONV, EBREAKDOWN, ENONFINITE):
        _check(rc)
    return [infos[i].as_dict() for i in range(n)]


class Engine:
    """Batched Krylov engine (lqcd_engine): many solves advance in the same launches."""

    def __init__(self, ctx: Context, opts: SolveOpts | None = None, hbm_budget=0, max_slots=64):
        self._lib = ctx._lib
        self.ctx = ctx
        h = _VP()
        o = opts if opts is not None else solve_opts()
        _check(self._lib.lqcd_engine_create(ctx.h, C.byref(o), C.c_size_t(int(hbm_budget)),
                                            int(max_slots), C.byref(h)))
        self.h = h

    def request_bytes(self, dims) -> int:
        return int(self._lib.lqcd_engine_request_bytes(self.h, _dims(dims)))

    def submit(self, gauge: Gauge, src: Field, kappa, tol, mu=None, normal=False):
        """Returns a request id, or None when the engine is busy (retry later). mu: the
        request's twisted mass (None: the engine's option). normal: solve
        (Mhat^dag Mhat) x_e = src_e instead of M x = src."""
        rid = C.c_longlong()
        if normal:
            m = 0.0 if mu is None else float(mu)
            rc = self._lib.lqcd_engine_submit_normal(self.h, gauge.h, src.h, float(kappa), m, float(tol),
                                                     C.byref(rid))
        elif mu is None:
            rc = self._lib.lqcd_engine_submit(self.h, gauge.h, src.h, float(kappa), float(tol),
                                              C.byref(rid))
        else:
            rc = self._lib.lqcd_engine_submit_tm(self.h, gauge.h, src.h, float(kappa), float(mu),
                                                 float(tol), C.byref(rid))
        if rc == EBUSY:
            return None
        _check(rc)
        return rid.value

    def step(self) -> int:
        n = C.c_int()
        _check(self._lib.lqcd_engine_step(self.h, C.byref(n)))
        return n.value

    def completed(self, max_ids=1024):
        ids = (C.c_longlong * max_ids)()
        n = C.c_int()
        _check(self._lib.lqcd_engine_completed(self.h, ids, max_ids, C.byref(n)))
        return [ids[i] for i in range(n.value)]

    def result(self, rid, x: Field):
        info = SolveInfo()
        _check(self._lib.lqcd_engine_result(self.h, C.c_longlong(rid), x.h, C.byref(info)))
        return info.as_dict()

    def cancel(self, rid, status=ETIMEOUT):
        _check(self._lib.lqcd_engine_cancel(self.h, C.c_longlong(rid), int(status)))

    def stats(self):
        a = C.c_int()
        b = C.c_size_t()
        _check(self._lib.lqcd_engine_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if self.h:
            self._lib.lqcd_engine_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
