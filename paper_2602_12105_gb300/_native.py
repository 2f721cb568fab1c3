"""ctypes binding of libiskra_gb300.so (include/iskra_gb300.h): argument marshalling only.

The library is loaded on first use; if it is missing or cannot be loaded an ImportError-like
NativeLibraryError is raised. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
# ISKRA_GB300_CHECK=1 selects the bounds-checked build (libiskra_gb300_check.so, -DIG_CHECK)
CHECKED = os.environ.get("ISKRA_GB300_CHECK", "0") not in ("", "0")
LIB_PATH = os.path.join(HERE, "libiskra_gb300_check.so" if CHECKED else "libiskra_gb300.so")

IG_OK = 0
IG_ERR_INVALID_ARG = 1
IG_ERR_INDEX_OUT_OF_RANGE = 2
IG_ERR_DEGENERATE_FACE = 3
IG_ERR_NOT_CONVERGED = 4
IG_ERR_NONFINITE = 5
IG_ERR_OOM = 6
IG_ERR_CUDA = 7
IG_ERR_STATE = 8

IG_PRECISION_FP64 = 0
IG_PRECISION_MIXED = 1
IG_PRECISION_MIXED_GEOM32 = 2
IG_LAUNCH_GRAPH = 0
IG_LAUNCH_HOST = 1


class NativeLibraryError(RuntimeError):
    pass


class IgError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("launch", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("k", ctypes.c_int), ("iterations", ctypes.c_int),
                ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double * 4),
                ("true_rel_residual", ctypes.c_double * 4)]

    def as_dict(self):
        k = self.k
        return {"status": self.status, "k": k, "iterations": self.iterations, "refinements": self.refinements,
                "rel_residual": list(self.rel_residual[:k]), "true_rel_residual": list(self.true_rel_residual[:k])}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


_vp, _i32, _i64, _dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_P = ctypes.POINTER

# name -> (restype, argtypes); the declarations of include/iskra_gb300.h
SIGNATURES = {
    "ig_status_str": (ctypes.c_char_p, [_i32]),
    "ig_default_opts": (None, [_P(SolveOpts)]),
    "ig_create": (_i32, [_P(_vp), _i32, _vp]),
    "ig_set_stream": (_i32, [_vp, _vp]),
    "ig_destroy": (_i32, [_vp]),
    "ig_last_error": (ctypes.c_char_p, [_vp]),
    "ig_mesh_upload": (_i32, [_vp, _vp, _i64, _i64, _P(_vp)]),
    "ig_mesh_free": (_i32, [_vp]),
    "ig_mesh_info": (_i32, [_vp, _P(_i64), _P(_i64), _P(_i64), _P(_i64)]),
    "ig_mesh_pattern": (_i32, [_vp, _vp, _vp]),
    "ig_assemble": (_i32, [_vp, _vp, _dbl, _i32]),
    "ig_check": (_i32, [_vp]),
    "ig_operator": (_i32, [_vp, _vp, _vp]),
    "ig_operator32": (_i32, [_vp, _vp]),
    "ig_solve": (_i32, [_vp, _vp, _i32, _vp, _P(SolveOpts), _P(SolveInfo)]),
    "ig_adjoint": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp, _vp, _P(SolveOpts), _P(SolveInfo)]),
    "ig_batch_create": (_i32, [_vp, _P(_vp), _i32, _P(_vp)]),
    "ig_batch_free": (_i32, [_vp]),
    "ig_batch_assemble": (_i32, [_vp, _P(_vp), _P(_dbl), _i32]),
    "ig_batch_solve": (_i32, [_vp, _P(_vp), _i32, _P(_vp), _P(SolveOpts), _P(SolveInfo)]),
    "ig_batch_adjoint": (_i32, [_vp, _P(_vp), _P(_vp), _i32, _P(_vp), _P(_vp), _i32, _P(_vp), _P(_vp), _vp,
                                _P(SolveOpts), _P(SolveInfo)]),
    "ig_solve_begin": (_i32, [_vp, _vp, _i32, _i32, _P(SolveOpts)]),
    "ig_batch_iterate": (_i32, [_vp, _i32, _i32, _P(_i32)]),
    "ig_solve_end": (_i32, [_vp, _i32, _vp, _P(SolveInfo)]),
    "ig_vjp": (_i32, [_vp, _vp, _vp, _i32, _vp, _i32, _vp, _vp, _vp]),
    "ig_mass_vjp": (_i32, [_vp, _vp, _vp, _vp]),
    "ig_fairing_step": (_i32, [_vp, _vp, _vp, _dbl, _dbl, _i32, _P(SolveOpts), _P(_dbl), _P(SolveInfo)]),
    "ig_eigs": (_i32, [_vp, _i32, _i32, _vp, _P(_dbl), _P(SolveOpts), _P(SolveInfo)]),
    "ig_eigs_vjp": (_i32, [_vp, _vp, _i32, _i32, _vp, _vp, _vp, _P(SolveOpts)]),
    "ig_rgd_u_step": (_i32, [_vp, _vp, _P(_i32), _i32, _vp, _vp, _dbl, _dbl, _vp, _P(SolveOpts), _P(SolveInfo)]),
    "ig_rgd_u_step_vjp": (_i32, [_vp, _vp, _P(_i32), _i32, _vp, _vp, _dbl, _dbl, _vp, _vp, _vp, _vp, _vp,
                                 _P(SolveOpts)]),
    "ig_rgd_admm": (_i32, [_vp, _vp, _P(_i32), _i32, _dbl, _dbl, _dbl, _i32, _dbl, _i32, _vp, _vp, _vp, _P(_dbl),
                           _P(SolveOpts)]),
    "ig_rgd_admm_vjp": (_i32, [_vp, _vp, _P(_i32), _i32, _dbl, _dbl, _dbl, _vp, _vp, _vp, _i32, _i32, _dbl, _vp, _vp,
                               _P(_dbl), _P(SolveOpts)]),
    "ig_solve_csr_noalloc": (_i32, [_vp, _vp, _vp, _vp, _i64, _i64, _vp, _i32, _vp, _vp, _P(SolveOpts),
                                     _P(SolveInfo)]),
    "ig_profile_enable": (_i32, [_i32]),
    "ig_profile_read": (_i32, [_P(KernelStat), _i32]),
    "ig_measure_fma_peak": (_i32, [_i32, _i32, _vp, _P(_dbl), _P(_dbl)]),
    "ig_mesh_set_cot_clamp": (_i32, [_vp, _i32, _dbl]),
}

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load the native library (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path) or (CHECKED and path == LIB_PATH):
            try:
                from . import build as _build
                _build.build(checked=CHECKED and path == LIB_PATH)
            except Exception as exc:  # noqa: BLE001 - re-raised with context
                raise NativeLibraryError(f"libiskra_gb300.so is missing and could not be built: {exc}") from exc
        try:
            lib = ctypes.CDLL(path)
        except OSError as exc:
            raise NativeLibraryError(f"cannot load {path}: {exc}") from exc
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_str(status: int) -> str:
    return load().ig_status_str(status).decode()


def check(status: int, ctx=None):
    if status != IG_OK:
        msg = ""
        if ctx is not None:
            msg = load().ig_last_error(ctx).decode()
        raise IgError(status, f"{status_str(status)}: {msg}" if msg else status_str(status))


def profile_enable(on: bool = True):
    load().ig_profile_enable(1 if on else 0)


def measure_fma_peak(fp64: bool = True, steps: int = 0, stream=None):
    """(flops/s, seconds) of the FMA-throughput kernel (see ig_measure_fma_peak) on `stream` (a
    cudaStream_t as an int, or None for the legacy default stream)."""
    lib = load()
    if steps <= 0:
        steps = 50000 if fp64 else 1000000
    rate, secs = ctypes.c_double(0.0), ctypes.c_double(0.0)
    check(lib.ig_measure_fma_peak(IG_PRECISION_FP64 if fp64 else IG_PRECISION_MIXED, int(steps),
                                  ctypes.c_void_p(stream) if stream else None, ctypes.byref(rate),
                                  ctypes.byref(secs)))
    return rate.value, secs.value


def profile_read():
    """{kernel name: (launches, total device ms)} accumulated since profile_enable."""
    lib = load()
    cnt = lib.ig_profile_read(None, 0)
    arr = (KernelStat * max(cnt, 1))()
    cnt = lib.ig_profile_read(arr, cnt)
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms)) for i in range(cnt)}
