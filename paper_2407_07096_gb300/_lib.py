"""ctypes binding of the C-ABI in include/stag_kde.h (argument marshalling only).

The shared library is built in-tree by ``paper_2407_07096_gb300.build``. Loading fails
loudly if it is missing: there is no CPU fallback anywhere in the package.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

OK = 0
EINVAL, ENOMEM, ECUDA, ETIMEDOUT, ECANCELED, EUNSUPPORTED = -1, -2, -3, -4, -5, -6
F32, F64 = 0, 1
FORM_AUTO, FORM_SIMT_F32, FORM_TC, FORM_SIMT_F64 = 0, 1, 2, 3
FORM_NAMES = {FORM_AUTO: "auto", FORM_SIMT_F32: "simt_f32", FORM_TC: "tc", FORM_SIMT_F64: "simt_f64"}
FORMS = {v: k for k, v in FORM_NAMES.items()}
KERNEL_GAUSSIAN, KERNEL_EXPONENTIAL, KERNEL_LOGISTIC = 0, 1, 2
KERNELS = {"gaussian": KERNEL_GAUSSIAN, "exponential": KERNEL_EXPONENTIAL, "logistic": KERNEL_LOGISTIC}


class StagKdeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"stag_kde error {code}: {msg}")
        self.code = code


class SrvOpts(ctypes.Structure):
    _fields_ = [("datasets", ctypes.POINTER(ctypes.c_void_p)), ("n_datasets", ctypes.c_int),
                ("slots", ctypes.c_int), ("max_rows", ctypes.c_int64), ("mem_budget_bytes", ctypes.c_int64),
                ("reserved", ctypes.c_int * 4)]


class Opts(ctypes.Structure):
    _fields_ = [("form", ctypes.c_int), ("normalise", ctypes.c_int), ("device", ctypes.c_int),
                ("tc_no_check", ctypes.c_int), ("kernel", ctypes.c_int), ("reserved", ctypes.c_int * 3)]


# (name, restype, argtypes) for every entry point declared in include/stag_kde.h
_VP, _I64, _INT, _DBL = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
SIGNATURES = [
    ("stag_kde_opts_init", None, [ctypes.POINTER(Opts)]),
    ("stag_kde_create", _VP, [_VP, _I64, _I64, _DBL]),
    ("stag_kde_create_ex", _VP, [_VP, _INT, _I64, _I64, _DBL, ctypes.POINTER(Opts)]),
    ("stag_kde_query", _INT, [_VP, _VP, _I64, _VP]),
    ("stag_kde_query_dev", _INT, [_VP, _VP, _I64, _VP, _VP]),
    ("stag_kde_set_wait_limit", _INT, [_VP, _I64]),
    ("stag_kde_probe_ex2", _INT, [_I64, _VP, _VP]),
    ("stag_kde_query_subset", _INT, [_VP, _VP, _I64, _VP, _VP, _VP, _VP]),
    ("stag_kde_query_subset_dev", _INT, [_VP, _VP, _I64, _VP, _VP, _VP, _VP, _VP]),
    ("stag_lsh_create", _VP, [_VP, _I64, _I64, _INT, _INT, _VP, _VP, _INT]),
    ("stag_lsh_hash_dev", _INT, [_VP, _VP, _I64, _VP, _VP]),
    ("stag_lsh_query", _INT, [_VP, _VP, _I64, _VP, _VP, _I64, _VP]),
    ("stag_lsh_query_dev", _INT, [_VP, _VP, _I64, _VP, _VP, _I64, _VP, _VP]),
    ("stag_lsh_fetch", _INT, [_VP, _VP, _I64]),
    ("stag_lsh_fetch_dev", _INT, [_VP, _VP, _I64, _VP]),
    ("stag_lsh_info", _INT, [_VP, _VP, _VP, _VP, _VP]),
    ("stag_lsh_destroy", None, [_VP]),
    ("stag_kde_reserve", _INT, [_VP, _I64]),
    ("stag_kde_query_batch", _INT, [ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_I64),
                                    ctypes.POINTER(_VP), _I64, _VP]),
    ("stag_kde_autotune", _INT, [_VP, _VP, _I64]),
    ("stag_kde_degrees", _INT, [_VP, _INT, _VP, _VP]),
    ("stag_kde_info", _INT, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_DBL),
                             ctypes.POINTER(_INT), ctypes.POINTER(_INT)]),
    ("stag_kde_destroy", None, [_VP]),
    ("stag_kde_last_recomputed", _INT, [_VP, ctypes.POINTER(_I64)]),
    ("stag_kde_last_error", ctypes.c_char_p, []),
    ("stag_kde_last_error_code", _INT, []),
    ("stag_kde_version", ctypes.c_char_p, []),
    ("stag_kde_launch_count", ctypes.c_uint64, []),
    ("stag_kde_profile_begin", _INT, [_VP]),
    ("stag_srv_opts_init", None, [ctypes.POINTER(SrvOpts)]),
    ("stag_srv_start", _VP, [ctypes.POINTER(SrvOpts)]),
    ("stag_srv_submit", _INT, [_VP, _INT, _VP, _I64, _VP, ctypes.POINTER(ctypes.c_uint64)]),
    ("stag_srv_wait", _INT, [_VP, ctypes.c_uint64, _I64]),
    ("stag_srv_cancel", _INT, [_VP, ctypes.c_uint64]),
    ("stag_srv_stats", _INT, [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_DBL),
                              ctypes.POINTER(_DBL)]),
    ("stag_srv_reset_stats", _INT, [_VP]),
    ("stag_srv_stop", _INT, [_VP]),
    ("stag_kde_eval_noalloc", _INT, [_VP, _I64, _VP, _I64, _I64, _DBL, _VP, _VP]),
    ("stag_kde_profile_end", _INT, [_VP, ctypes.POINTER(_DBL), ctypes.POINTER(_I64), ctypes.POINTER(_DBL)]),
]


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Loads the library (never builds it implicitly: call ``build.build()`` first)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or os.environ.get("STAG_KDE_LIB") or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built ({p} missing): run __graft_entry__.build() "
                               "or python -m paper_2407_07096_gb300.build")
        lib = ctypes.CDLL(p)
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        if path is None:
            _lib = lib
        return lib


def last_error() -> str:
    return load().stag_kde_last_error().decode()


def check(rc: int) -> int:
    if rc != OK:
        raise StagKdeError(rc, last_error())
    return rc
