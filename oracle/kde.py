"""ctypes front end of ``kde_oracle.c`` (FP64 double loop; test infrastructure only).

Every function converts its inputs to contiguous float64 (exact for float32 inputs)
and calls the C double loop. ``kde`` is the plain definition of Sec. 3,
K(q) = sum_i exp(-a ||q - x_i||^2) (unnormalised; multiply by 1/n for the paper's
normalised form). ``avg_rel_err`` is the paper's accuracy metric of Sec. 6.1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kde_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libkdeoracle.so")
_SRC_LSH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lsh_oracle.c")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math: IEEE double, libm exp)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    srcs = [_SRC, _SRC_LSH]
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(os.path.getmtime(p) for p in srcs):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
                        "-o", tmp, *srcs, "-lm", "-lpthread"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, c_int, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.oracle_kde.argtypes = [_D, i64, _D, i64, i64, dbl, _D, c_int]
            lib.oracle_kde_weighted.argtypes = [_D, _D, i64, _D, i64, i64, dbl, _D, c_int]
            lib.oracle_kde_self.argtypes = [_D, i64, i64, dbl, _D, c_int]
            lib.oracle_kde_log.argtypes = [_D, i64, _D, i64, i64, dbl, _D, _D, _D, c_int]
            lib.oracle_kde_kernel.argtypes = [c_int, _D, i64, _D, i64, i64, dbl, _D, c_int]
            _I = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_kde_subset.argtypes = [c_int, _D, i64, _D, i64, i64, dbl, _I, _I, _D, _D, c_int]
            for f in (lib.oracle_kde, lib.oracle_kde_weighted, lib.oracle_kde_self, lib.oracle_kde_log,
                      lib.oracle_kde_kernel, lib.oracle_kde_subset):
                f.restype = c_int
            F, I32 = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)
            lib.oracle_lsh_hash.argtypes = [F, i64, i64, i64, F, F, I32]
            lib.oracle_lsh_hash.restype = c_int
            lib.oracle_lsh_candidates.argtypes = [I32, i64, I32, i64, c_int, c_int, _I, _I, i64]
            lib.oracle_lsh_candidates.restype = i64
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _threads(threads):
    return int(threads) if threads else (os.cpu_count() or 1)


def _check(X, Q):
    X = _f64(X)
    Q = _f64(Q)
    if X.ndim != 2 or Q.ndim != 2 or X.shape[1] != Q.shape[1]:
        raise ValueError("X (n x d) and Q (m x d) must be 2-D with the same d")
    return X, Q


def kde(X, Q, a: float, threads: int | None = None) -> np.ndarray:
    """K(q_j) = sum_i exp(-a ||q_j - x_i||^2) for every row q_j of Q (FP64)."""
    X, Q = _check(X, Q)
    out = np.empty(Q.shape[0], dtype=np.float64)
    rc = _load().oracle_kde(_p(X), X.shape[0], _p(Q), Q.shape[0], X.shape[1], float(a), _p(out),
                            _threads(threads))
    if rc:
        raise ValueError("oracle_kde rejected its arguments")
    return out


def kde_weighted(X, W, Q, a: float, threads: int | None = None) -> np.ndarray:
    """sum_i w_i exp(-a ||q_j - x_i||^2) (the subset estimators' inner sum)."""
    X, Q = _check(X, Q)
    W = _f64(W).reshape(-1)
    if W.shape[0] != X.shape[0]:
        raise ValueError("W must have n entries")
    out = np.empty(Q.shape[0], dtype=np.float64)
    rc = _load().oracle_kde_weighted(_p(X), _p(W), X.shape[0], _p(Q), Q.shape[0], X.shape[1],
                                     float(a), _p(out), _threads(threads))
    if rc:
        raise ValueError("oracle_kde_weighted rejected its arguments")
    return out


KERNELS = {"gaussian": 0, "exponential": 1, "logistic": 2}


def kde_kernel(X, Q, a: float, kernel: str = "gaussian", threads: int | None = None) -> np.ndarray:
    """sum_i k(||q - x_i||) in FP64 for the kernel functions of Sec. 3: "gaussian"
    exp(-a r^2), "exponential" exp(-a r), "logistic" 4 / (2 + exp(a r) + exp(-a r))."""
    X, Q = _check(X, Q)
    out = np.empty(Q.shape[0], dtype=np.float64)
    rc = _load().oracle_kde_kernel(KERNELS[kernel], _p(X), X.shape[0], _p(Q), Q.shape[0], X.shape[1],
                                   float(a), _p(out), _threads(threads))
    if rc:
        raise ValueError(f"oracle_kde_kernel failed ({rc})")
    return out


def kde_subset(X, Q, a: float, offsets, idx, W=None, kernel: str = "gaussian",
               threads: int | None = None) -> np.ndarray:
    """out_j = sum over query j's list entries p = offsets[j] .. offsets[j+1]-1 of
    W[p] k(||q_j - x_{idx[p]}||) (W = None: weights 1), in list order (Sec. 3.1)."""
    X, Q = _check(X, Q)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
    if off.shape != (Q.shape[0] + 1,) or ix.shape != (int(off[-1]) if len(off) else 0,):
        raise ValueError("offsets must have m + 1 entries and idx offsets[-1]")
    w = None if W is None else _f64(W)
    if w is not None and w.shape != ix.shape:
        raise ValueError("W must match idx")
    out = np.empty(Q.shape[0], dtype=np.float64)
    I = ctypes.POINTER(ctypes.c_int64)
    rc = _load().oracle_kde_subset(KERNELS[kernel], _p(X), X.shape[0], _p(Q), Q.shape[0], X.shape[1], float(a),
                                   off.ctypes.data_as(I), ix.ctypes.data_as(I), None if w is None else _p(w),
                                   _p(out), _threads(threads))
    if rc:
        raise ValueError(f"oracle_kde_subset failed ({rc})")
    return out


def lsh_hash(X, A, B) -> np.ndarray:
    """E2LSH hash values floor((<x, a_f> + b_f) / 4) of the rows of X under the functions
    (rows of A, offsets B), taken in FP32 (fused multiply-adds in coordinate order), as an
    n x nf int32 array (Sec. 2)."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float32))
    B = np.ascontiguousarray(np.asarray(B, dtype=np.float32)).reshape(-1)
    if X.ndim != 2 or A.ndim != 2 or A.shape[1] != X.shape[1] or B.shape[0] != A.shape[0]:
        raise ValueError("X (n x d), A (nf x d), B (nf)")
    H = np.empty((X.shape[0], A.shape[0]), dtype=np.int32)
    F, I32 = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)
    rc = _load().oracle_lsh_hash(X.ctypes.data_as(F), X.shape[0], X.shape[1], A.shape[0], A.ctypes.data_as(F),
                                 B.ctypes.data_as(F), H.ctypes.data_as(I32))
    if rc:
        raise ValueError("oracle_lsh_hash failed")
    return H


def lsh_candidates(HX, HQ, K: int, L: int):
    """Near-neighbour lists (Sec. 2): for each query row of HQ, the distinct indices i, in
    increasing order, whose K hash values equal the query's in at least one of the L
    tables. Returns (offsets[m + 1], idx)."""
    HX = np.ascontiguousarray(HX, dtype=np.int32)
    HQ = np.ascontiguousarray(HQ, dtype=np.int32)
    if HX.shape[1] != K * L or HQ.shape[1] != K * L:
        raise ValueError("hash arrays must have K * L columns")
    lib = _load()
    I32, I = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    off = np.empty(HQ.shape[0] + 1, dtype=np.int64)
    total = lib.oracle_lsh_candidates(HX.ctypes.data_as(I32), HX.shape[0], HQ.ctypes.data_as(I32), HQ.shape[0],
                                      K, L, off.ctypes.data_as(I), None, 0)
    idx = np.empty(max(total, 1), dtype=np.int64)
    lib.oracle_lsh_candidates(HX.ctypes.data_as(I32), HX.shape[0], HQ.ctypes.data_as(I32), HQ.shape[0],
                              K, L, off.ctypes.data_as(I), idx.ctypes.data_as(I), total)
    return off, idx[:total]


def kde_self(X, a: float, threads: int | None = None) -> np.ndarray:
    """deg(i) = sum_{j != i} exp(-a ||x_i - x_j||^2) (similarity-graph degrees, Sec. 4)."""
    X = _f64(X)
    out = np.empty(X.shape[0], dtype=np.float64)
    rc = _load().oracle_kde_self(_p(X), X.shape[0], X.shape[1], float(a), _p(out), _threads(threads))
    if rc:
        raise ValueError("oracle_kde_self rejected its arguments")
    return out


def kde_log(X, Q, a: float, threads: int | None = None):
    """(log K, d2min, kappa) per query, exact even when every term underflows double."""
    X, Q = _check(X, Q)
    m = Q.shape[0]
    logk, d2min, kappa = (np.empty(m, dtype=np.float64) for _ in range(3))
    rc = _load().oracle_kde_log(_p(X), X.shape[0], _p(Q), m, X.shape[1], float(a), _p(logk),
                                _p(d2min), _p(kappa), _threads(threads))
    if rc:
        raise ValueError("oracle_kde_log rejected its arguments")
    return logk, d2min, kappa


def rel_err(est, ref) -> np.ndarray:
    """|est - ref| / |ref| per query (0 where both are 0)."""
    est = np.asarray(est, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    diff = np.abs(est - ref)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(ref != 0, diff / np.abs(ref), np.where(diff == 0, 0.0, np.inf))
    return r


def avg_rel_err(est, ref) -> float:
    """The paper's accuracy metric (Sec. 6.1): (1/m) sum_i |mu_i - mu_i*| / mu_i*."""
    return float(np.mean(rel_err(est, ref)))
