"""Python front end of the exact Gaussian KDE library (marshalling over the C-ABI only).

``ExactGaussianKDE(X, a)`` mirrors the paper's class of the same name (Sec. 5.3 and
App. A): it is built from a data matrix and the bandwidth a, and ``query`` returns the
kernel density of every row of a query matrix,
    K(q) = sum_i exp(-a ||q - x_i||^2)            (normalise=False, the default)
    K(q) = (1/n) sum_i exp(-a ||q - x_i||^2)      (normalise=True, Sec. 3's definition)
``kernel`` selects Sec. 3's other kernel functions of r = ||q - x_i||: "exponential",
exp(-a r), or "logistic", 4 / (2 + exp(a r) + exp(-a r)) (plain FP32 and FP64 forms).
All arithmetic happens in the CUDA kernels behind ``libstagkde.so``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L


def _as_host(a, dtype):
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if arr.ndim == 1:
        arr = arr.reshape(1, -1)
    return arr


class ExactGaussianKDE:
    """Exact Gaussian kernel density over a point set resident on one GPU."""

    def __init__(self, X, a: float, form: str = "auto", normalise: bool = False,
                 device: int | None = None, dtype=None, tc_check: bool = True, kernel: str = "gaussian"):
        lib = L.load()
        try:
            import torch
            if isinstance(X, torch.Tensor):
                X = X.detach().cpu().numpy()
        except ImportError:
            pass
        X = np.asarray(X)
        if dtype is None:
            dtype = np.float64 if X.dtype == np.float64 else np.float32
        self._np_dtype = np.dtype(dtype)
        self._dt = L.F64 if self._np_dtype == np.float64 else L.F32
        Xh = _as_host(X, self._np_dtype)
        opts = L.Opts()
        lib.stag_kde_opts_init(ctypes.byref(opts))
        opts.form = L.FORMS[form]
        opts.normalise = 1 if normalise else 0
        opts.device = -1 if device is None else int(device)
        opts.tc_no_check = 0 if tc_check else 1
        if kernel not in L.KERNELS:
            raise ValueError(f"unknown kernel {kernel!r}; one of {sorted(L.KERNELS)}")
        opts.kernel = L.KERNELS[kernel]
        h = lib.stag_kde_create_ex(Xh.ctypes.data, self._dt, Xh.shape[0], Xh.shape[1], float(a),
                                   ctypes.byref(opts))
        if not h:
            raise L.StagKdeError(lib.stag_kde_last_error_code() or L.EINVAL, L.last_error())
        self._h = ctypes.c_void_p(h)
        self._lib = lib
        self.n, self.d, self.a = int(Xh.shape[0]), int(Xh.shape[1]), float(a)
        self.kernel = kernel

    @property
    def form(self) -> str:
        f = ctypes.c_int()
        L.check(self._lib.stag_kde_info(self._h, None, None, None, None, ctypes.byref(f)))
        return L.FORM_NAMES[f.value]

    def query(self, Q) -> np.ndarray:
        """Densities of the rows of Q (host array) as float64, synchronously."""
        Qh = _as_host(Q, self._np_dtype)
        if Qh.shape[1] != self.d:
            raise ValueError(f"Q has d={Qh.shape[1]}, the data has d={self.d}")
        out = np.empty(Qh.shape[0], dtype=np.float64)
        L.check(self._lib.stag_kde_query(self._h, Qh.ctypes.data, Qh.shape[0], out.ctypes.data))
        return out

    def query_dev(self, Q, out=None, stream=None):
        """Queues the densities of the rows of the CUDA tensor Q into the CUDA float64
        tensor ``out`` on ``stream`` (a torch.cuda.Stream, default: the current one)."""
        import torch
        if not (isinstance(Q, torch.Tensor) and Q.is_cuda and Q.is_contiguous()):
            raise ValueError("Q must be a contiguous CUDA tensor")
        if Q.dim() != 2 or Q.shape[1] != self.d:
            raise ValueError("Q must be m x d")
        want = torch.float64 if self._dt == L.F64 else torch.float32
        if Q.dtype != want:
            raise ValueError(f"Q must be {want}")
        m = Q.shape[0]
        if out is None:
            out = torch.empty(m, dtype=torch.float64, device=Q.device)
        if out.dtype != torch.float64 or not out.is_cuda or out.numel() < m:
            raise ValueError("out must be a CUDA float64 tensor with m entries")
        s = stream if stream is not None else torch.cuda.current_stream(Q.device)
        L.check(self._lib.stag_kde_query_dev(self._h, Q.data_ptr(), m, out.data_ptr(),
                                             ctypes.c_void_p(s.cuda_stream)))
        return out

    def set_wait_limit(self, limit_ns: int):
        """Limit of each bounded wait in the tensor-core kernel (0: the default, 2 s)."""
        L.check(self._lib.stag_kde_set_wait_limit(self._h, int(limit_ns)))

    def last_recomputed(self) -> int:
        """Queries of the last call that the tensor-core error estimate sent to FP32."""
        c = ctypes.c_int64()
        L.check(self._lib.stag_kde_last_recomputed(self._h, ctypes.byref(c)))
        return c.value

    def profile_begin(self):
        L.check(self._lib.stag_kde_profile_begin(self._h))

    def profile_end(self):
        """(summed main-kernel ms, launches, pairs) since profile_begin (event-timed)."""
        ms, n, pairs = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        L.check(self._lib.stag_kde_profile_end(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(pairs)))
        return ms.value, n.value, pairs.value

    def query_subset(self, Q, offsets, idx, W=None) -> np.ndarray:
        """Weighted subset sums (Sec. 3.1): out[j] = sum over query j's list entries
        p = offsets[j] .. offsets[j+1]-1 of W[p] k(||q_j - x_{idx[p]}||) (W None: all 1),
        host arrays, synchronous."""
        Qh = _as_host(Q, np.float32)
        if Qh.shape[1] != self.d:
            raise ValueError(f"Q has d={Qh.shape[1]}, the data has d={self.d}")
        m = Qh.shape[0]
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int64))
        if off.shape != (m + 1,):
            raise ValueError("offsets must have m + 1 entries")
        w = None if W is None else np.ascontiguousarray(np.asarray(W, dtype=np.float32))
        out = np.empty(m, dtype=np.float64)
        L.check(self._lib.stag_kde_query_subset(self._h, Qh.ctypes.data, m, off.ctypes.data,
                                                ix.ctypes.data if ix.size else None,
                                                None if w is None else w.ctypes.data, out.ctypes.data))
        return out

    def query_subset_dev(self, Q, offsets, idx, W=None, out=None, stream=None):
        """Device variant of query_subset on CUDA tensors (Q float32 m x d, offsets and
        idx int64, W float32 or None); queued on ``stream``, returns ``out``."""
        import torch
        for t in (Q, offsets, idx) + (() if W is None else (W,)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
                raise ValueError("Q, offsets, idx and W must be contiguous CUDA tensors")
        if Q.dtype != torch.float32 or offsets.dtype != torch.int64 or idx.dtype != torch.int64:
            raise ValueError("Q float32, offsets and idx int64")
        if W is not None and W.dtype != torch.float32:
            raise ValueError("W must be float32")
        m = Q.shape[0]
        if Q.dim() != 2 or Q.shape[1] != self.d or offsets.numel() != m + 1:
            raise ValueError("Q must be m x d and offsets m + 1 long")
        if out is None:
            out = torch.empty(m, dtype=torch.float64, device=Q.device)
        s = (stream or torch.cuda.current_stream()).cuda_stream
        L.check(self._lib.stag_kde_query_subset_dev(self._h, Q.data_ptr(), m, offsets.data_ptr(),
                                                    idx.data_ptr() if idx.numel() else offsets.data_ptr(),
                                                    None if W is None else W.data_ptr(), out.data_ptr(), s))
        return out

    def degrees(self, exclude_self: bool = False, stream=None):
        """Similarity-graph degrees of the handle's own points (Sec. 4.1), a CUDA tensor."""
        import torch
        out = torch.empty(self.n, dtype=torch.float64, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        L.check(self._lib.stag_kde_degrees(self._h, 1 if exclude_self else 0, out.data_ptr(),
                                           ctypes.c_void_p(s.cuda_stream)))
        return out

    def autotune(self, Q):
        """Tunes the tensor-core launch settings on the CUDA query tensor Q."""
        L.check(self._lib.stag_kde_autotune(self._h, Q.data_ptr(), Q.shape[0]))

    def reserve(self, m: int):
        L.check(self._lib.stag_kde_reserve(self._h, int(m)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stag_kde_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def query_batch(kdes, Qs, outs=None, stream=None):
    """Evaluates ``Qs[i]`` (contiguous CUDA tensors) against ``kdes[i]`` in one batched
    call (one persistent tensor-core launch serving every operand width, replayed from a
    captured CUDA graph on repeated calls with the same tensors). Returns the output tensors."""
    import torch
    lib = L.load()
    n = len(kdes)
    if outs is None:
        outs = [torch.empty(q.shape[0], dtype=torch.float64, device=q.device) for q in Qs]
    hs = (ctypes.c_void_p * n)(*[k._h.value for k in kdes])
    qs = (ctypes.c_void_p * n)(*[q.data_ptr() for q in Qs])
    ms = (ctypes.c_int64 * n)(*[q.shape[0] for q in Qs])
    os_ = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    s = stream if stream is not None else torch.cuda.current_stream()
    L.check(lib.stag_kde_query_batch(hs, qs, ms, os_, n, ctypes.c_void_p(s.cuda_stream)))
    return outs
