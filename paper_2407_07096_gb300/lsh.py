"""Python front end of the GPU E2LSH tables (Sec. 2), marshalling over the C-ABI only.

``E2LSH(X, K, L)`` builds L hash tables of K functions h(x) = floor((<x, a> + b) / 4)
over the rows of X; ``query`` returns every query's distinct near-neighbour candidates
(points sharing its bucket in at least one table) as CSR lists, the input the weighted
subset sums (``ExactGaussianKDE.query_subset``) take. The random functions are drawn on
the host by the package's seeded generator (a ~ N(0, I), b ~ U(0, 4)) unless given, and
passed to the library as inputs.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L
from . import datagen as G

S_LSH_A, S_LSH_B = 21, 22  # generator streams of the functions


def draw_functions(d: int, K: int, Lt: int, seed: int = 0):
    """L*K functions for d-dimensional data: A (L*K x d) ~ N(0, I), B (L*K) ~ U(0, 4), FP32."""
    nf = K * Lt
    A = G.normal(seed, S_LSH_A, nf * d).reshape(nf, d).astype(np.float32)
    B = (4.0 * G.uniform(seed, S_LSH_B, nf)).astype(np.float32)
    return A, B


class E2LSH:
    """Euclidean locality-sensitive hash tables over a point set resident on one GPU."""

    def __init__(self, X, K: int, L_tables: int, A=None, B=None, seed: int = 0, device: int | None = None):
        lib = L.load()
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        if X.ndim != 2:
            raise ValueError("X must be n x d")
        n, d = X.shape
        if A is None:
            A, B = draw_functions(d, K, L_tables, seed)
        A = np.ascontiguousarray(np.asarray(A, dtype=np.float32))
        B = np.ascontiguousarray(np.asarray(B, dtype=np.float32)).reshape(-1)
        if A.shape != (K * L_tables, d) or B.shape != (K * L_tables,):
            raise ValueError("A must be (K*L) x d and B K*L long")
        h = lib.stag_lsh_create(X.ctypes.data, n, d, int(K), int(L_tables), A.ctypes.data, B.ctypes.data,
                                -1 if device is None else int(device))
        if not h:
            raise L.StagKdeError(lib.stag_kde_last_error_code() or L.EINVAL, L.last_error())
        self._h = ctypes.c_void_p(h)
        self._lib = lib
        self.n, self.d, self.K, self.L = n, d, int(K), int(L_tables)
        self.A, self.B = A, B

    def hash_dev(self, Q, out=None, stream=None):
        """Hash values (m x K*L int32, CUDA) of the rows of the CUDA float32 tensor Q."""
        import torch
        if not (isinstance(Q, torch.Tensor) and Q.is_cuda and Q.is_contiguous() and Q.dtype == torch.float32):
            raise ValueError("Q must be a contiguous CUDA float32 tensor")
        if out is None:
            out = torch.empty((Q.shape[0], self.K * self.L), dtype=torch.int32, device=Q.device)
        s = (stream or torch.cuda.current_stream()).cuda_stream
        L.check(self._lib.stag_lsh_hash_dev(self._h, Q.data_ptr(), Q.shape[0], out.data_ptr(), s))
        return out

    def query(self, Q, out=None):
        """(offsets[m + 1], idx) of every query's distinct candidates, host arrays.

        out: optional (offsets, idx) host int64 arrays to fill, for instance in pinned
        memory so that the lists come back at full copy bandwidth: offsets of at least
        m + 1 entries, idx of any size (used when it holds every candidate, otherwise a
        new array is made). The returned arrays are then views of them."""
        Qh = np.ascontiguousarray(np.asarray(Q, dtype=np.float32))
        if Qh.ndim != 2 or Qh.shape[1] != self.d:
            raise ValueError("Q must be m x d")
        m = Qh.shape[0]
        if out is None:
            off, buf = np.zeros(m + 1, dtype=np.int64), None
        else:
            off, buf = out
            for a in (off, buf):
                if a.dtype != np.int64 or a.ndim != 1 or not a.flags.c_contiguous:
                    raise ValueError("out arrays must be contiguous 1-D int64")
            if off.size < m + 1:
                raise ValueError("out offsets need m + 1 entries")
            off = off[: m + 1]
        total = ctypes.c_int64()
        cap = buf.size if buf is not None else 0
        L.check(self._lib.stag_lsh_query(self._h, Qh.ctypes.data, m, off.ctypes.data,
                                         buf.ctypes.data if cap else None, cap, ctypes.byref(total)))
        if buf is not None and cap >= total.value:
            return off, buf[: total.value]
        idx = np.empty(max(total.value, 1), dtype=np.int64)
        if total.value:  # the lists the call kept, without recomputing them
            L.check(self._lib.stag_lsh_fetch(self._h, idx.ctypes.data, idx.size))
        return off, idx[: total.value]

    def query_dev(self, Q, stream=None):
        """(offsets, idx) CUDA int64 tensors of every query's distinct candidates."""
        import torch
        if not (isinstance(Q, torch.Tensor) and Q.is_cuda and Q.is_contiguous() and Q.dtype == torch.float32):
            raise ValueError("Q must be a contiguous CUDA float32 tensor")
        m = Q.shape[0]
        off = torch.zeros(m + 1, dtype=torch.int64, device=Q.device)
        total = ctypes.c_int64()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        L.check(self._lib.stag_lsh_query_dev(self._h, Q.data_ptr(), m, off.data_ptr(), None, 0,
                                             ctypes.byref(total), s))
        idx = torch.empty(max(total.value, 1), dtype=torch.int64, device=Q.device)
        L.check(self._lib.stag_lsh_fetch_dev(self._h, idx.data_ptr(), idx.numel(), s))
        return off, idx[:total.value]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stag_lsh_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
