"""The allocation-free entry point (stag_kde_eval_noalloc) against the handle API.

It is for callers that cannot allocate device memory at call time (code inside an
allocator callback, loops that must not synchronise the device, fixed memory budgets);
it keeps its scratch in a fixed array inside the library. This file is named so that
pytest runs it last: a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
from tests._common import mixture_inputs, tol_f32

pytestmark = pytest.mark.gpu

MAX_M = 699050  # the documented per-call maximum (8 MiB of partials / 12 bytes)


def _lib():
    from paper_2407_07096_gb300 import build, _lib as L
    build.build()
    return L, L.load()


def _noalloc(lib, dX, n, dQ, m, d, a, out, stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return lib.stag_kde_eval_noalloc(dX.data_ptr(), n, dQ.data_ptr(), m, d, a, out.data_ptr(),
                                     ctypes.c_void_p(s.cuda_stream))


def test_noalloc_matches_handle_api_on_two_calls_in_a_row():
    import torch
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    L, lib = _lib()
    X, Q = mixture_inputs(21, 5003, 1031, 16)
    a = 0.2
    dX = torch.from_numpy(X).cuda()
    dQ = torch.from_numpy(Q).cuda()
    with ExactGaussianKDE(X, a, form="simt_f32") as kde:
        want = kde.query_dev(dQ).cpu().numpy()
    ref = oracle.kde(X, Q, a)
    _, _, kappa = oracle.kde_log(X, Q, a)
    tol = tol_f32(kappa, X.shape[1])
    for _ in range(2):
        out = torch.full((len(Q),), -1.0, dtype=torch.float64, device="cuda")
        rc = _noalloc(lib, dX, X.shape[0], dQ, Q.shape[0], X.shape[1], a, out)
        assert rc == 0, L.last_error()
        got = out.cpu().numpy()
        assert np.all(oracle.rel_err(got, want) <= tol)
        assert np.all(oracle.rel_err(got, ref) <= tol)


@pytest.mark.parametrize("n,m,d", [(5, 3, 2), (5, 3, 130), (700, 70, 33), (1000, 129, 64), (300, 65, 130)])
def test_noalloc_shapes_against_the_oracle(n, m, d):
    # d > 32 runs several coordinate chunks, d = 33 / 130 leave a ragged last chunk, and
    # n, m below one 64-row tile exercise the zero-filled tile edges
    import torch
    L, lib = _lib()
    X, Q = mixture_inputs(n + m + d, n, m, d)
    a = 0.3 / d
    dX, dQ = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    out = torch.full((m,), -1.0, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, dX, n, dQ, m, d, a, out) == 0, L.last_error()
    torch.cuda.synchronize()
    ref = oracle.kde(X, Q, a)
    _, _, kappa = oracle.kde_log(X, Q, a)
    assert np.all(oracle.rel_err(out.cpu().numpy(), ref) <= tol_f32(kappa, d))


def test_noalloc_accepts_the_documented_maximum_m():
    import torch
    L, lib = _lib()
    d, n, a = 2, 200, 0.5
    X, Q = mixture_inputs(5, n, MAX_M, d)
    dX, dQ = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    out = torch.full((MAX_M,), -1.0, dtype=torch.float64, device="cuda")
    assert _noalloc(lib, dX, n, dQ, MAX_M, d, a, out) == 0, L.last_error()
    got = out.cpu().numpy()
    idx = np.linspace(0, MAX_M - 1, 3000).astype(int)
    ref = oracle.kde(X, Q[idx], a)
    _, _, kappa = oracle.kde_log(X, Q[idx], a)
    assert np.all(oracle.rel_err(got[idx], ref) <= tol_f32(kappa, d))


def test_noalloc_rejects_m_beyond_its_scratch():
    import torch
    L, lib = _lib()
    d = 2
    m = MAX_M + 1
    dX = torch.zeros((4, d), dtype=torch.float32, device="cuda")
    dQ = torch.zeros((m, d), dtype=torch.float32, device="cuda")
    out = torch.empty(m, dtype=torch.float64, device="cuda")
    rc = lib.stag_kde_eval_noalloc(dX.data_ptr(), 4, dQ.data_ptr(), m, d, 1.0, out.data_ptr(), None)
    assert rc == L.EINVAL and "scratch" in L.last_error()
