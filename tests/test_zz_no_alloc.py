"""The allocation-free entry point (stag_kde_eval_noalloc) against the handle API.

It is for callers that cannot allocate device memory at call time; it keeps its
scratch in a fixed array inside the library. This file is named so that pytest runs it
last: a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
from tests._common import mixture_inputs, tol_f32

pytestmark = pytest.mark.gpu


def test_noalloc_matches_handle_api_on_two_calls_in_a_row():
    import torch
    from paper_2407_07096_gb300 import build, _lib as L
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    build.build()
    lib = L.load()
    X, Q = mixture_inputs(21, 5003, 1031, 16)
    a = 0.2
    dX = torch.from_numpy(X).cuda()
    dQ = torch.from_numpy(Q).cuda()
    with ExactGaussianKDE(X, a, form="simt_f32") as kde:
        want = kde.query_dev(dQ).cpu().numpy()
    stream = torch.cuda.current_stream()
    ref = oracle.kde(X, Q, a)
    _, _, kappa = oracle.kde_log(X, Q, a)
    tol = tol_f32(kappa, X.shape[1])
    for _ in range(2):
        out = torch.full((len(Q),), -1.0, dtype=torch.float64, device="cuda")
        rc = lib.stag_kde_eval_noalloc(dX.data_ptr(), X.shape[0], dQ.data_ptr(), Q.shape[0], X.shape[1], a,
                                       out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.last_error()
        got = out.cpu().numpy()
        assert np.all(oracle.rel_err(got, want) <= tol)
        assert np.all(oracle.rel_err(got, ref) <= tol)


def test_noalloc_rejects_m_beyond_its_scratch():
    import torch
    from paper_2407_07096_gb300 import build, _lib as L
    build.build()
    lib = L.load()
    d = 2
    m = 699051
    dX = torch.zeros((4, d), dtype=torch.float32, device="cuda")
    dQ = torch.zeros((m, d), dtype=torch.float32, device="cuda")
    out = torch.empty(m, dtype=torch.float64, device="cuda")
    rc = lib.stag_kde_eval_noalloc(dX.data_ptr(), 4, dQ.data_ptr(), m, d, 1.0, out.data_ptr(), None)
    assert rc == L.EINVAL and "scratch" in L.last_error()
