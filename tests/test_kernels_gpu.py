"""Sec. 3's exponential kernel exp(-a r) and logistic kernel 4 / (2 + e^{ar} + e^{-ar})
(r = ||q - x||) on the plain FP32 and FP64 forms, element by element against the FP64
oracle, plus their routing: AUTO picks the plain form, the tensor-core form refuses.

Tolerance (FP32): the squared distance carries ~sqrt(d) 2^-24 relative error, r half of
that, and a term's relative error is a r times it; kappa is the kernel's condition number
of the dominant terms (sum_i w_i a r_i (tanh(a r_i / 2) for the logistic) / sum_i w_i),
computed here in FP64 from the same inputs, and the bound is tests._common.tol_f32."""
import numpy as np
import pytest

import oracle
from paper_2407_07096_gb300 import datagen as G
from tests._common import mixture_inputs, tol_f32

pytestmark = pytest.mark.gpu


def _kde_cls():
    from paper_2407_07096_gb300 import build
    build.build()
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    return ExactGaussianKDE


def _kappa(X, Q, a, kernel):
    X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
    x2 = (X64 ** 2).sum(1)
    out = np.empty(len(Q64))
    for j0 in range(0, len(Q64), 64):
        q = Q64[j0:j0 + 64]
        # (only the tolerance depends on kappa: the expanded form is accurate enough here)
        d2 = np.maximum((q ** 2).sum(1)[:, None] + x2[None, :] - 2.0 * q @ X64.T, 0.0)
        x = a * np.sqrt(d2)
        if kernel == "exponential":
            w, g = np.exp(-(x - x.min(1, keepdims=True))), x
        else:
            # sech^2(x/2) = 4 e^-x / (1 + e^-x)^2, relative to the row's largest term
            lw = -x - 2.0 * np.log1p(np.exp(-x))
            w = np.exp(lw - lw.max(1, keepdims=True))
            g = x * np.tanh(x / 2)
        out[j0:j0 + 64] = (w * g).sum(1) / w.sum(1)
    return out


@pytest.mark.parametrize("kernel", ["exponential", "logistic"])
@pytest.mark.parametrize("d,a", [(1, 2.0), (3, 0.7), (16, 0.3), (64, 0.1), (100, 0.05)])
def test_plain_fp32_matches_oracle(kernel, d, a):
    K = _kde_cls()
    X, Q = mixture_inputs(7 + d, 2900, 333, d)
    want = oracle.kde_kernel(X, Q, a, kernel)
    with K(X, a, form="simt_f32", kernel=kernel) as kde:
        got = kde.query(Q)
    err = oracle.rel_err(got, want)
    assert np.all(err <= tol_f32(_kappa(X, Q, a, kernel), d)), err.max()


@pytest.mark.parametrize("kernel", ["exponential", "logistic", "gaussian"])
def test_fp64_form_matches_oracle(kernel):
    K = _kde_cls()
    X, Q = mixture_inputs(21, 1500, 200, 6, dtype=np.float64)
    want = oracle.kde_kernel(X, Q, 0.4, kernel)
    with K(X, 0.4, kernel=kernel) as kde:
        assert kde.form == "simt_f64"
        got = kde.query(Q)
    assert oracle.rel_err(got, want).max() <= 1e-12


@pytest.mark.parametrize("kernel", ["exponential", "logistic"])
def test_routing_auto_plain_and_tc_refused(kernel):
    from paper_2407_07096_gb300 import _lib as L
    K = _kde_cls()
    X, _ = mixture_inputs(3, 500, 1, 16)
    with K(X, 0.2, kernel=kernel) as kde:
        assert kde.form == "simt_f32"
    with pytest.raises(L.StagKdeError) as e:
        K(X, 0.2, form="tc", kernel=kernel)
    assert e.value.code == L.EUNSUPPORTED


@pytest.mark.parametrize("kernel", ["exponential", "logistic"])
def test_far_queries_underflow_fp32(kernel):
    # every term below FP32's range (a r ~ 300-600): the per-row shift keeps them
    K = _kde_cls()
    X, Q = mixture_inputs(5, 1200, 64, 4)
    Q = Q + np.float32(40.0)
    a = 12.0
    want = oracle.kde_kernel(X, Q, a, kernel)
    assert want.max() < 1e-100
    with K(X, a, form="simt_f32", kernel=kernel) as kde:
        got = kde.query(Q)
    assert np.all(oracle.rel_err(got, want) <= tol_f32(_kappa(X, Q, a, kernel), 4))


@pytest.mark.parametrize("kernel", ["exponential", "logistic"])
def test_ragged_sizes_normalise_and_zero_bandwidth(kernel):
    K = _kde_cls()
    X, Q = mixture_inputs(9, 4097, 65, 5)
    with K(X, 0.0, form="simt_f32", kernel=kernel) as kde:
        assert np.all(kde.query(Q) == 4097.0)
    want = oracle.kde_kernel(X, Q, 0.9, kernel) / 4097.0
    with K(X, 0.9, form="simt_f32", kernel=kernel, normalise=True) as kde:
        got = kde.query(Q)
        assert kde.query(np.zeros((0, 5), np.float32)).shape == (0,)
    assert np.all(oracle.rel_err(got, want) <= tol_f32(_kappa(X, Q, 0.9, kernel), 5))


@pytest.mark.parametrize("kernel", ["exponential", "logistic"])
def test_degrees_and_batch(kernel):
    import torch
    from paper_2407_07096_gb300.kde import query_batch
    K = _kde_cls()
    X, _ = mixture_inputs(11, 2000, 1, 8)
    a = 0.6
    want = oracle.kde_kernel(X, X, a, kernel)  # includes k(0) = 1 per row
    with K(X, a, kernel=kernel) as kde:
        deg = kde.degrees().cpu().numpy()
        excl = kde.degrees(exclude_self=True).cpu().numpy()
    kap = _kappa(X, X, a, kernel)
    assert np.all(oracle.rel_err(deg, want) <= tol_f32(kap, 8))
    assert np.all(np.abs(excl - (want - 1.0)) / want <= tol_f32(kap, 8))
    # a batch of handles of this kernel: each result bitwise equal to its solo query
    kdes = [K(G.sample(G.make_mixture(s, 3, 8, -3, 3, 1.0), s, 700 + 100 * s, "data"), 0.3 + 0.1 * s,
              kernel=kernel) for s in range(3)]
    Qs = [torch.from_numpy(G.sample(G.make_mixture(s, 3, 8, -3, 3, 1.0), s, 50 + 7 * s, "query")).cuda()
          for s in range(3)]
    outs = [torch.empty(len(q), dtype=torch.float64, device="cuda") for q in Qs]
    query_batch(kdes, Qs, outs)
    torch.cuda.synchronize()
    for kde, q, o in zip(kdes, Qs, outs):
        solo = kde.query(q.cpu().numpy())
        assert np.array_equal(o.cpu().numpy(), solo)
        kde.close()


@pytest.mark.slow
@pytest.mark.parametrize("kernel", ["exponential", "logistic"])
def test_kernels_workload_size_sampled(kernel):
    # the benchmark's kernel-function workload in full (n = m = 100000, d = 16, a = 0.3),
    # 256 sampled queries checked one by one against the oracle
    K = _kde_cls()
    X, Q = G.workload_single_d16(0)
    a = 0.3
    with K(X, a, form="simt_f32", kernel=kernel) as kde:
        got = kde.query(Q)
    rows = np.random.default_rng(6).choice(len(Q), 256, replace=False)
    want = oracle.kde_kernel(X, Q[rows], a, kernel)
    kap = _kappa(X, Q[rows], a, kernel)
    assert np.all(oracle.rel_err(got[rows], want) <= tol_f32(kap, 16))
