"""Weighted subset sums (Sec. 3.1's sampling estimators) on the GPU against the FP64
oracle's subset sums, element by element: ragged per-query lists with empty lists and
repeated indices, every kernel function, both entry points, edge cases, and sampled
rows at the benchmark's size. The per-term arithmetic is the plain FP32 form's, so the
tolerance is tests._common.tol_f32 with the condition number of each query's own list
(its weighted mean of a d2 for the Gaussian, a r for the others)."""
import numpy as np
import pytest

import oracle
from tests._common import mixture_inputs, tol_f32

pytestmark = pytest.mark.gpu


def _kde_cls():
    from paper_2407_07096_gb300 import build
    build.build()
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    return ExactGaussianKDE


def _ragged(seed, m, n, max_len, empty_every=7):
    r = np.random.default_rng(seed)
    lens = r.integers(0, max_len + 1, size=m)
    lens[::empty_every] = 0
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    idx = r.integers(0, n, size=int(off[-1])).astype(np.int64)
    # some repeated entries next to each other
    if len(idx) > 10:
        idx[1::9] = idx[0:-1:9][: len(idx[1::9])]
    W = r.uniform(0.1, 3.0, size=len(idx)).astype(np.float32)
    return off, idx, W


def _kappa(X, Q, a, off, idx, W, kernel):
    X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
    out = np.zeros(len(Q))
    for j in range(len(Q)):
        ii = idx[off[j]:off[j + 1]]
        if len(ii) == 0:
            continue
        d2 = ((X64[ii] - Q64[j]) ** 2).sum(1)
        g = a * d2 if kernel == "gaussian" else a * np.sqrt(d2)
        w = W[off[j]:off[j + 1]] * np.exp(-(g - g.min()))
        out[j] = (w * g).sum() / w.sum()
    return out


def _check(got, want, kap, d):
    nz = want != 0
    assert np.all(got[~nz] == 0.0)
    err = np.abs(got[nz] - want[nz]) / np.abs(want[nz])
    assert np.all(err <= tol_f32(kap[nz], d)), err.max()


@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "logistic"])
@pytest.mark.parametrize("d,a", [(3, 0.8), (16, 0.1), (64, 0.02)])
def test_subset_matches_oracle(kernel, d, a):
    K = _kde_cls()
    X, Q = mixture_inputs(40 + d, 3000, 257, d)
    off, idx, W = _ragged(d, 257, 3000, 700)
    want = oracle.kde_subset(X, Q, a, off, idx, W, kernel=kernel)
    with K(X, a, form="simt_f32", kernel=kernel) as kde:
        got = kde.query_subset(Q, off, idx, W)
    _check(got, want, _kappa(X, Q, a, off, idx, W, kernel), d)


def test_device_entry_point_and_tensor_core_handle():
    import torch
    K = _kde_cls()
    X, Q = mixture_inputs(5, 5000, 300, 16)
    off, idx, W = _ragged(5, 300, 5000, 400)
    with K(X, 0.1) as kde:  # AUTO: the tensor-core form; subsets gather from its points
        assert kde.form == "tc"
        host = kde.query_subset(Q, off, idx, W)
        dev = kde.query_subset_dev(torch.from_numpy(Q).cuda(), torch.from_numpy(off).cuda(),
                                   torch.from_numpy(idx).cuda(), torch.from_numpy(W).cuda())
        torch.cuda.synchronize()
        ones = kde.query_subset(Q, off, idx)
    assert np.array_equal(dev.cpu().numpy(), host)
    want = oracle.kde_subset(X, Q, 0.1, off, idx, W)
    _check(host, want, _kappa(X, Q, 0.1, off, idx, W, "gaussian"), 16)
    want1 = oracle.kde_subset(X, Q, 0.1, off, idx)
    _check(ones, want1, _kappa(X, Q, 0.1, off, idx, np.ones_like(W), "gaussian"), 16)


def test_full_lists_equal_the_plain_query():
    K = _kde_cls()
    X, Q = mixture_inputs(6, 2048, 64, 8)
    off = np.arange(0, 2048 * 65, 2048, dtype=np.int64)
    idx = np.tile(np.arange(2048, dtype=np.int64), 64)
    with K(X, 0.3, form="simt_f32", normalise=True) as kde:
        sub = kde.query_subset(Q, off, idx)
        full = kde.query(Q)
    assert np.max(np.abs(sub / full - 1)) <= 2e-6


def test_edge_cases_and_validation():
    import torch
    from paper_2407_07096_gb300 import _lib as L
    K = _kde_cls()
    X, Q = mixture_inputs(8, 1000, 9, 5)
    with K(X, 0.5, form="simt_f32") as kde:
        assert kde.query_subset(Q[:0], np.zeros(1, np.int64), np.zeros(0, np.int64)).shape == (0,)
        z = kde.query_subset(Q, np.zeros(10, np.int64), np.zeros(0, np.int64))
        assert np.all(z == 0.0)
        for off, idx, W in ((np.array([0] + [1] * 9), np.array([1000]), None),        # index = n
                            (np.array([0] + [1] * 9), np.array([-1]), None),          # negative index
                            (np.array([1] + [1] * 9), np.array([0]), None),           # off[0] != 0
                            (np.array([0, 2, 1] + [2] * 7), np.array([0, 1]), None),  # decreasing
                            (np.array([0] + [1] * 9), np.array([0]), np.array([-1.0]))):  # negative weight
            with pytest.raises(L.StagKdeError) as e:
                kde.query_subset(Q, off, idx, W)
            assert e.value.code == L.EINVAL
        # a non-finite query coordinate (checked on the device before out is written)
        Qbad = Q.copy()
        Qbad[4, 2] = np.float32(np.inf)
        with pytest.raises(L.StagKdeError) as e:
            kde.query_subset(Qbad, np.array([0] + [1] * 9), np.array([0]))
        assert e.value.code == L.EINVAL
        # device entry point: out-of-range entries contribute nothing
        off = np.array([0, 3, 3, 5, 6, 6, 6, 6, 6, 8], np.int64)
        idx = np.array([0, 1000, 2, -5, 7, 999, 4, 1 << 40], np.int64)
        got = kde.query_subset_dev(torch.from_numpy(Q).cuda(), torch.from_numpy(off).cuda(),
                                   torch.from_numpy(idx).cuda()).cpu().numpy()
        keep = (idx >= 0) & (idx < 1000)
        off_k = np.concatenate([[0], np.cumsum([keep[off[j]:off[j + 1]].sum() for j in range(9)])])
        want = oracle.kde_subset(X, Q, 0.5, off_k, idx[keep])
        _check(got, want, _kappa(X, Q, 0.5, off_k, idx[keep], np.ones(keep.sum()), "gaussian"), 5)


def test_far_queries_underflow():
    K = _kde_cls()
    X, Q = mixture_inputs(9, 1500, 40, 16)
    Q = Q + np.float32(30.0)
    off, idx, W = _ragged(9, 40, 1500, 300)
    want = oracle.kde_subset(X, Q, 1.0, off, idx, W)
    assert want.max() < 1e-200
    with K(X, 1.0, form="simt_f32") as kde:
        got = kde.query_subset(Q, off, idx, W)
    _check(got, want, _kappa(X, Q, 1.0, off, idx, W, "gaussian"), 16)


@pytest.mark.slow
def test_benchmark_size_sampled_rows():
    # the benchmark's subset workload: n = 10^6 points (d = 16), 10^5 queries with 1000
    # uniform candidates each (weight n / 1000); 256 sampled queries checked one by one
    import torch
    from paper_2407_07096_gb300 import datagen as G
    K = _kde_cls()
    X, Q = G.workload_single_d16(1, n=1_000_000, m=100_000)
    L_, n, m = 1000, 1_000_000, 100_000
    idx = torch.randint(0, n, (m * L_,), generator=torch.Generator().manual_seed(3), dtype=torch.int64)
    off = torch.arange(0, (m + 1) * L_, L_, dtype=torch.int64)
    W = torch.full((m * L_,), n / L_, dtype=torch.float32)
    with K(X, 0.1) as kde:
        got = kde.query_subset_dev(torch.from_numpy(Q).cuda(), off.cuda(), idx.cuda(), W.cuda()).cpu().numpy()
    rows = np.random.default_rng(4).choice(m, 256, replace=False)
    idx_np = idx.numpy()
    sub_off = np.arange(0, 257 * L_, L_, dtype=np.int64)
    sub_idx = np.concatenate([idx_np[j * L_:(j + 1) * L_] for j in rows])
    want = oracle.kde_subset(X, Q[rows], 0.1, sub_off, sub_idx, np.full(len(sub_idx), n / L_))
    kap = _kappa(X, Q[rows], 0.1, sub_off, sub_idx, np.ones(len(sub_idx)), "gaussian")
    _check(got[rows], want, kap, 16)
