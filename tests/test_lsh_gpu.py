"""GPU E2LSH (Sec. 2) against the CPU oracle: hash values bit for bit (integers decided in
the same FP32 arithmetic on both sides), near-neighbour lists as exact index sets (the
result is unique: the distinct points sharing a bucket, in increasing order), edge cases,
and the pipeline into the weighted subset sums (Sec. 3.1)."""
import numpy as np
import pytest

import oracle
from tests._common import mixture_inputs

pytestmark = pytest.mark.gpu


def _cls():
    from paper_2407_07096_gb300 import build
    build.build()
    from paper_2407_07096_gb300.lsh import E2LSH
    return E2LSH


def _lists(off, idx):
    return [idx[off[j]:off[j + 1]].tolist() for j in range(len(off) - 1)]


@pytest.mark.parametrize("d", [1, 3, 16, 100])
def test_hash_values_bit_exact(d):
    import torch
    E = _cls()
    X, Q = mixture_inputs(60 + d, 3000, 200, d, spread=8.0)
    Q[:4] = np.float32(1e15) * np.sign(Q[:4] + 0.5)  # saturating values
    with E(X, 4, 10, seed=d) as lsh:
        got = lsh.hash_dev(torch.from_numpy(Q).cuda()).cpu().numpy()
        gx = lsh.hash_dev(torch.from_numpy(X).cuda()).cpu().numpy()
        A, B = lsh.A, lsh.B
    assert np.array_equal(got, oracle.lsh_hash(Q, A, B))
    assert np.array_equal(gx, oracle.lsh_hash(X, A, B))


@pytest.mark.parametrize("K,L", [(3, 8), (2, 1), (1, 63), (5, 20)])
def test_candidates_exact(K, L):
    E = _cls()
    X, Q = mixture_inputs(70 + K * L, 6000, 300, 8, spread=6.0)
    Q[::9] += np.float32(500.0)  # far queries: empty lists
    with E(X, K, L, seed=K * 100 + L) as lsh:
        off, idx = lsh.query(Q)
        A, B = lsh.A, lsh.B
    woff, widx = oracle.lsh_candidates(oracle.lsh_hash(X, A, B), oracle.lsh_hash(Q, A, B), K, L)
    assert np.array_equal(off, woff)
    assert np.array_equal(idx, widx)
    assert all(len(c) == 0 for c in _lists(off, idx)[::9])


def test_device_entry_point_edges_and_identical_points():
    import torch
    E = _cls()
    X, Q = mixture_inputs(80, 2000, 64, 5)
    with E(X, 3, 6, seed=1) as lsh:
        off_h, idx_h = lsh.query(Q)
        off_d, idx_d = lsh.query_dev(torch.from_numpy(Q).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(off_d.cpu().numpy(), off_h) and np.array_equal(idx_d.cpu().numpy(), idx_h)
        # caller-provided output arrays (large enough, then too small for the lists)
        ob, ib = np.full(70, -1, np.int64), np.full(len(idx_h) + 5, -1, np.int64)
        o2, i2 = lsh.query(Q, out=(ob, ib))
        assert np.array_equal(o2, off_h) and np.array_equal(i2, idx_h) and np.shares_memory(i2, ib)
        o3, i3 = lsh.query(Q, out=(ob, np.zeros(3, np.int64)))
        assert np.array_equal(o3, off_h) and np.array_equal(i3, idx_h)
        o0, i0 = lsh.query(Q[:0])
        assert o0.tolist() == [0] and len(i0) == 0
        # every data point finds itself
        off_x, idx_x = lsh.query(X[:100])
        assert all(j in c for j, c in enumerate(_lists(off_x, idx_x)))
    # all points identical: a query at that point gets every index once
    Xs = np.repeat(X[:1], 777, axis=0)
    with E(Xs, 4, 5, seed=2) as lsh:
        off, idx = lsh.query(Xs[:3])
    assert off.tolist() == [0, 777, 1554, 2331] and np.array_equal(idx[:777], np.arange(777))
    with E(X[:1], 2, 2, seed=3) as lsh:  # n = 1
        off, idx = lsh.query(X[:1])
    assert off.tolist() == [0, 1] and idx.tolist() == [0]


def test_validation():
    from paper_2407_07096_gb300 import _lib as L
    E = _cls()
    X, _ = mixture_inputs(81, 100, 1, 4)
    for K, Lt in ((0, 3), (2, 0), (2, 64)):
        with pytest.raises(L.StagKdeError) as e:
            E(X, K, Lt)
        assert e.value.code == L.EINVAL
    bad = X.copy()
    bad[3, 1] = np.nan
    with pytest.raises(L.StagKdeError):
        E(bad, 2, 2)
    with E(X, 2, 2) as lsh:
        with pytest.raises(L.StagKdeError):
            lsh.query(bad[:5])


def test_pipeline_into_subset_sums():
    # candidate lists from the tables, evaluated by the weighted subset sums
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    from tests.test_subset_gpu import _check, _kappa
    E = _cls()
    X, Q = mixture_inputs(82, 5000, 150, 6, spread=5.0)
    with E(X, 3, 10, seed=5) as lsh:
        off, idx = lsh.query(Q)
        A, B = lsh.A, lsh.B
    woff, widx = oracle.lsh_candidates(oracle.lsh_hash(X, A, B), oracle.lsh_hash(Q, A, B), 3, 10)
    assert np.array_equal(off, woff) and np.array_equal(idx, widx)
    W = np.full(len(idx), 2.0, dtype=np.float32)
    with ExactGaussianKDE(X, 0.2, form="simt_f32") as kde:
        got = kde.query_subset(Q, off, idx, W)
        full = kde.query(Q)
    want = oracle.kde_subset(X, Q, 0.2, woff, widx, W)
    _check(got, want, _kappa(X, Q, 0.2, woff, widx, W, "gaussian"), 6)
    assert np.all(got <= 2.0 * full * (1 + 1e-5))  # a subset of the points, weight 2


@pytest.mark.slow
def test_sort_path_beyond_the_bitmap():
    # n above what the shared-memory bitmap path serves (2^22 points): repeats across
    # tables are removed by the radix-sort path instead; the lists are the same
    E = _cls()
    r = np.random.default_rng(17)
    X = r.normal(scale=40.0, size=(4_500_000, 2)).astype(np.float32)
    Q = r.normal(scale=40.0, size=(40, 2)).astype(np.float32)
    with E(X, 4, 3, seed=17) as lsh:
        off, idx = lsh.query(Q)
        A, B = lsh.A, lsh.B
    woff, widx = oracle.lsh_candidates(oracle.lsh_hash(X, A, B), oracle.lsh_hash(Q, A, B), 4, 3)
    assert woff[-1] > 1000
    assert np.array_equal(off, woff)
    assert np.array_equal(idx, widx)


@pytest.mark.slow
def test_bitmap_slices_and_duplicates():
    # n spanning two slices of the bitmap path (at most 1572864 points each), with every
    # point repeated three times (identical hash values: the same buckets)
    E = _cls()
    r = np.random.default_rng(18)
    base = r.normal(scale=6.0, size=(600_000, 3)).astype(np.float32)
    X = np.concatenate([base, base[::-1], base])
    Q = np.concatenate([base[:30], r.normal(scale=6.0, size=(30, 3)).astype(np.float32)])
    with E(X, 3, 4, seed=18) as lsh:
        off, idx = lsh.query(Q)
        A, B = lsh.A, lsh.B
    woff, widx = oracle.lsh_candidates(oracle.lsh_hash(X, A, B), oracle.lsh_hash(Q, A, B), 3, 4)
    assert np.array_equal(off, woff)
    assert np.array_equal(idx, widx)
    lists = _lists(off, idx)
    for j in range(30):  # a data point finds all three copies of itself
        assert {j, len(X) - 600_000 + j, 2 * 600_000 - 1 - j} <= set(lists[j])


@pytest.mark.slow
def test_paper_parameters_sampled():
    # the paper's example tables (K = 6, L = 50) over 200000 points, 2000 queries; 40 lists
    # checked against the oracle
    from paper_2407_07096_gb300 import datagen as G
    E = _cls()
    X, Q = G.workload_single_d16(4, n=200_000, m=2000)
    with E(X, 6, 50, seed=9) as lsh:
        off, idx = lsh.query(Q)
        A, B = lsh.A, lsh.B
    rows = np.random.default_rng(5).choice(len(Q), 40, replace=False)
    woff, widx = oracle.lsh_candidates(oracle.lsh_hash(X, A, B), oracle.lsh_hash(Q[rows], A, B), 6, 50)
    got = _lists(off, idx)
    want = _lists(woff, widx)
    for r, w in zip(rows, want):
        assert got[r] == w


def test_membership_is_exact_when_keys_collide(monkeypatch):
    # With 12-bit bucket keys (a test hook; the library uses 58 bits) many different
    # K-tuples share a key: the build must pick a salt under which no two tuples of the
    # points share a key, and each lookup must reject a run whose tuple differs from the
    # query's. Tight data (few tuples per table) and far queries (new tuples only):
    # hundreds of lookups land on another tuple's key, and the lists must still equal
    # the oracle's, which compares tuples.
    E = _cls()
    rng = np.random.default_rng(5)
    X = (0.3 * rng.normal(size=(3000, 8))).astype(np.float32)
    near = (0.3 * rng.normal(size=(2000, 8))).astype(np.float32)
    far = rng.uniform(-200, 200, size=(20000, 8)).astype(np.float32)
    Q = np.concatenate([near, far])
    monkeypatch.setenv("STAG_KDE_LSH_KEY_BITS", "12")
    with E(X, 3, 8, seed=11) as lsh:
        off, idx = lsh.query(Q)
        A, B = lsh.A, lsh.B
    monkeypatch.delenv("STAG_KDE_LSH_KEY_BITS")
    HX, HQ = oracle.lsh_hash(X, A, B), oracle.lsh_hash(Q, A, B)
    woff, widx = oracle.lsh_candidates(HX, HQ, 3, 8)
    assert np.array_equal(off, woff)
    assert np.array_equal(idx, widx)
    assert off[len(near)] > 0  # the near queries found their buckets
    # the far queries' tuples are new: count the lookups whose 12-bit key space alone
    # would have matched a bucket (distinct tuples per table vs 4096 keys)
    tuples = sum(len({tuple(r) for r in HX[:, l * 3:(l + 1) * 3]}) for l in range(8))
    assert tuples * len(far) / 4096 > 100
