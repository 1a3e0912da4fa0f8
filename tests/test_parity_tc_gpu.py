"""Parity of the tcgen05/TMEM tensor-core form with the FP64 oracle through the C-ABI.

Tolerance (tests/_common.py): 1e-4 relative for every query with condition number
kappa <= 400, the plain FP32 form's measured bound above. The split form's own error
grows with a * ||u|| * ||v|| (query distance from the data mean times tile radius, see
kde_tc.cu); every query gets an error estimate and those above 7.5e-5 are recomputed
with the plain FP32 form, whose error (~3 kappa 2^-24) is below 1e-4 up to kappa ~400.
Tests with the check switched off measure the tensor-core arithmetic alone where it is
well inside the bar. Sizes span several 128-query and 256-point tiles with ragged
tails; the full-size workloads are checked on every query (n = m = 1e5, d = 16) and on
1000 sampled queries (n = 2e6, d = 64)."""
import math

import numpy as np
import pytest

import oracle
from paper_2407_07096_gb300 import datagen as G
from tests._common import mixture_inputs

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def K():
    from paper_2407_07096_gb300 import build
    build.build()
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    return ExactGaussianKDE


def check_tc(K, X, Q, a, tol=TOL, tc_check=True):
    with K(X, a, form="tc", tc_check=tc_check) as kde:
        assert kde.form == "tc"
        got = kde.query(Q)
    ref = oracle.kde(X, Q, a)
    err = oracle.rel_err(got, ref)
    assert err.max() <= tol, f"max rel err {err.max():.3e} (median {np.median(err):.3e})"
    return got, ref


@pytest.mark.parametrize("d", [1, 2, 3, 7, 8, 15, 16, 17, 31, 32, 33, 48, 63, 64, 65, 100, 127, 128])
def test_tc_dims(K, d):
    X, Q = mixture_inputs(d, 1500, 300, d)
    check_tc(K, X, Q, 0.5 / d)


@pytest.mark.parametrize("n,m", [(1, 1), (1, 200), (255, 127), (256, 128), (257, 129), (5000, 1), (3001, 1000)])
def test_tc_ragged_sizes(K, n, m):
    X, Q = mixture_inputs(n + 7 * m, n, m, 16)
    check_tc(K, X, Q, 0.1)


@pytest.mark.parametrize("a", [0.01, 0.1, 1.0, 4.0])
def test_tc_bandwidths(K, a):
    X, Q = mixture_inputs(11, 6000, 400, 8, spread=4.0)
    check_tc(K, X, Q, a)


@pytest.mark.parametrize("d,a", [(8, 0.5), (16, 0.3), (64, 0.02)])
def test_tc_arithmetic_alone_without_recompute(K, d, a):
    # the tensor-core results themselves, no FP32 recompute of any query
    X, Q = mixture_inputs(40 + d, 6000, 500, d, spread=4.0)
    check_tc(K, X, Q, a, tc_check=False)


def test_tc_ill_conditioned_queries_are_recomputed(K):
    # d = 128, a = 1: the exponent's condition number is ~150, far outside what split
    # FP16 products can carry; the estimate must hand those queries to the FP32 form
    X, Q = mixture_inputs(13, 4000, 300, 128, k=4, spread=3.0)
    with K(X, 1.0, form="tc") as kde:
        got = kde.query(Q)
        redo = kde.last_recomputed()
    ref = oracle.kde(X, Q, 1.0)
    _, _, kappa = oracle.kde_log(X, Q, 1.0)
    from tests._common import tol_tc
    assert redo > 0.9 * len(Q)
    assert kappa.max() > 100 and kappa.max() <= 400
    err = oracle.rel_err(got, ref)
    assert np.all(err <= tol_tc(kappa, 128)), err.max()
    assert err.max() <= TOL  # every query here has kappa <= 400


def test_tc_queries_beyond_the_split_range(K):
    # queries ~1000 from a unit cloud (more than 64x the data's extent from its centre):
    # their scaled coordinates leave FP16's range, so they are flagged and recomputed by
    # the FP32 form; a tiny a keeps their densities far from zero
    r = np.random.default_rng(21)
    X = r.normal(size=(3000, 4)).astype(np.float32)
    Q = r.normal(size=(200, 4)).astype(np.float32)
    Q[::4, 0] += np.float32(1000.0)
    a = 1e-6
    with K(X, a, form="tc") as kde:
        got = kde.query(Q)
        redo = kde.last_recomputed()
    ref = oracle.kde(X, Q, a)
    assert redo >= 50
    assert oracle.rel_err(got, ref).max() <= TOL
    assert np.all(ref[::4] > 0.3 * 3000)


@pytest.mark.parametrize("a", [1.0, 4.0])
def test_tc_pruned_recompute_of_flagged_queries(K, a):
    # the benchmark's mixture at large a, d = 16: the queries the estimate flags are
    # recomputed over the tiles that can matter; every query against the oracle
    from paper_2407_07096_gb300 import datagen as G
    X, Q = G.workload_single_d16(0, n=30_000, m=4_000)
    with K(X, a, form="tc") as kde:
        got = kde.query(Q)
        redo = kde.last_recomputed()
    ref = oracle.kde(X, Q, a)
    if a == 4.0:
        assert redo > 100
    err = oracle.rel_err(got, ref)
    assert err.max() <= TOL, err.max()


def test_tc_normalise_option(K):
    X, Q = mixture_inputs(22, 3000, 200, 16)
    with K(X, 0.2, form="tc", normalise=True) as kde:
        got = kde.query(Q)
    assert oracle.rel_err(got, oracle.kde(X, Q, 0.2) / 3000.0).max() <= TOL


def test_tc_a_zero_is_exactly_n(K):
    X, Q = mixture_inputs(3, 5001, 300, 16)
    with K(X, 0.0, form="tc") as kde:
        assert np.all(kde.query(Q) == 5001.0)


def test_tc_underflow_shift(K):
    # d = 64 with a wide kernel far away: every term below FP32 range, shift keeps them
    X, Q = mixture_inputs(12, 2000, 100, 64, k=2, spread=1.0)
    Q = Q + 6.0  # move the queries away: a d^2 ~ 0.05 * (64 * 36) > 100
    got, ref = check_tc(K, X, Q, 0.05)
    assert np.all(ref < 1e-38) and np.all(got > 0)


def test_tc_lattice_closed_form(K):
    h, a, d = 0.5, 0.15, 3
    R = math.sqrt(45.0 / a) + 2.0
    t = np.arange(-math.ceil(R / h), math.ceil(R / h) + 1) * h
    g = np.meshgrid(t, t, t, indexing="ij")
    X = np.stack([x.reshape(-1) for x in g], axis=1).astype(np.float32)
    Q = np.random.default_rng(0).uniform(-1, 1, size=(300, d)).astype(np.float32)
    want = (math.sqrt(math.pi / a) / h) ** d
    with K(X, a, form="tc") as kde:
        got = kde.query(Q)
    assert np.max(np.abs(got / want - 1)) < TOL


def test_tc_translation_and_permutation_invariance(K):
    # dyadic data, exact shift in FP32: the result must not depend on where the cloud sits
    r = np.random.default_rng(3)
    X = (np.round(r.normal(size=(4000, 16)) * 256) / 256).astype(np.float32)
    Q = (np.round(r.normal(size=(300, 16)) * 256) / 256).astype(np.float32)
    a = 0.3
    with K(X, a, form="tc") as k0, K(X + 1024.0, a, form="tc") as k1, K(X[r.permutation(len(X))], a, form="tc") as k2:
        b0, b1, b2 = k0.query(Q), k1.query(Q + 1024.0), k2.query(Q)
    ref = oracle.kde(X, Q, a)
    for b in (b0, b1, b2):
        assert oracle.rel_err(b, ref).max() <= TOL


def test_tc_deterministic_and_dev_path(K):
    import torch
    X, Q = mixture_inputs(4, 20000, 1000, 32)
    with K(X, 0.05, form="tc") as kde:
        a1 = kde.query(Q)
        a2 = kde.query(Q)
        a3 = kde.query_dev(torch.from_numpy(Q).cuda()).cpu().numpy()
    assert np.array_equal(a1, a2) and np.array_equal(a1, a3)


def test_tc_result_independent_of_batch_composition(K):
    # a query's density must not depend on the other queries of its batch
    X, Q = mixture_inputs(5, 8000, 700, 16)
    with K(X, 0.2, form="tc") as kde:
        full = kde.query(Q)
        part = kde.query(Q[100:229])
        one = kde.query(Q[300:301])
    assert oracle.rel_err(part, full[100:229]).max() <= TOL
    assert oracle.rel_err(one, full[300:301]).max() <= TOL


@pytest.fixture(scope="module")
def single_d16():
    """The n = m = 1e5, d = 16 workload and the oracle's value of EVERY query at each of
    its bandwidths (3e10 FP64 evaluations, ~25 s on 16 host cores)."""
    X, Q = G.workload_single_d16(0)
    refs = {}
    for a in (0.01, 0.1, 1.0):
        logk, _, kappa = oracle.kde_log(X, Q, a)  # K = exp(log K), to ~1e-15
        refs[a] = (np.exp(logk), kappa)
    return X, Q, refs


@pytest.mark.slow
@pytest.mark.parametrize("form", ["tc", "simt_f32"])
def test_single_instance_d16_workload_every_query(K, single_d16, form):
    # n = m = 100000, d = 16, a in {0.01, 0.1, 1}: the benchmark's workload in the
    # launch configuration it times (autotuned settings), every query against the oracle
    import torch
    from tests._common import tol_f32, tol_tc
    X, Q, refs = single_d16
    Qd = torch.from_numpy(Q).cuda()
    for a in (0.01, 0.1, 1.0):
        ref, kappa = refs[a]
        with K(X, a, form=form) as kde:
            kde.autotune(Qd)
            got = kde.query(Q)
            redo = kde.last_recomputed()
        err = oracle.rel_err(got, ref)
        tol = tol_tc(kappa, 16) if form == "tc" else tol_f32(kappa, 16)
        assert np.all(err <= tol), (a, float(err.max()), int(np.sum(err > tol)))
        if form == "tc":
            assert redo <= 0.05 * len(Q), (a, redo)


@pytest.mark.slow
def test_tc_large_d64_workload_1000_sampled_queries(K):
    # n = 2e6, m = 1e5, d = 64, a = 0.05: error on 1000 sampled queries
    from tests._common import tol_tc
    X, Q, a = G.workload_large_d64(0)
    with K(X, a, form="tc") as kde:
        got = kde.query(Q)
    idx = np.linspace(0, len(Q) - 1, 1000).astype(int)
    logk, _, kappa = oracle.kde_log(X, Q[idx], a)
    assert np.all(oracle.rel_err(got[idx], np.exp(logk)) <= tol_tc(kappa, 64))


@pytest.mark.parametrize("d,n", [(5, 7001), (16, 20011), (33, 10007), (64, 9001), (100, 5003), (128, 12345)])
def test_tc_grouped_recompute_of_flagged_queries(K, d, n):
    # 10-component mixtures (means U[-10, 10]^d, std 1) at bandwidths whose condition
    # numbers send most queries to the FP32 recompute, which runs in groups of 64 sorted
    # queries over the union of their kept tiles. Ragged n leaves the last point tile
    # partial in both the 128/256-point and the 64-point tilings.
    from paper_2407_07096_gb300 import datagen as G
    from tests._common import tol_tc
    mix = G.make_mixture(d, 10, d, -10.0, 10.0, 1.0)
    X, Q = G.sample(mix, d, n, "data"), G.sample(mix, d, 900, "query")
    a = 60.0 / (2.0 * d)
    with K(X, a, form="tc") as kde:
        got = kde.query(Q)
        redo = kde.last_recomputed()
        again = kde.query(Q)
    logk, _, kappa = oracle.kde_log(X, Q, a)
    assert redo > (300 if d >= 16 else 100)
    assert np.array_equal(got, again)
    err = oracle.rel_err(got, np.exp(logk))
    assert np.all(err <= tol_tc(kappa, d)), err.max()
