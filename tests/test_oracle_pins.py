"""Pins for the FP64 oracle against facts fixed by the mathematics, not by itself.

The paper prints no kernel-density values (its only numbers for exact KDE are CPU
timings, Table "kde_times"), so the oracle is pinned by closed forms, invariances,
special cases and a library routine:

* a = 0 gives exactly n; q = x gives exactly 1 (kernel axioms, Sec. 3).
* A lattice X = h Z^d inside a large box: by Poisson summation the sum equals
  (sqrt(pi/a)/h)^d up to exp(-pi^2/(a h^2)) (Jacobi theta function), for any q.
* Cartesian products separate: K_{X1 x X2}(q1, q2) = K_{X1}(q1) K_{X2}(q2).
* A 1-D Gaussian mixture: E[k(q - x)] is an analytic convolution; a z-test at n = 1e6.
* Translation, permutation and scaling invariance; duplication gives multiples.
* Every term underflowing double: the log-domain routine against a closed form.
* Q = X against torch.cdist (no matmul path) in float64 on CPU.
* A 50-digit decimal brute force on tiny inputs (arithmetic only).

Each of the plausible oracle mistakes (dropped term, wrong sign, missing square,
transposed operands, wrong stride, off-by-one loop bounds) fails at least one test.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from paper_2407_07096_gb300 import datagen as G


def _rng(seed):
    return np.random.default_rng(seed)


def test_a_zero_gives_n_exactly():
    X = _rng(0).normal(size=(1234, 5))
    Q = _rng(1).normal(size=(17, 5))
    out = oracle.kde(X, Q, 0.0)
    assert np.all(out == 1234.0)


def test_single_point_special_values():
    x = np.array([[0.25, -1.5, 3.0]])
    # q = x: exp(0) = 1 exactly
    assert oracle.kde(x, x, 7.3)[0] == 1.0
    # distance 1 along one axis, a = ln 2: exactly 1/2 up to rounding of ln 2
    q = x + np.array([[0.0, 1.0, 0.0]])
    assert abs(oracle.kde(x, q, math.log(2.0))[0] - 0.5) < 1e-15
    # distance^2 = 3 (1 on each axis), a = 1: e^-3
    q = x + 1.0
    assert abs(oracle.kde(x, q, 1.0)[0] - math.exp(-3.0)) < 1e-16


def test_two_points_order_and_count():
    # points at distance^2 1 and 4 from q; a = 1 -> e^-1 + e^-4 (detects dropped/duplicated terms)
    X = np.array([[1.0, 0.0], [0.0, 2.0]])
    q = np.zeros((1, 2))
    assert abs(oracle.kde(X, q, 1.0)[0] - (math.exp(-1) + math.exp(-4))) < 1e-15
    # reversed data order, transposed roles
    assert abs(oracle.kde(X[::-1], q, 1.0)[0] - (math.exp(-1) + math.exp(-4))) < 1e-15
    out = oracle.kde(q, X, 1.0)  # one data point, two queries
    assert np.allclose(out, [math.exp(-1), math.exp(-4)], rtol=0, atol=1e-16)


def _lattice(h, R, d, center=None):
    ticks = np.arange(-math.ceil(R / h), math.ceil(R / h) + 1) * h
    grids = np.meshgrid(*([ticks] * d), indexing="ij")
    pts = np.stack([g.reshape(-1) for g in grids], axis=1)
    return pts if center is None else pts + center


@pytest.mark.parametrize("d,h,a", [(1, 0.5, 0.2), (2, 0.5, 0.2), (3, 0.5, 0.15), (2, 0.25, 0.5)])
def test_lattice_poisson_closed_form(d, h, a):
    # X = h Z^d truncated to |x_k| <= R with a R^2 >= 40 around every query: the
    # truncated tail is < e^-40 relative; the Poisson-summation correction is
    # 2 exp(-pi^2 / (a h^2)) per axis < e^-90. So K = (sqrt(pi/a)/h)^d to ~1e-15.
    R = math.sqrt(45.0 / a) + 2.0
    X = _lattice(h, R, d)
    Q = _rng(d).uniform(-1.0, 1.0, size=(5, d))  # queries anywhere near the origin
    want = (math.sqrt(math.pi / a) / h) ** d
    got = oracle.kde(X, Q, a)
    assert np.max(np.abs(got / want - 1.0)) < 2e-13, (got, want)


def test_cartesian_product_separates():
    r = _rng(3)
    X1 = r.normal(size=(37, 2))
    X2 = r.normal(size=(29, 3))
    q1 = r.normal(size=(4, 2))
    q2 = r.normal(size=(4, 3))
    X = np.concatenate([np.repeat(X1, len(X2), axis=0), np.tile(X2, (len(X1), 1))], axis=1)
    Q = np.concatenate([q1, q2], axis=1)
    a = 0.7
    want = oracle.kde(X1, q1, a) * oracle.kde(X2, q2, a)
    got = oracle.kde(X, Q, a)
    assert np.max(np.abs(got / want - 1.0)) < 1e-13


def test_one_d_mixture_analytic_convolution():
    # X ~ sum_j w_j N(mu_j, s_j^2). For fixed q, k(q - x) has mean
    #   E = sum_j w_j (1 + 2 a s_j^2)^(-1/2) exp(-a (q - mu_j)^2 / (1 + 2 a s_j^2))
    # and second moment E2 = the same with a -> 2a. K(q)/n is the sample mean of n
    # i.i.d. draws, so z = (K/n - E) / sqrt((E2 - E^2)/n) is ~N(0,1) (seeded: deterministic).
    mix = G.Mixture(means=np.array([[-2.0], [0.5], [3.0]]), stds=np.array([0.5, 1.0, 2.0]))
    n = 1_000_000
    X = G.sample(mix, seed=11, count=n, which="data", dtype=np.float64)
    Q = np.array([[-2.5], [0.0], [1.0], [4.0]])
    a = 0.3

    def mean_k(aa, q):
        s2 = mix.stds ** 2
        f = 1.0 + 2.0 * aa * s2
        return np.sum((1.0 / 3.0) * f ** -0.5 * np.exp(-aa * (q - mix.means[:, 0]) ** 2 / f))

    K = oracle.kde(X, Q, a)
    for j, q in enumerate(Q[:, 0]):
        E, E2 = mean_k(a, q), mean_k(2 * a, q)
        z = (K[j] / n - E) / math.sqrt((E2 - E * E) / n)
        assert abs(z) < 6.0, (q, z)
    # a wrong sign or a missing square moves the estimate by far more than 6 sigma
    assert abs(K[1] / n - mean_k(a, 0.0)) / mean_k(a, 0.0) < 5e-3


def test_translation_permutation_duplication_scaling():
    r = _rng(5)
    # dyadic data so that shifts and power-of-two scalings are exact in FP64
    X = np.round(r.normal(size=(300, 4)) * 1024) / 1024
    Q = np.round(r.normal(size=(20, 4)) * 1024) / 1024
    a = 0.9
    base = oracle.kde(X, Q, a)
    t = 1024.0
    assert np.allclose(oracle.kde(X + t, Q + t, a), base, rtol=1e-13, atol=0)
    p = r.permutation(len(X))
    assert np.allclose(oracle.kde(X[p], Q, a), base, rtol=1e-13, atol=0)
    pq = r.permutation(len(Q))
    assert np.array_equal(oracle.kde(X, Q[pq], a), base[pq])
    assert np.allclose(oracle.kde(np.concatenate([X, X, X]), Q, a), 3 * base, rtol=1e-13, atol=0)
    s = 8.0
    assert np.allclose(oracle.kde(X * s, Q * s, a / (s * s)), base, rtol=1e-13, atol=0)


def test_bounds_and_monotone_in_a():
    r = _rng(6)
    X = r.normal(size=(200, 3))
    Q = r.normal(size=(30, 3))
    k1 = oracle.kde(X, Q, 0.5)
    k2 = oracle.kde(X, Q, 1.0)
    assert np.all(k2 < k1) and np.all(k1 <= len(X))
    logk, d2min, kappa = oracle.kde_log(X, Q, 1.0)
    assert np.all(np.exp(-1.0 * d2min) <= k2 * (1 + 1e-15))
    assert np.allclose(np.exp(logk), k2, rtol=1e-13, atol=0)
    assert np.all(kappa >= 1.0 * d2min - 1e-12)


def test_log_domain_underflow_closed_form():
    # two points with a d^2 = 300 and 310 (a = 1): K = e^-300 (1 + e^-10), which
    # underflows nothing but exercises the shifted sum; then a = 3 -> e^-900 underflows
    # double entirely and only the log-domain routine can represent it.
    X = np.array([[math.sqrt(300.0), 0.0], [0.0, math.sqrt(310.0)]])
    q = np.zeros((1, 2))
    logk, d2min, _ = oracle.kde_log(X, q, 1.0)
    assert abs(logk[0] - (-300.0 + math.log1p(math.exp(-10.0)))) < 1e-12
    assert abs(d2min[0] - 300.0) < 1e-12
    logk3, _, _ = oracle.kde_log(X, q, 3.0)
    assert abs(logk3[0] - (-900.0 + math.log1p(math.exp(-30.0)))) < 1e-11
    assert oracle.kde(X, q, 3.0)[0] == 0.0


def test_q_equals_x_against_torch_cdist():
    torch = pytest.importorskip("torch")
    r = _rng(7)
    X = r.normal(size=(700, 6)) * 2.0
    a = 0.4
    D = torch.cdist(torch.from_numpy(X), torch.from_numpy(X),
                    compute_mode="donot_use_mm_for_euclid_dist").numpy()
    want = np.exp(-a * D * D).sum(axis=1)
    got = oracle.kde(X, X, a)
    assert np.allclose(got, want, rtol=1e-12, atol=0)
    # self-KDE (similarity-graph degrees) excludes the diagonal term exp(0) = 1
    assert np.allclose(oracle.kde_self(X, a), want - 1.0, rtol=1e-12, atol=0)


def test_weighted_sum_linear_in_weights():
    r = _rng(8)
    X = r.normal(size=(120, 3))
    Q = r.normal(size=(9, 3))
    a = 0.6
    assert np.allclose(oracle.kde_weighted(X, np.ones(len(X)), Q, a), oracle.kde(X, Q, a),
                       rtol=1e-14, atol=0)
    w = r.integers(1, 4, size=len(X)).astype(np.float64)
    rep = np.repeat(X, w.astype(int), axis=0)
    assert np.allclose(oracle.kde_weighted(X, w, Q, a), oracle.kde(rep, Q, a), rtol=1e-13, atol=0)


def _decimal_kde(X, Q, a):
    getcontext().prec = 50
    out = []
    for q in Q:
        s = Decimal(0)
        for x in X:
            d2 = sum((Decimal(float(qk)) - Decimal(float(xk))) ** 2 for qk, xk in zip(q, x))
            s += (-Decimal(float(a)) * d2).exp()
        out.append(s)
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_decimal_brute_force_tiny(seed):
    r = _rng(100 + seed)
    n, m, d = r.integers(1, 17), r.integers(1, 17), r.integers(1, 9)
    X = r.normal(size=(n, d)) * 2
    Q = r.normal(size=(m, d)) * 2
    a = float(r.uniform(0.01, 2.0))
    want = _decimal_kde(X, Q, a)
    got = oracle.kde(X, Q, a)
    # FP64 rounding of each d^2 is amplified by the exponent's condition number kappa
    _, _, kappa = oracle.kde_log(X, Q, a)
    for g, w, k in zip(got, want, kappa):
        tol = Decimal(float(1e-15 * (4.0 + 2.0 * k)))
        assert abs(Decimal(float(g)) - w) <= tol * abs(w)


def test_thread_count_does_not_change_results():
    r = _rng(9)
    X = r.normal(size=(500, 7))
    Q = r.normal(size=(61, 7))
    assert np.array_equal(oracle.kde(X, Q, 0.3, threads=1), oracle.kde(X, Q, 0.3, threads=7))


def test_rel_err_metric():
    assert oracle.avg_rel_err([1.1, 2.0], [1.0, 2.0]) == pytest.approx(0.05)
    assert oracle.rel_err([0.0], [0.0])[0] == 0.0
