"""Pins of the oracle's other kernel functions (Sec. 3: exponential exp(-a r), logistic
4 / (2 + e^{ar} + e^{-ar})) and of its subset sums (the estimator of Sec. 3.1), against
facts fixed by mathematics rather than by the oracle itself:

* Exponential kernel on the 1-D lattice hZ: a two-sided geometric series,
      sum_k exp(-a |q - k h|) = cosh(a (q - h/2)) / sinh(a h / 2),   0 <= q <= h.
* Logistic kernel on hZ: by Poisson summation the sum is (1/h) times the integral of
  k(a x) over the line, 4 / (a h), plus Fourier terms of size ~ e^{-2 pi^2 / (a h)} (the
  transform of sech^2(x/2) is 4 pi w / sinh(pi w)), below 1e-30 relative for a h <= 0.25.
* a = 0 gives n for both (k(0) = 1); 50-digit decimal brute force on tiny inputs.
* Subset sums: a full, ordered list equals the (pinned) full sum bit for bit; repeated
  indices add their weights; an empty list gives 0; weights act linearly.
"""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle

LATTICE_TAIL = 45.0  # truncate where the kernel is below e^-45 of its peak


def _lattice_1d(h, a):
    K = int(math.ceil(LATTICE_TAIL / (a * h))) + 2
    return (np.arange(-K, K + 1) * h).reshape(-1, 1)


@pytest.mark.parametrize("a,h", [(0.7, 0.25), (2.0, 0.5), (0.05, 1.0)])
def test_exponential_lattice_closed_form(a, h):
    X = _lattice_1d(h, a)
    q = np.array([0.0, 0.1 * h, 0.5 * h, 0.9 * h, h]).reshape(-1, 1)
    got = oracle.kde_kernel(X, q, a, "exponential")
    want = np.cosh(a * (q[:, 0] - h / 2)) / math.sinh(a * h / 2)
    assert np.max(np.abs(got / want - 1)) < 1e-12


def test_exponential_lattice_on_a_line_in_3d():
    # the same lattice placed on a line in R^3, the query on that line
    a, h = 0.7, 0.25
    X1 = _lattice_1d(h, a)
    X = np.concatenate([X1, 2.0 * X1, -X1], axis=1) / 3.0  # direction (1, 2, -1)/3, step h*sqrt(6)/3
    step = h * math.sqrt(6.0) / 3.0
    t = 0.2
    q = np.array([[t, 2 * t, -t]]) / 3.0  # distance t*sqrt(6)/3 (< one step) along the line
    got = oracle.kde_kernel(X, q, a, "exponential")[0]
    s = t * math.sqrt(6.0) / 3.0
    want = math.cosh(a * (s - step / 2)) / math.sinh(a * step / 2)
    assert abs(got / want - 1) < 1e-12


@pytest.mark.parametrize("a,h", [(1.0, 0.25), (2.0, 0.125), (0.5, 0.25)])
def test_logistic_lattice_poisson(a, h):
    assert a * h <= 0.25
    X = _lattice_1d(h, a)
    q = np.array([0.0, 0.3 * h, 0.5 * h, 0.77 * h]).reshape(-1, 1)
    got = oracle.kde_kernel(X, q, a, "logistic")
    assert np.max(np.abs(got / (4.0 / (a * h)) - 1)) < 1e-12


@pytest.mark.parametrize("kernel", ["exponential", "logistic"])
def test_bandwidth_zero_gives_n(kernel):
    r = np.random.default_rng(3)
    X, Q = r.normal(size=(37, 4)), r.normal(size=(5, 4))
    assert np.all(oracle.kde_kernel(X, Q, 0.0, kernel) == 37.0)


@pytest.mark.parametrize("kernel", ["exponential", "logistic"])
def test_bounds_and_monotonicity(kernel):
    # 0 < k <= 1, k(0) = 1, K decreasing in a (Sec. 3's conditions on a kernel)
    r = np.random.default_rng(4)
    X, Q = r.normal(size=(60, 3)), r.normal(size=(6, 3))
    k = [oracle.kde_kernel(X, Q, a, kernel) for a in (0.1, 0.5, 2.0)]
    assert np.all(k[0] > k[1]) and np.all(k[1] > k[2]) and np.all(k[2] > 0) and np.all(k[0] <= 60)
    assert np.all(oracle.kde_kernel(X, X[:3], 5.0, kernel) >= 1.0)


def _decimal_ref(X, Q, a, kernel):
    getcontext().prec = 50
    out = []
    for q in Q:
        s = Decimal(0)
        for x in X:
            d2 = sum((Decimal(float(qk)) - Decimal(float(xk))) ** 2 for qk, xk in zip(q, x))
            t = Decimal(float(a)) * d2.sqrt()
            if kernel == "exponential":
                s += (-t).exp()
            else:
                s += Decimal(4) / (Decimal(2) + t.exp() + (-t).exp())
        out.append(s)
    return out


@pytest.mark.parametrize("kernel", ["exponential", "logistic"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_decimal_brute_force_tiny(kernel, seed):
    r = np.random.default_rng(100 + seed)
    n, m, d = int(r.integers(1, 9)), int(r.integers(1, 5)), int(r.integers(1, 5))
    X, Q = r.normal(size=(n, d)), r.normal(size=(m, d))
    a = float(r.uniform(0.1, 3.0))
    got = oracle.kde_kernel(X, Q, a, kernel)
    for g, w in zip(got, _decimal_ref(X, Q, a, kernel)):
        assert abs(Decimal(float(g)) - w) <= Decimal(1e-14) * abs(w)


# ---------------------------------------------------------------- subset sums (Sec. 3.1)

def _ragged(r, m, n, max_len):
    lens = r.integers(0, max_len + 1, size=m)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    idx = r.integers(0, n, size=int(off[-1])).astype(np.int64)
    return off, idx


@pytest.mark.parametrize("kernel", ["gaussian", "exponential", "logistic"])
def test_subset_full_list_is_the_full_sum(kernel):
    r = np.random.default_rng(5)
    X, Q = r.normal(size=(80, 5)), r.normal(size=(9, 5))
    off = np.arange(0, 80 * 10, 80, dtype=np.int64)
    idx = np.tile(np.arange(80, dtype=np.int64), 9)
    got = oracle.kde_subset(X, Q, 0.4, off, idx, kernel=kernel)
    full = oracle.kde(X, Q, 0.4) if kernel == "gaussian" else oracle.kde_kernel(X, Q, 0.4, kernel)
    assert np.array_equal(got, full)
    # with per-point weights: the weighted full sum
    W = r.uniform(0.5, 2.0, size=80)
    got_w = oracle.kde_subset(X, Q, 0.4, off, idx, np.tile(W, 9))
    assert np.array_equal(got_w, oracle.kde_weighted(X, W, Q, 0.4))


def test_subset_lattice_closed_form():
    # every query's list is the 2-D lattice, weight 2: twice the Poisson closed form
    h, a = 0.5, 0.2
    R = math.sqrt(45.0 / a) + 2.0
    t = np.arange(-math.ceil(R / h), math.ceil(R / h) + 1) * h
    g = np.meshgrid(t, t, indexing="ij")
    L = np.stack([x.reshape(-1) for x in g], axis=1)
    q = np.random.default_rng(6).uniform(-1, 1, size=(3, 2))
    off = np.arange(0, len(L) * 4, len(L), dtype=np.int64)
    idx = np.tile(np.arange(len(L), dtype=np.int64), 3)
    got = oracle.kde_subset(L, q, a, off, idx, np.full(len(idx), 2.0))
    assert np.max(np.abs(got / (2.0 * math.pi / (a * h * h)) - 1)) < 2e-13


def test_subset_repeats_weights_empty_and_linearity():
    r = np.random.default_rng(7)
    X, Q = r.normal(size=(30, 3)), r.normal(size=(4, 3))
    off, idx = _ragged(r, 4, 30, 12)
    W = r.uniform(0.1, 3.0, size=len(idx))
    base = oracle.kde_subset(X, Q, 0.6, off, idx, W)
    # weights act linearly
    assert np.allclose(oracle.kde_subset(X, Q, 0.6, off, idx, 3.0 * W), 3.0 * base, rtol=1e-15, atol=0)
    # each entry duplicated with its weight split in two halves
    off2 = 2 * off
    idx2 = np.repeat(idx, 2)
    W2 = np.repeat(W / 2.0, 2)
    assert np.allclose(oracle.kde_subset(X, Q, 0.6, off2, idx2, W2), base, rtol=1e-14, atol=0)
    # empty lists give exactly 0
    z = oracle.kde_subset(X, Q, 0.6, np.zeros(5, dtype=np.int64), np.zeros(0, dtype=np.int64))
    assert np.all(z == 0.0)
    # single entries: w k(r) at the known distance
    off1 = np.arange(5, dtype=np.int64)
    one = oracle.kde_subset(X, Q, 0.6, off1, np.array([0, 1, 2, 3]), np.array([1.0, 2.0, 0.5, 4.0]))
    want = np.array([w * math.exp(-0.6 * np.sum((Q[j] - X[j]) ** 2)) for j, w in enumerate([1.0, 2.0, 0.5, 4.0])])
    assert np.allclose(one, want, rtol=1e-15, atol=0)


def test_subset_rejects_bad_index():
    X, Q = np.zeros((3, 2)), np.zeros((1, 2))
    with pytest.raises(ValueError):
        oracle.kde_subset(X, Q, 1.0, np.array([0, 1]), np.array([3]))
