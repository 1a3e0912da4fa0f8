"""Strength of the oracle pins: plausible mistakes planted in a copy of the oracle's C
source (on the CPU) must each fail at least one closed-form pin. The pins used here are
the paper-independent facts of tests/test_oracle_pins.py and tests/test_oracle_kernels.py:
a = 0 gives n, two points at known distances, the lattice (Poisson summation) closed
form, a Cartesian product; for the exponential and logistic kernels their lattice closed
forms; for the subset sums the lattice closed form through a list and single entries."""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "kde_oracle.c")

MUTANTS = {
    "missing square": ("s += t * t;", "s += t;"),
    "exponent sign": ("if (kind == 0) return exp(-a * d2);", "if (kind == 0) return exp(a * d2);"),
    "bandwidth dropped": ("if (kind == 0) return exp(-a * d2);", "if (kind == 0) return exp(-d2);"),
    "last point dropped": ("for (int64_t i = 0; i < J->n; ++i) {\n            if (J->self_skip",
                           "for (int64_t i = 0; i < J->n - 1; ++i) {\n            if (J->self_skip"),
    "row stride lost": ("double e = kern(J->kind, J->a, sqdist(q, J->X + i * J->d, J->d));",
                        "double e = kern(J->kind, J->a, sqdist(q, J->X + i, J->d));"),
    "exponential kernel squared": ("if (kind == 1) return exp(-x);", "if (kind == 1) return exp(-x * x);"),
    "sqrt dropped": ("double x = a * sqrt(d2);", "double x = a * d2;"),
    "logistic factor 4 dropped": ("return 4.0 / (2.0 + exp(x) + exp(-x));", "return 1.0 / (2.0 + exp(x) + exp(-x));"),
    "logistic sign": ("return 4.0 / (2.0 + exp(x) + exp(-x));", "return 4.0 / (2.0 + exp(x) - exp(-x));"),
    "subset weight ignored": ("s += J->W ? J->W[e] * k : k;", "s += k;"),
    "subset index ignored": ("sqdist(q, J->X + J->idx[e] * J->d, J->d)", "sqdist(q, J->X + e * J->d, J->d)"),
    "subset last entry dropped": ("for (int64_t e = J->off[j]; e < J->off[j + 1]; ++e) {",
                                  "for (int64_t e = J->off[j]; e + 1 < J->off[j + 1]; ++e) {"),
    "last coordinate dropped": ("for (int64_t k = 0; k < d; ++k) {", "for (int64_t k = 0; k + 1 < d; ++k) {"),
    "query/point swapped stride": ("const double *q = J->Q + j * J->d;\n        double s = 0.0;",
                                   "const double *q = J->Q + j;\n        double s = 0.0;"),
}


def _compile(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation site for {name!r} not found"
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-o", str(so), str(path), "-lm", "-lpthread"], check=True)
    lib = ctypes.CDLL(str(so))
    D = ctypes.POINTER(ctypes.c_double)
    lib.oracle_kde.argtypes = [D, ctypes.c_int64, D, ctypes.c_int64, ctypes.c_int64, ctypes.c_double, D, ctypes.c_int]
    lib.oracle_kde.restype = ctypes.c_int
    lib.oracle_kde_kernel.argtypes = [ctypes.c_int, D, ctypes.c_int64, D, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_double, D, ctypes.c_int]
    lib.oracle_kde_kernel.restype = ctypes.c_int
    I = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_kde_subset.argtypes = [ctypes.c_int, D, ctypes.c_int64, D, ctypes.c_int64, ctypes.c_int64,
                                      ctypes.c_double, I, I, D, D, ctypes.c_int]
    lib.oracle_kde_subset.restype = ctypes.c_int

    def kde(X, Q, a, kind=None, off=None, idx=None, W=None):
        X = np.ascontiguousarray(X, dtype=np.float64)
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.empty(len(Q))
        if off is not None:
            off = np.ascontiguousarray(off, dtype=np.int64)
            idx = np.ascontiguousarray(idx, dtype=np.int64)
            W = np.ascontiguousarray(W, dtype=np.float64)
            lib.oracle_kde_subset(0, X.ctypes.data_as(D), len(X), Q.ctypes.data_as(D), len(Q), X.shape[1], a,
                                  off.ctypes.data_as(I), idx.ctypes.data_as(I), W.ctypes.data_as(D),
                                  out.ctypes.data_as(D), 2)
        elif kind is not None:
            lib.oracle_kde_kernel(kind, X.ctypes.data_as(D), len(X), Q.ctypes.data_as(D), len(Q), X.shape[1], a,
                                  out.ctypes.data_as(D), 2)
        else:
            lib.oracle_kde(X.ctypes.data_as(D), len(X), Q.ctypes.data_as(D), len(Q), X.shape[1], a,
                           out.ctypes.data_as(D), 2)
        return out
    return kde


def _pins_pass(kde):
    """True if every pin holds for this implementation."""
    r = np.random.default_rng(0)
    ok = True
    X = r.normal(size=(50, 3))
    ok &= bool(np.all(kde(X, r.normal(size=(4, 3)), 0.0) == 50.0))
    X2 = np.array([[1.0, 0.0], [0.0, 2.0]])
    ok &= abs(kde(X2, np.zeros((1, 2)), 1.0)[0] - (math.exp(-1) + math.exp(-4))) < 1e-15
    ok &= abs(kde(X2, np.array([[1.0, 0.0], [0.0, 2.0]]), 1.0)[1] - (1.0 + math.exp(-5.0))) < 1e-15
    h, a, d = 0.5, 0.2, 2
    R = math.sqrt(45.0 / a) + 2.0
    t = np.arange(-math.ceil(R / h), math.ceil(R / h) + 1) * h
    g = np.meshgrid(t, t, indexing="ij")
    L = np.stack([x.reshape(-1) for x in g], axis=1)
    got = kde(L, r.uniform(-1, 1, size=(3, d)), a)
    ok &= bool(np.max(np.abs(got / (math.pi / (a * h * h)) - 1)) < 2e-13)
    X1, Xb = r.normal(size=(7, 2)), r.normal(size=(5, 3))
    q1, qb = r.normal(size=(2, 2)), r.normal(size=(2, 3))
    P = np.concatenate([np.repeat(X1, 5, axis=0), np.tile(Xb, (7, 1))], axis=1)
    ok &= bool(np.max(np.abs(kde(P, np.concatenate([q1, qb], 1), 0.7) / (kde(X1, q1, 0.7) * kde(Xb, qb, 0.7)) - 1)) < 1e-13)
    # exponential and logistic kernels: 1-D lattice closed forms
    for kind, a1, h1 in ((1, 0.7, 0.25), (2, 1.0, 0.25)):
        K = int(math.ceil(45.0 / (a1 * h1))) + 2
        X1d = (np.arange(-K, K + 1) * h1).reshape(-1, 1)
        qs = np.array([[0.0], [0.1], [0.2]])
        want = (np.cosh(a1 * (qs[:, 0] - h1 / 2)) / math.sinh(a1 * h1 / 2)) if kind == 1 else 4.0 / (a1 * h1)
        ok &= bool(np.max(np.abs(kde(X1d, qs, a1, kind=kind) / want - 1)) < 1e-12)
    # subset sums: the 2-D lattice through every query's list with weight 2, and single
    # entries at known distances
    n_l = len(L)
    qq = r.uniform(-1, 1, size=(2, d))
    got = kde(L, qq, a, off=[0, n_l, 2 * n_l], idx=np.tile(np.arange(n_l), 2), W=np.full(2 * n_l, 2.0))
    ok &= bool(np.max(np.abs(got / (2.0 * math.pi / (a * h * h)) - 1)) < 2e-13)
    got = kde(X2, np.zeros((2, 2)), 1.0, off=[0, 2, 3], idx=[0, 1, 1], W=[1.0, 3.0, 0.5])
    ok &= abs(got[0] - (math.exp(-1) + 3.0 * math.exp(-4))) < 1e-15 and abs(got[1] - 0.5 * math.exp(-4)) < 1e-15
    return ok


def test_unmutated_copy_passes(tmp_path):
    assert _pins_pass(_compile(tmp_path, "none", "s += t * t;", "s += t * t;"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_mutant_fails_a_pin(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _pins_pass(_compile(tmp_path, name, old, new)), f"mutant {name!r} survived the pins"
