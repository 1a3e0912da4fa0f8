"""Strength of the oracle pins: plausible mistakes planted in a copy of the oracle's C
source (on the CPU) must each fail at least one closed-form pin. The pins used here are
the paper-independent facts of tests/test_oracle_pins.py: a = 0 gives n, two points at
known distances, the lattice (Poisson summation) closed form, a Cartesian product."""
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
    "exponent sign": ("double e = exp(-J->a * sqdist(q, J->X + i * J->d, J->d));",
                      "double e = exp(J->a * sqdist(q, J->X + i * J->d, J->d));"),
    "bandwidth dropped": ("double e = exp(-J->a * sqdist(q, J->X + i * J->d, J->d));",
                          "double e = exp(-sqdist(q, J->X + i * J->d, J->d));"),
    "last point dropped": ("for (int64_t i = 0; i < J->n; ++i) {\n            if (J->self_skip",
                           "for (int64_t i = 0; i < J->n - 1; ++i) {\n            if (J->self_skip"),
    "row stride lost": ("double e = exp(-J->a * sqdist(q, J->X + i * J->d, J->d));",
                        "double e = exp(-J->a * sqdist(q, J->X + i, J->d));"),
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

    def kde(X, Q, a):
        X = np.ascontiguousarray(X, dtype=np.float64)
        Q = np.ascontiguousarray(Q, dtype=np.float64)
        out = np.empty(len(Q))
        lib.oracle_kde(X.ctypes.data_as(D), len(X), Q.ctypes.data_as(D), len(Q), X.shape[1], a, out.ctypes.data_as(D), 2)
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
    return ok


def test_unmutated_copy_passes(tmp_path):
    assert _pins_pass(_compile(tmp_path, "none", "s += t * t;", "s += t * t;"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_mutant_fails_a_pin(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _pins_pass(_compile(tmp_path, name, old, new)), f"mutant {name!r} survived the pins"
