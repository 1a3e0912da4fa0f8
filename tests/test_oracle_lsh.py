"""Pins of the E2LSH oracle (Sec. 2) against facts that do not come from the oracle:

* the collision probability of one hash function at distance c, printed in closed form
  in Sec. 2 (p(c) = erf(2 sqrt 2 / c) - c (1 - e^{-8/c^2}) / (2 sqrt(2 pi))), as a z-test
  over many independently drawn functions;
* the boosted probability 1 - (1 - p(c)^K)^L of colliding in at least one of L tables of
  K functions (Sec. 2, "Boosting the Probability"), also as a z-test;
* exact bucket values for axis-aligned functions on dyadic inputs, and the int32 clamp
  (rounding instead of flooring is a pure relabelling under a uniform offset, so only
  these exact values can tell the two apart);
* structure of the candidate lists: a point is its own candidate, L tables give the union
  of the single tables' lists, one table of one function partitions the points;
* planted mistakes in a copy of the oracle's C source each fail one of these.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lsh_oracle.c")


def p_collide(c):
    """Sec. 2's closed form of the collision probability at distance c (bucket width 4)."""
    return (-(1.0 / (2.0 * math.sqrt(2.0 * math.pi))) * c * math.exp(-8.0 / c ** 2) * (math.exp(8.0 / c ** 2) - 1.0)
            + math.erf(2.0 * math.sqrt(2.0) / c))


def _functions(r, nf, d):
    return r.normal(size=(nf, d)).astype(np.float32), r.uniform(0.0, 4.0, size=nf).astype(np.float32)


def _collision_rate(hash_fn, c, N=20000, d=6, seed=0):
    r = np.random.default_rng(seed)
    A, B = _functions(r, N, d)
    u = r.normal(size=d)
    u /= np.linalg.norm(u)
    X = np.stack([np.zeros(d), c * u]).astype(np.float32)
    H = hash_fn(X, A, B)
    return float(np.mean(H[0] == H[1]))


def _z(freq, p, N):
    return (freq - p) / math.sqrt(max(p * (1 - p), 1e-12) / N)


AXIS_X = np.array([[-4.0, 9.0], [3.999, 0.0], [0.0, 0.0], [-0.5, 0.0], [2.0, 0.0], [1.999, 0.0], [8.0, 0.0]],
                  dtype=np.float32)
AXIS_A = np.array([[1.0, 0.0], [1.0, 0.0]], dtype=np.float32)
AXIS_B = np.array([0.0, 2.0], dtype=np.float32)
AXIS_H = [[-1, 0, 0, -1, 0, 0, 2], [-1, 1, 0, 0, 1, 0, 2]]


def _pins_hold(hash_fn, cand_fn):
    ok = True
    H = hash_fn(AXIS_X, AXIS_A, AXIS_B)
    ok &= H[:, 0].tolist() == AXIS_H[0] and H[:, 1].tolist() == AXIS_H[1]
    for c in (0.5, 1.0, 2.0, 4.0, 9.0):
        ok &= abs(_z(_collision_rate(hash_fn, c), p_collide(c), 20000)) < 5.0
    # boosting over K x L functions
    r = np.random.default_rng(11)
    K, L, c, N, d = 3, 4, 1.5, 3000, 5
    hits = 0
    for t in range(N):
        A, B = _functions(r, K * L, d)
        u = r.normal(size=d)
        X = np.stack([np.zeros(d), c * u / np.linalg.norm(u)]).astype(np.float32)
        H = hash_fn(X, A, B)
        off, _ = cand_fn(H[:1], H[1:], K, L)
        hits += int(off[1] > 0)
    pb = 1.0 - (1.0 - p_collide(c) ** K) ** L
    ok &= abs(_z(hits / N, pb, N)) < 5.0
    # union over tables
    r = np.random.default_rng(12)
    X = r.normal(scale=2.0, size=(300, 4)).astype(np.float32)
    A, B = _functions(r, 2 * 3, 4)
    H = hash_fn(X, A, B)
    off, idx = cand_fn(H, H[:40], 2, 3)
    for j in range(40):
        got = set(idx[off[j]:off[j + 1]].tolist())
        want = set()
        for l in range(3):
            o1, i1 = cand_fn(H[:, 2 * l:2 * l + 2], H[j:j + 1, 2 * l:2 * l + 2], 2, 1)
            want |= set(i1.tolist())
        ok &= got == want and j in got
    return bool(ok)


@pytest.mark.parametrize("c", [0.5, 1.0, 2.0, 4.0, 9.0])
def test_collision_probability_closed_form(c):
    assert abs(_z(_collision_rate(oracle.lsh_hash, c), p_collide(c), 20000)) < 5.0


def test_closed_form_matches_its_integral():
    # Sec. 2 defines p(c) = int_0^4 (1/c) f(t/c) (1 - t/4) dt, f the density of |N(0,1)|
    for c in (0.3, 1.0, 2.5, 7.0):
        t = np.linspace(0.0, 4.0, 400001)
        f = np.sqrt(2.0 / np.pi) * np.exp(-(t / c) ** 2 / 2.0) / c
        integral = np.trapezoid(f * (1.0 - t / 4.0), t)
        assert abs(integral - p_collide(c)) < 1e-9


def test_all_pins_on_the_oracle():
    assert _pins_hold(oracle.lsh_hash, oracle.lsh_candidates)


def test_exact_values_axis_aligned():
    # floor((x_1 + b) / 4) for dyadic x_1; b = 2 moves the boundaries by half a bucket
    H = oracle.lsh_hash(AXIS_X, AXIS_A, AXIS_B)
    assert H[:, 0].tolist() == AXIS_H[0]
    assert H[:, 1].tolist() == AXIS_H[1]
    big = oracle.lsh_hash(np.array([[1e15], [-1e15]], dtype=np.float32), np.ones((1, 1), np.float32),
                          np.zeros(1, np.float32))
    assert big[:, 0].tolist() == [2 ** 31 - 1, -2 ** 31]


def test_one_function_partitions_the_points():
    r = np.random.default_rng(13)
    X = r.normal(scale=3.0, size=(500, 3)).astype(np.float32)
    A, B = _functions(r, 1, 3)
    H = oracle.lsh_hash(X, A, B)
    off, idx = oracle.lsh_candidates(H, H, 1, 1)
    for j in range(len(X)):
        members = idx[off[j]:off[j + 1]]
        assert np.all(H[members, 0] == H[j, 0]) and np.all(np.diff(members) > 0)
        assert len(members) == int(np.sum(H[:, 0] == H[j, 0]))


# ------------------------------------------------------------------ planted mistakes

MUTANTS = {
    "bucket width 2": ("const float v = (s + B[f]) * 0.25f;", "const float v = (s + B[f]) * 0.5f;"),
    "offset dropped": ("const float v = (s + B[f]) * 0.25f;", "const float v = s * 0.25f;"),
    "round instead of floor": ("float f = floorf(v);", "float f = roundf(v);"),
    "all tables instead of any": ("for (int l = 0; l < L && !hit; ++l) {", "hit = 1;\n            for (int l = 0; l < L && hit; ++l) {"),
    "last coordinate dropped": ("for (int64_t k = 0; k < d; ++k) s = fmaf(x[k], a[k], s);",
                                "for (int64_t k = 0; k + 1 < d; ++k) s = fmaf(x[k], a[k], s);"),
}


def _compile(tmp_path, old, new):
    src = open(SRC).read()
    assert old in src
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so), str(path), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    F, I32, I = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    i64 = ctypes.c_int64
    lib.oracle_lsh_hash.argtypes = [F, i64, i64, i64, F, F, I32]
    lib.oracle_lsh_candidates.argtypes = [I32, i64, I32, i64, ctypes.c_int, ctypes.c_int, I, I, i64]
    lib.oracle_lsh_candidates.restype = i64

    def hash_fn(X, A, B):
        X, A, B = (np.ascontiguousarray(v, dtype=np.float32) for v in (X, A, B))
        H = np.empty((X.shape[0], A.shape[0]), dtype=np.int32)
        lib.oracle_lsh_hash(X.ctypes.data_as(F), X.shape[0], X.shape[1], A.shape[0], A.ctypes.data_as(F),
                            B.ctypes.data_as(F), H.ctypes.data_as(I32))
        return H

    def cand_fn(HX, HQ, K, L):
        HX, HQ = np.ascontiguousarray(HX, dtype=np.int32), np.ascontiguousarray(HQ, dtype=np.int32)
        off = np.empty(HQ.shape[0] + 1, dtype=np.int64)
        total = lib.oracle_lsh_candidates(HX.ctypes.data_as(I32), HX.shape[0], HQ.ctypes.data_as(I32), HQ.shape[0],
                                          K, L, off.ctypes.data_as(I), None, 0)
        idx = np.empty(max(total, 1), dtype=np.int64)
        lib.oracle_lsh_candidates(HX.ctypes.data_as(I32), HX.shape[0], HQ.ctypes.data_as(I32), HQ.shape[0],
                                  K, L, off.ctypes.data_as(I), idx.ctypes.data_as(I), total)
        return off, idx[:total]
    return hash_fn, cand_fn


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_every_lsh_mutant_fails_a_pin(tmp_path, name):
    assert not _pins_hold(*_compile(tmp_path, *MUTANTS[name])), f"mutant {name!r} survived"
