"""Stored FP64 oracle values for the n = m = 1000, d = 2 workload (written by
tests/golden/make_golden.py from the oracle alone) and the generator digests."""
import hashlib
import os

import numpy as np

import oracle
from paper_2407_07096_gb300 import datagen as G

GOLD = os.path.join(os.path.dirname(__file__), "golden", "small_f64_d2.txt")


def load_golden():
    digests, vals = {}, []
    with open(GOLD) as f:
        for line in f:
            if line.startswith("# sha256"):
                _, _, name, h = line.split()
                digests[name] = h
            elif not line.startswith("#"):
                vals.append(float(line.split()[1]))
    return digests, np.array(vals)


def test_generator_is_stable():
    digests, _ = load_golden()
    X, Q, _ = G.workload_small_f64(0)
    assert hashlib.sha256(X.tobytes()).hexdigest() == digests["X"]
    assert hashlib.sha256(Q.tobytes()).hexdigest() == digests["Q"]


def test_oracle_matches_stored_values():
    _, want = load_golden()
    X, Q, a = G.workload_small_f64(0)
    got = oracle.kde(X, Q, a)
    # libm exp may differ by an ulp between machines; kappa is small here (d = 2)
    assert np.max(oracle.rel_err(got, want)) < 1e-13
