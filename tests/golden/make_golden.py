"""Writes the stored expected values under tests/golden/ by calling the FP64 oracle.

Run from the repository root: ``python tests/golden/make_golden.py``. Inputs come from
the seeded generator; expected values come from ``oracle/`` alone.

small_f64_d2.txt: the FP64 workload n = m = 1000, d = 2, 3-component mixture with means
in [-5, 5]^2 and std 1, a = 1, seed 0. One line per query: index, K(q) (repr of a
double). The header holds SHA-256 digests of the generated X and Q bytes so that a
change of the generator is caught before the values are compared.
"""
import hashlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2407_07096_gb300 import datagen as G  # noqa: E402


def main():
    X, Q, a = G.workload_small_f64(0)
    K = oracle.kde(X, Q, a)
    path = os.path.join(ROOT, "tests", "golden", "small_f64_d2.txt")
    with open(path, "w") as f:
        f.write("# exact Gaussian KDE, K(q) = sum_i exp(-a ||q - x_i||^2) (Sec. 3), FP64 oracle\n")
        f.write("# workload: n=m=1000 d=2, 3-component mixture means U[-5,5]^2 std 1, a=1, seed 0\n")
        f.write(f"# sha256 X {hashlib.sha256(X.tobytes()).hexdigest()}\n")
        f.write(f"# sha256 Q {hashlib.sha256(Q.tobytes()).hexdigest()}\n")
        for j, v in enumerate(K):
            f.write(f"{j} {float(v)!r}\n")


if __name__ == "__main__":
    main()
