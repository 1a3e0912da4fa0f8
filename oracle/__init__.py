"""FP64 CPU oracle for exact Gaussian KDE.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may use it; the library's product path never imports it, and it
imports nothing from the library. It implements the paper's definition of the
kernel density (Sec. 3) with the Gaussian kernel (Sec. 3) as a plain double loop, the
same for Sec. 3's exponential and logistic kernels, and the weighted subset sums of the
sampling estimators (Sec. 3.1); and the Euclidean LSH of Sec. 2 (hash values and
near-neighbour candidate lists, lsh_oracle.c).
"""
from .kde import (build, kde, kde_weighted, kde_self, kde_log, kde_kernel, kde_subset,  # noqa: F401
                  KERNELS, lsh_hash, lsh_candidates, rel_err, avg_rel_err)
